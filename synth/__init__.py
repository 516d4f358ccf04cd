"""Seeded synthetic inputs shared by the oracle and the CUDA library.

Holds input generation only (counter-based random streams, network topology
and rate-parameter draws, cell conditions, initial abundances); none of the
method's arithmetic lives here.
"""
