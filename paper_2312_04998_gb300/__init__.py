"""GB300 (sm_103a) library for the stoichiometry-matrix chemistry hot path.

`binding` wraps the C ABI of include/stoich.h (libstoich.so, built in-tree by
`build.build()`); all computation runs in the library's CUDA kernels.
"""
__all__ = ["binding", "build"]
