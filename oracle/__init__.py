"""CPU oracle for the stoichiometry-matrix method (test infrastructure only).

Plain, slow, FP64 NumPy restatements of what the paper's method computes:
dense stoichiometry matrix and the four storage formats (Section 2, Eq. 7,
Listings 1-4), row reorderings (Section 3), rate coefficients, the right-hand
side dn/dt = S.R, its analytic Jacobian, a variable-order BDF integrator with
Newton iterations (the DLSODES role of Section 3) and its discrete adjoint.

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA library:
both sides receive the same input arrays from `synth` and nothing else.
"""
