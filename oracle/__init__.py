"""Plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The product path (the CUDA
library under ``paper_1707_08900_gb300/``) never imports it, and the two
share no code: the only thing both sides see is the seeded input generator
module, which holds none of the method's arithmetic.

``oracle.fd`` wraps the C oracle (``fd_oracle.c``): derivative operators
(Eqs. 6-8), the right-hand side of Eqs. 1-3, the 2N-storage RK3 substep in
the 55-point single-pass form (Eq. 10, Algorithm 2) and the 19-point
two-pass form (Eqs. 14-16, Algorithm 3), FP64 diagnostics and the box
filter.  ``oracle.cnn`` holds the FP64 NumPy reference of the coarse-grid
correction network.
"""
