"""GB300-native complex Helmholtz Krylov solver.

The hot path of Cheik Ahamed & Magoules, "Accelerated solution of Helmholtz
equation with Iterative Krylov Methods on GPU": complex128 CSR / SELL-C-sigma
SpMV (Section 6), complex BLAS-1 (Section 5) and BiCGStab (Section 7,
preconditioner-free or Jacobi), as hand-written sm_103a CUDA kernels behind the C ABI of
include/hz.h (libhz.so), with a mixed-precision refinement solver, a batched
persistent sweep solver and an adjoint backward.

``import paper_2112_06465_gb300`` loads libhz.so and raises ImportError if
it has not been built: there is no CPU path.
"""

from .hz import (  # noqa: F401
    Matrix, SolveInfo, HzError, cspmv, diag_grad, dznrm2, mat_set_diag, outer_on_pattern,
    version, zaxpy, zconj, zcopy, zdotc, zdotu, zmul_elementwise, zscal, zsolve, zsolve_batched, zspmv,
)
from .adjoint import DiagParamSolve, ValuesSolve, solve_diag_param, solve_values  # noqa: F401
