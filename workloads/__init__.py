"""Seeded synthetic inputs for the complex Helmholtz Krylov path.

This package only builds problems: matrices in CSR form, right-hand sides and
random vectors.  It holds none of the solver arithmetic (no SpMV, no dot
products, no Krylov steps), so both the CPU oracle and the CUDA path can read
its output without sharing any of the method's code.

The paper (Section 3.1, "Matrices tested") measures on finite-element
Helmholtz matrices from a cylinder and two car cavities that are not
distributed with it; the generators here stand in for them with the same
structure: complex-symmetric, CSR, 7 to 300 nonzeros per row, RCM-ordered.
"""

from .csr import CSR, complex_normal  # noqa: F401
from .fd import fd_helmholtz_box, fd_laplacian_eig  # noqa: F401
from .cylinder import cylinder_helmholtz  # noqa: F401
from .hexcar import hexcar_helmholtz  # noqa: F401
from .configs import (  # noqa: F401
    c1_small_fd, c2_cylinder, c3_cylinder_large, c4_sweep_systems, c5_inverse_problem, h1_hexcar,
    c5_directions, blas_sweep_sizes, blas_vectors,
)
