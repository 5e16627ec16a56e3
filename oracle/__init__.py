"""CPU oracle for the complex Helmholtz Krylov path -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product library never does, and the two share no
code: the oracle is plain C (``hz_oracle.c``) plus this ctypes wrapper.

What pins each function to the paper and to mathematics, independently of
itself, is in ``tests/test_oracle_pins.py`` (one or more tests per function).
"""

from .oracle import (  # noqa: F401
    build, load, zspmv, cspmv, zdotc, zdotu, dznrm2, zaxpy, zscal, zcopy,
    bicgstab, cbicgstab, refine_mixed, outer_on_pattern, OracleInfo, jacobi_dinv, zmul_elementwise, bicgstabl, tfqmr,
    build_omp, bicgstab_omp,
)
