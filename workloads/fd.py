"""7-point finite-difference Helmholtz operator on the unit cube.

Section 2 of the paper states the problem as -lap(u) - k^2 u = g with Dirichlet
conditions on part of the boundary.  On an m^3 interior grid of the unit cube
with h = 1/(m+1) and homogeneous Dirichlet data on the whole boundary, the
discrete operator is

    A = -Lap_h - shift * I,         shift = k^2 (1 + i*damping),

with -Lap_h u_{abc} = (6 u_{abc} - sum of the 6 neighbours) / h^2.  A is
complex symmetric (A = A^T) but not Hermitian.  A per-unknown shift may be
given instead of a scalar one (the inverse-problem workload uses
shift_i = kappa^2 * theta_i).
"""

import numpy as np
import scipy.sparse as sp

from .csr import CSR


def _lap1d(m: int, h: float):
    e = np.ones(m)
    return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], shape=(m, m)) / (h * h)


def fd_laplacian(m: int) -> sp.csr_matrix:
    """-Lap_h on the m^3 interior grid, lexicographic order (x fastest)."""
    h = 1.0 / (m + 1)
    t = _lap1d(m, h)
    i = sp.identity(m, format="csr")
    lap = sp.kron(sp.kron(i, i), t) + sp.kron(sp.kron(i, t), i) + sp.kron(sp.kron(t, i), i)
    return sp.csr_matrix(lap)


def fd_helmholtz_box(m: int, kh: float = 0.5, damping: float = 0.05, diag_shift=None) -> CSR:
    """A = -Lap_h - k^2 (1 + i*damping) I on the m^3 interior grid, k = kh/h.

    If ``diag_shift`` (complex array of length m^3) is given it replaces the
    scalar shift: A = -Lap_h - diag(diag_shift).
    """
    h = 1.0 / (m + 1)
    k = kh / h
    lap = fd_laplacian(m).astype(np.complex128)
    n = m ** 3
    if diag_shift is None:
        shift = np.full(n, k * k * (1.0 + 1j * damping), dtype=np.complex128)
    else:
        shift = np.asarray(diag_shift, dtype=np.complex128)
    a = lap - sp.diags(shift, 0, shape=(n, n), format="csr")
    return CSR.from_scipy(a, meta={"kind": "fd_box", "m": m, "h": h, "k": k,
                                   "kh": kh, "damping": damping})


def fd_laplacian_eig(m: int, a: int, b: int, c: int):
    """Closed-form eigenpair of -Lap_h on the m^3 interior grid.

    v(i,j,l) = sin(a pi i h) sin(b pi j h) sin(c pi l h), 1 <= a,b,c <= m, is an
    eigenvector with eigenvalue (4/h^2) * sum of sin^2(q pi h / 2) over q in
    (a, b, c).  Returns (eigenvalue, v) with v in the generator's ordering.
    """
    h = 1.0 / (m + 1)
    g = np.arange(1, m + 1) * h
    sx = np.sin(a * np.pi * g)
    sy = np.sin(b * np.pi * g)
    sz = np.sin(c * np.pi * g)
    v = (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]).reshape(-1)
    lam = (4.0 / (h * h)) * sum(np.sin(q * np.pi * h / 2.0) ** 2 for q in (a, b, c))
    return float(lam), v.astype(np.complex128)
