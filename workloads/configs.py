"""The five seeded workloads of the Helmholtz Krylov path.

C1  small FD box       16^3 7-point operator, kh = 0.5, shift k^2 (1 + 0.05i)
C2  P1 FEM cylinder    nr=40, ntheta=96, nz=160, k=20, impedance ends (~618k unknowns)
C3  large cylinder     nr=60, ntheta=128, nz=256, k=20 (~1.97M unknowns)
C4  frequency sweep    8 geometries x 8 wavenumbers (64 systems of uneven size)
C5  inverse problem    64^3 FD operator A(theta) = -Lap_h - kappa^2 diag(theta)
H1  car cabin          Q1 hexahedra, 27-entry rows (stand-in for the car-cavity matrices)

Seeds (numpy PCG64): C1 b 1001, x* 1002; C2 jitter 2001; C3 jitter 3001;
C4 system s uses 4000 + s; C5 theta field 5001, sample points 5002, data 5003,
directions 5004, right-hand side 5000; BLAS-1 sweep 6001.
"""

import numpy as np

from .csr import CSR, complex_normal
from .fd import fd_helmholtz_box
from .cylinder import cylinder_helmholtz
from .hexcar import hexcar_helmholtz


def c1_small_fd(m: int = 16):
    """C1: returns (A, b_random, x_star, b_manufactured=None).  b = A x* is
    formed by the caller with its own SpMV so that no arithmetic lives here."""
    A = fd_helmholtz_box(m, kh=0.5, damping=0.05)
    b = complex_normal(np.random.default_rng(1001), A.n)
    xs = complex_normal(np.random.default_rng(1002), A.n)
    return A, b, xs


def c2_cylinder(nr: int = 40, ntheta: int = 96, nz: int = 160, k: float = 20.0):
    """C2: jittered P1 cylinder, k = 20, impedance ends, RCM order."""
    return cylinder_helmholtz(nr, ntheta, nz, k=k, jitter=0.2, seed=2001)


def c3_cylinder_large():
    """C3: the C2 operator on a finer grid (~2M unknowns, ~28M nonzeros)."""
    return cylinder_helmholtz(60, 128, 256, k=20.0, jitter=0.2, seed=3001)


# C4 geometries: three FD boxes and five cylinder resolutions
C4_BOXES = (24, 40, 64)
C4_CYLINDERS = ((12, 32, 52), (16, 40, 76), (20, 52, 96), (26, 64, 120), (32, 84, 148))
C4_KH = tuple(np.linspace(0.2, 0.8, 8))


def c4_sweep_systems(boxes=C4_BOXES, cylinders=C4_CYLINDERS, kh_list=C4_KH, damping=0.05):
    """C4: list of (name, A, b) for every geometry x wavenumber, in that order.

    Boxes: -Lap_h - k^2 (1 + 0.05i) I with k = kh/h.  Cylinders: K - k^2
    (1 + 0.05i) M - i k B with k = kh/dz.  System s gets b from seed 4000 + s.
    """
    out = []
    s = 0
    for m in boxes:
        for kh in kh_list:
            A = fd_helmholtz_box(m, kh=float(kh), damping=damping)
            b = complex_normal(np.random.default_rng(4000 + s), A.n)
            out.append((f"box{m}_kh{kh:.3f}", A, b))
            s += 1
    for (nr, nth, nz) in cylinders:
        for kh in kh_list:
            A, _ = cylinder_helmholtz(nr, nth, nz, kh=float(kh), damping=damping,
                                      jitter=0.2, seed=4000 + s)
            b = complex_normal(np.random.default_rng(4000 + s), A.n)
            out.append((f"cyl{nr}x{nth}x{nz}_kh{kh:.3f}", A, b))
            s += 1
    return out


def h1_hexcar(nx: int = 192):
    """H1: Q1 hexahedral car-cabin cavity, kh = 0.5, 0.05 damping; nx = 192
    gives about 684k nodes and 17.8M nonzeros with 27-entry rows, the size of
    the paper's largest car-cavity matrix (649k rows, 15.4M nonzeros)."""
    return hexcar_helmholtz(nx=nx, kh=0.5, damping=0.05)


def smooth_field(m: int, rng: np.random.Generator, sigma: float = 4.0) -> np.ndarray:
    """Gaussian-filtered complex normal field on the m^3 grid, max |f| = 1."""
    from scipy.ndimage import gaussian_filter
    re = gaussian_filter(rng.standard_normal((m, m, m)), sigma, mode="wrap")
    im = gaussian_filter(rng.standard_normal((m, m, m)), sigma, mode="wrap")
    f = (re + 1j * im).reshape(-1)
    return (f / np.max(np.abs(f))).astype(np.complex128)


def c5_inverse_problem(m: int = 64, nsample: int = 512, kh: float = 0.5):
    """C5: returns a dict with the Laplacian part, kappa^2, theta, b, sample
    indices and data.  A(theta) = L - kappa^2 diag(theta) with L = -Lap_h."""
    h = 1.0 / (m + 1)
    kappa = kh / h
    n = m ** 3
    theta = 1.0 + 0.2 * smooth_field(m, np.random.default_rng(5001))
    L = fd_helmholtz_box(m, kh=kh, damping=0.0, diag_shift=np.zeros(n))
    A = fd_helmholtz_box(m, kh=kh, damping=0.0, diag_shift=kappa * kappa * theta)
    idx = np.sort(np.random.default_rng(5002).choice(n, size=min(nsample, n), replace=False))
    d = complex_normal(np.random.default_rng(5003), idx.size)
    b = complex_normal(np.random.default_rng(5000), n)
    return {"m": m, "h": h, "kappa2": kappa * kappa, "theta": theta, "L": L, "A": A,
            "b": b, "sample_idx": idx.astype(np.int64), "data": d}


def c5_directions(n: int, count: int = 20):
    """Seeded complex directions for the finite-difference gradient check."""
    rng = np.random.default_rng(5004)
    return [complex_normal(rng, n) for _ in range(count)]


def blas_sweep_sizes():
    """complex128 vector lengths 1e3 .. 1e8 in half decades."""
    return [int(round(10 ** (3 + 0.5 * i))) for i in range(11)]


def blas_vectors(n: int, count: int = 2):
    rng = np.random.default_rng(6001)
    return [complex_normal(rng, n) for _ in range(count)]


__all__ = ["CSR", "c1_small_fd", "c2_cylinder", "c3_cylinder_large", "c4_sweep_systems",
           "c5_inverse_problem", "c5_directions", "blas_sweep_sizes", "blas_vectors",
           "smooth_field"]
