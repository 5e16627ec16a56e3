"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle (oracle/hz_oracle.c) against something other
than itself: the paper's worked CSR example (Section 3.2), brute-force dense
products, closed-form eigenpairs of the finite-difference Laplacian, exact
integer arithmetic, dense LU, constructed breakdowns and finite differences.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from tests import _cases as K


# --------------------------------------------------------------------------- SpMV
def test_worked_example_structure():
    """The CSR arrays of the paper's 5x5 example match its printed pattern
    and the 1-based end marker IA(n+1) = nz + 1 (Section 3.2)."""
    dense, pattern = K.worked_example()
    A = K.worked_example_csr()
    assert A.n == 5 and A.nnz == 11 == len(pattern)
    rows = np.repeat(np.arange(5), np.diff(A.rowptr))
    assert [(int(r) + 1, int(c) + 1) for r, c in zip(rows, A.col)] == pattern
    assert int(A.rowptr[-1]) + 1 == 12
    assert list(A.rowptr) == [0, 2, 4, 6, 9, 11]
    assert list(A.col) == [0, 1, 1, 2, 0, 2, 1, 3, 4, 2, 4]
    assert list(A.val.real) == [3, 14, 8, 1, 2, 6, 4, 2, -1, 9, 7]


def test_worked_example_products(oracle):
    dense, _ = K.worked_example()
    for scale in (1.0, 1 + 2j):
        A = K.worked_example_csr(scale)
        y = oracle.zspmv(A, np.ones(5, dtype=np.complex128))
        assert np.array_equal(y, np.array([17, 9, 8, 5, 16]) * scale)
        for j in range(5):
            e = np.zeros(5, dtype=np.complex128)
            e[j] = 1.0
            assert np.array_equal(oracle.zspmv(A, e), dense[:, j] * scale)


@pytest.mark.parametrize("seed,n", [(1, 1), (2, 17), (3, 300), (4, 999)])
def test_spmv_brute_force_dense(oracle, seed, n):
    A = K.random_csr(n, seed, max_row=30, long_rows=(n,) if n > 100 else ())
    x = K.vectors(n, seed + 10)[0]
    ref = A.to_scipy().toarray() @ x
    assert np.all(np.abs(oracle.zspmv(A, x) - ref) <= 1e-13 * K.row_abs_scale(A, x) + 1e-300)


def test_cspmv_brute_force_dense(oracle):
    """complex64 product with binary32 sums against the exact product of the
    same rounded data (binary32 error bound ~ row length * 2^-24)."""
    A = K.random_csr(400, 21, max_row=30, long_rows=(300,))
    x = K.vectors(400, 22)[0].astype(np.complex64)
    a32 = A.val.astype(np.complex64)
    exact = sp.csr_matrix((a32.astype(np.complex128), A.col, A.rowptr), shape=(400, 400)) @ x.astype(np.complex128)
    got = oracle.cspmv(A, x, val32=a32)
    scale = sp.csr_matrix((np.abs(a32).astype(np.float64), A.col, A.rowptr), shape=(400, 400)) @ np.abs(x)
    lens = np.diff(A.rowptr)
    assert np.all(np.abs(got - exact) <= (lens + 2) * 2.0 ** -23 * scale + 1e-30)
    assert np.any(np.abs(got - exact) > 0)        # really binary32 arithmetic


def test_spmv_complex_symmetry_invariant(oracle):
    """Helmholtz matrices are complex symmetric: u^T (A v) = v^T (A u)."""
    for A in (W.c1_small_fd()[0], K.small_cylinder()[0]):
        u, v = K.vectors(A.n, 33)
        lhs = np.sum(u * oracle.zspmv(A, v))
        rhs = np.sum(v * oracle.zspmv(A, u))
        assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(u) * K.row_abs_scale(A, v))
        S = A.to_scipy()
        assert abs(S - S.T).max() <= 1e-14 * abs(S).max()


def test_fd_closed_form_eigenpairs(oracle):
    """-Lap_h v = lambda v for the sine modes; A v = (lambda - k^2(1+0.05i)) v."""
    A, _, _ = W.c1_small_fd()
    m, k = 16, 8.5
    assert abs(A.meta["k"] - k) < 1e-12
    shift = k * k * (1 + 0.05j)
    for (a, b, c) in ((1, 1, 1), (3, 5, 7), (16, 16, 16), (2, 9, 1)):
        lam, v = W.fd_laplacian_eig(m, a, b, c)
        mu = lam - shift
        assert np.allclose(oracle.zspmv(A, v), mu * v, rtol=0, atol=1e-10 * abs(lam))
    lam_min, _ = W.fd_laplacian_eig(m, 1, 1, 1)
    lam_max, _ = W.fd_laplacian_eig(m, 16, 16, 16)
    assert abs(lam_min - 29.52) < 0.01 and abs(lam_max - 3438.5) < 0.1   # derived: C1 spectrum


def test_fd_closed_form_solve(oracle):
    A, _, _ = W.c1_small_fd()
    lam, v = W.fd_laplacian_eig(16, 2, 3, 4)
    mu = lam - 72.25 * (1 + 0.05j)
    x, info = oracle.bicgstab(A, v, tol=1e-12, maxit=500)
    assert info.status == 0
    assert np.linalg.norm(x - v / mu) <= 1e-10 * np.linalg.norm(v / mu)


# --------------------------------------------------------------------------- FEM generator invariants
def test_cylinder_fem_invariants():
    nr, nth, nz, R, L = 6, 16, 20, 1.0, 4.0
    A, b, parts = W.cylinder_helmholtz(nr, nth, nz, kh=0.5, damping=0.05, jitter=0.2, seed=7,
                                       rcm=False, return_parts=True)
    Kst, M, B, xyz = parts["K"], parts["M"], parts["B"], parts["xyz"]
    one = np.ones(Kst.shape[0])
    assert np.abs(Kst @ one).max() < 1e-10 * abs(Kst).max()                  # K 1 = 0
    vol = 0.5 * nth * np.sin(2 * np.pi / nth) * R * R * L                     # polygonal cylinder
    assert abs(one @ (M @ one) - vol) < 1e-10 * vol                           # jitter keeps volume
    area = 0.5 * nth * np.sin(2 * np.pi / nth) * R * R
    assert abs(one @ (B @ one) - 2 * area) < 1e-10 * area                      # two end faces
    assert abs(Kst - Kst.T).max() < 1e-12 * abs(Kst).max()
    # linear fields are in the P1 space: K u = 0 away from the boundary
    u = 0.3 * xyz[:, 0] - 1.1 * xyz[:, 1] + 0.7 * xyz[:, 2]
    r = np.hypot(xyz[:, 0], xyz[:, 1])
    per = 1 + nr * nth
    k = np.arange(xyz.shape[0]) // per
    loc = np.arange(xyz.shape[0]) % per
    ring = np.where(loc == 0, 0, (loc - 1) // nth + 1)
    interior = (ring < nr) & (k > 0) & (k < nz)
    assert np.abs((Kst @ u)[interior]).max() < 1e-10 * abs(Kst).max()
    assert r.max() <= R + 1e-12


def test_hexcar_q1_invariants():
    """The Q1 car-cabin generator: rigid-body and volume identities of the
    stiffness and mass, the impedance area, symmetry, 27-entry rows, and the
    Q1 discrete Laplacian reproducing linear fields in the interior."""
    from workloads import hexcar as H
    Kr, Mr = H.q1_reference()
    assert np.allclose(Kr.sum(axis=1), 0, atol=1e-15) and abs(Mr.sum() - 1.0) < 1e-15
    assert np.sum(np.linalg.eigvalsh(Kr) < 1e-12) == 1                       # only constants in the null space
    A, b, P = H.hexcar_helmholtz(nx=40, rcm=False, return_parts=True)
    K, M, B, xyz, h = P["K"], P["M"], P["B"], P["xyz"], A.meta["h"]
    one = np.ones(K.shape[0])
    assert np.abs(K @ one).max() < 1e-12 * abs(K).max()
    assert abs(one @ (M @ one) - P["volume"]) < 1e-12 * P["volume"]
    faces = (one @ (B @ one)) / (h * h)
    assert faces > 0 and abs(faces - round(faces)) < 1e-9                       # whole seat faces
    S = A.to_scipy()
    assert abs(S - S.T).max() == 0
    lens = A.row_lengths()
    assert lens.max() == 27 and np.mean(lens == 27) > 0.5
    u = 0.3 * xyz[:, 0] - 1.1 * xyz[:, 1] + 0.7 * xyz[:, 2]
    full = lens == 27                                                       # nodes with all 8 cubes present
    assert np.abs((K @ u)[full]).max() < 1e-10 * abs(K).max()
    # the cut-outs: the cabin holds less air than its bounding box
    assert P["volume"] < 0.9 * (40 * h) * (round(1.8 / h) * h) * (round(1.3 / h) * h)


# --------------------------------------------------------------------------- BLAS-1
def test_blas1_closed_forms(oracle):
    n = 4096
    phi = np.random.default_rng(5).uniform(0, 2 * np.pi, n)
    x = np.exp(1j * phi)
    assert abs(oracle.dznrm2(x) ** 2 - n) < 1e-11 * n
    d = oracle.zdotc(x, x)
    assert abs(d - n) < 1e-11 * n and d.imag == 0.0
    one = np.ones(n, dtype=np.complex128)
    assert oracle.zdotc((1 + 1j) * one, (2 - 1j) * one) == n * (1 - 3j)
    assert oracle.zdotu((1 + 1j) * one, (2 - 1j) * one) == n * (3 + 1j)
    u, v = K.vectors(n, 8)
    assert abs(oracle.zdotc(u, v) - oracle.zdotu(np.conj(u), v)) <= 1e-13 * np.sum(np.abs(u * v))
    assert abs(oracle.zdotc(u, v) - np.conj(oracle.zdotc(v, u))) <= 1e-13 * np.sum(np.abs(u * v))


def test_blas1_exact_integer_data(oracle):
    rng = np.random.default_rng(6)
    x = rng.integers(-50, 50, 1000) + 1j * rng.integers(-50, 50, 1000)
    y = rng.integers(-50, 50, 1000) + 1j * rng.integers(-50, 50, 1000)
    a = 3 - 2j
    assert np.array_equal(oracle.zaxpy(a, x, y), a * x + y)
    assert np.array_equal(oracle.zscal(a, x), a * x)
    assert np.array_equal(oracle.zcopy(x), x)
    assert oracle.zdotc(x, y) == np.vdot(x, y)
    assert oracle.zdotu(x, y) == np.sum(x * y)


# --------------------------------------------------------------------------- BiCGStab
def test_bicgstab_dense_lu_8cubed(oracle):
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 1001)[0]
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    x, info = oracle.bicgstab(A, b, tol=1e-10, maxit=2000)
    assert info.status == 0 and info.relres_true <= 1e-10
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= 1e-8
    assert info.hist[0] == 1.0 and info.hist[-1] <= 1e-10


def test_bicgstab_general_nonsymmetric_dense_lu(oracle):
    """The iteration itself does not rely on symmetry: a random diagonally
    dominant complex matrix against dense LU."""
    A = K.random_csr(200, 12, max_row=10)
    S = A.to_scipy().tolil()
    S.setdiag(S.diagonal() + 12.0 + 3j)
    A = W.CSR.from_scipy(S.tocsr())
    b = K.vectors(200, 13)[0]
    x, info = oracle.bicgstab(A, b, tol=1e-12, maxit=500)
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    assert info.status == 0
    assert np.linalg.norm(x - x_lu) <= 1e-10 * np.linalg.norm(x_lu)


def test_bicgstab_manufactured(oracle):
    A, _, xs = W.c1_small_fd()
    b = A.to_scipy() @ xs
    x, info = oracle.bicgstab(A, b, tol=1e-12, maxit=2000)
    assert info.status == 0 and np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8


def test_bicgstab_identity_half_step(oracle):
    """A = I: one step, exact half-step exit with x = b."""
    A = W.CSR.from_scipy(sp.identity(50, dtype=np.complex128, format="csr"))
    b = K.vectors(50, 2)[0]
    x, info = oracle.bicgstab(A, b, tol=1e-10)
    assert info.status == 0 and info.iters == 1 and np.array_equal(x, b)


def test_bicgstab_special_cases(oracle):
    A, b, _ = W.c1_small_fd()
    x, info = oracle.bicgstab(A, np.zeros(A.n, np.complex128), x0=np.ones(A.n))
    assert info.status == 0 and info.iters == 0 and not x.any()
    x, info = oracle.bicgstab(A, b, maxit=0)
    assert info.status == 4 and info.iters == 0 and not x.any()
    x, info = oracle.bicgstab(K.breakdown_2x2(), np.array([1, 0], dtype=np.complex128))
    assert info.status == 5 and info.iters == 1
    bn = b.copy()
    bn[0] = np.nan
    x, info = oracle.bicgstab(A, bn)
    assert info.status == 6


# --------------------------------------------------------------------------- Jacobi
def test_zmul_elementwise_exact(oracle):
    """Section 5's element-wise product on small integers: exact."""
    rng = np.random.default_rng(31)
    x = rng.integers(-9, 10, 40) + 1j * rng.integers(-9, 10, 40)
    y = rng.integers(-9, 10, 40) + 1j * rng.integers(-9, 10, 40)
    assert np.array_equal(oracle.zmul_elementwise(x, y), x * y)


def test_jacobi_dinv_rule(oracle):
    """1 / (sum of the diagonal entries of the row); 1 where there is none or it is 0."""
    S = sp.lil_matrix((4, 4), dtype=np.complex128)
    S[0, 0] = 2 + 2j
    S[0, 1] = 5
    S[1, 0] = 1            # row 1 has no diagonal
    S[2, 2] = 0.0          # explicit zero
    S[3, 3] = 4.0
    A = W.CSR.from_scipy(S.tocsr())
    A.col = A.col.copy()
    d = oracle.jacobi_dinv(A)
    assert np.allclose(d, [1 / (2 + 2j), 1, 1, 0.25], rtol=1e-15, atol=0)
    # a diagonal split over two stored entries is summed
    rp = np.array([0, 2], dtype=np.int32)
    A2 = W.CSR(1, rp, np.array([0, 0], dtype=np.int32), np.array([1 + 1j, 3 - 1j]))
    assert oracle.jacobi_dinv(A2)[0] == 0.25


def test_jacobi_diagonal_matrix_one_step(oracle):
    """A = D: the right-preconditioned operator is I, so the first half step
    exits with x = D^-1 b (closed form)."""
    rng = np.random.default_rng(32)
    dvals = rng.uniform(0.5, 4, 60) * np.exp(1j * rng.uniform(0, 2 * np.pi, 60))
    A = W.CSR.from_scipy(sp.diags(dvals, format="csr").astype(np.complex128))
    b = K.vectors(60, 33)[0]
    x, info = oracle.bicgstab(A, b, tol=1e-12, precond="jacobi")
    assert info.status == 0 and info.iters == 1
    assert np.allclose(x, b / dvals, rtol=1e-14, atol=0)
    # without the preconditioner the same system needs many iterations
    _, info0 = oracle.bicgstab(A, b, tol=1e-12)
    assert info0.iters > 5


def test_jacobi_unit_diagonal_is_unpreconditioned(oracle):
    """With a_ii = 1 for every row, D^-1 = I and the preconditioned iteration
    is the plain one: identical histories and solutions."""
    A = W.fd_helmholtz_box(6, kh=0.5, damping=0.05)
    S = A.to_scipy()
    Dinv = sp.diags(1.0 / S.diagonal())
    A1 = W.CSR.from_scipy((Dinv @ S).tocsr())     # row-scaled: unit diagonal
    b = K.vectors(A1.n, 34)[0]
    x0, i0 = oracle.bicgstab(A1, b, tol=1e-10)
    x1, i1 = oracle.bicgstab(A1, b, tol=1e-10, precond="jacobi")
    assert i0.iters == i1.iters and np.array_equal(i0.hist, i1.hist) and np.array_equal(x0, x1)


def test_jacobi_dense_lu_and_column_scaling_invariance(oracle):
    """Against dense LU; and scaling the columns of A by S leaves the Jacobi
    operator A S (D S)^-1 = A D^-1 unchanged, so the iteration matches the
    unscaled one and the solution maps back as x_scaled = S^-1 x."""
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 35)[0]
    x, info = oracle.bicgstab(A, b, tol=1e-11, precond="jacobi")
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    assert info.status == 0 and np.linalg.norm(x - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
    rng = np.random.default_rng(36)
    sc = rng.uniform(0.01, 100, A.n) * np.exp(1j * rng.uniform(0, 2 * np.pi, A.n))
    As = W.CSR.from_scipy((A.to_scipy() @ sp.diags(sc)).tocsr())
    xs, infs = oracle.bicgstab(As, b, tol=1e-11, precond="jacobi")
    assert abs(infs.iters - info.iters) <= 1
    n = min(len(info.hist), len(infs.hist), 10)
    assert np.allclose(infs.hist[:n], info.hist[:n], rtol=1e-9, atol=0)
    assert np.linalg.norm(sc * xs - x) <= 1e-8 * np.linalg.norm(x)
    # the unpreconditioned solver sees the scaling: it needs many more iterations
    _, i0 = oracle.bicgstab(As, b, tol=1e-11, maxit=3000)
    assert i0.iters > 2 * infs.iters


# --------------------------------------------------------------------------- BiCGStab(l)
def test_bicgstabl_ell1_is_bicgstab(oracle):
    """BiCGStab(1) is BiCGStab in exact arithmetic (Sleijpen and Fokkema):
    the same residual history and solution up to rounding."""
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 1001)[0]
    x0, i0 = oracle.bicgstab(A, b, tol=1e-10)
    x1, i1 = oracle.bicgstabl(A, b, ell=1, tol=1e-10)
    assert i1.status == 0 and abs(i1.iters - i0.iters) <= 2
    assert np.allclose(i1.hist[:12], i0.hist[:12], rtol=1e-11, atol=0)
    assert np.linalg.norm(x1 - x0) <= 1e-8 * np.linalg.norm(x0)


@pytest.mark.parametrize("ell", [2, 4, 8])
def test_bicgstabl_dense_lu(oracle, ell):
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 1001)[0]
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    x, info = oracle.bicgstabl(A, b, ell=ell, tol=1e-11, maxit=2000)
    assert info.status == 0 and info.relres_true <= 1e-11
    assert np.linalg.norm(x - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
    assert info.hist[0] == 1.0


def test_bicgstabl_identity_and_special_cases(oracle):
    A = W.CSR.from_scipy(sp.identity(50, dtype=np.complex128, format="csr"))
    b = K.vectors(50, 2)[0]
    x, info = oracle.bicgstabl(A, b, ell=4, tol=1e-10)
    assert info.status == 0 and info.iters == 1 and np.array_equal(x, b)
    A, b, xs = W.c1_small_fd()
    x, info = oracle.bicgstabl(A, A.to_scipy() @ xs, ell=4, tol=1e-12)
    assert info.status == 0 and np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    x, info = oracle.bicgstabl(A, np.zeros(A.n, np.complex128), ell=2, x0=np.ones(A.n))
    assert info.status == 0 and info.iters == 0 and not x.any()
    x, info = oracle.bicgstabl(A, b, ell=2, maxit=0)
    assert info.status == 4 and info.iters == 0 and not x.any()
    bn = b.copy()
    bn[0] = np.nan
    assert oracle.bicgstabl(A, bn, ell=2)[1].status == 6
    with pytest.raises(ValueError):
        oracle.bicgstabl(A, b, ell=9)


def test_bicgstabl_beats_stagnation(oracle):
    """On the small jittered cylinder the minimal-residual steps of l = 4
    converge in fewer BiCG steps than BiCGStab needs iterations."""
    A, b = K.small_cylinder()
    _, i0 = oracle.bicgstab(A, b, tol=1e-10, maxit=3000)
    x4, i4 = oracle.bicgstabl(A, b, ell=4, tol=1e-10, maxit=3000)
    assert i4.status == 0 and i4.relres_true <= 1e-10
    assert i4.iters < i0.iters


# --------------------------------------------------------------------------- TFQMR
def test_tfqmr_dense_lu_and_manufactured(oracle):
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 1001)[0]
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    x, info = oracle.tfqmr(A, b, tol=1e-11, maxit=2000)
    assert info.status == 0 and info.relres_true <= 1e-11
    assert np.linalg.norm(x - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
    # the quasi-residual bound sqrt(m+1) tau_m is never below the true residual
    assert info.hist[0] == 1.0 and info.relres_true <= info.hist[-1]
    A, _, xs = W.c1_small_fd()
    x, info = oracle.tfqmr(A, A.to_scipy() @ xs, tol=1e-12, maxit=2000)
    assert info.status == 0 and np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)


def test_tfqmr_finite_termination(oracle):
    """A = I ends after one iteration with x = b; a diagonal matrix with three
    distinct eigenvalues is solved to rounding level within three iterations
    (the squared BiCG polynomial of degree 3 annihilates the spectrum)."""
    I = W.CSR.from_scipy(sp.identity(50, dtype=np.complex128, format="csr"))
    b = K.vectors(50, 2)[0]
    x, info = oracle.tfqmr(I, b, tol=1e-10)
    assert info.status == 0 and info.iters == 1 and np.array_equal(x, b)
    lam = np.repeat(np.array([1.0 + 0.5j, 3.0 - 1j, 7.0 + 2j]), 20)
    D = W.CSR.from_scipy(sp.diags(lam, format="csr"))
    b = K.vectors(60, 3)[0]
    x, info = oracle.tfqmr(D, b, tol=1e-13, maxit=50)
    assert info.status == 0 and info.iters <= 3
    assert np.linalg.norm(x - b / lam) <= 1e-12 * np.linalg.norm(b / lam)


def test_tfqmr_special_cases(oracle):
    A, b, _ = W.c1_small_fd()
    x, info = oracle.tfqmr(A, np.zeros(A.n, np.complex128), x0=np.ones(A.n))
    assert info.status == 0 and info.iters == 0 and not x.any()
    x, info = oracle.tfqmr(A, b, maxit=0)
    assert info.status == 4 and info.iters == 0 and not x.any()
    bn = b.copy()
    bn[0] = np.nan
    assert oracle.tfqmr(A, bn)[1].status == 6


def test_mixed_refinement(oracle):
    A, b, _ = W.c1_small_fd()
    x, d = oracle.refine_mixed(A, b, tol=1e-10)
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    assert d["status"] == 0 and d["relres"] <= 1e-10 and d["outer"] >= 2
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= 1e-8
    # the inner solve alone stops near single precision
    x32, it, st = oracle.cbicgstab(A, b.astype(np.complex64), tol=1e-5)
    r = np.linalg.norm(b - A.to_scipy() @ x32.astype(np.complex128)) / np.linalg.norm(b)
    assert 1e-8 < r < 1e-4


def test_cbicgstab_history_tracks_binary64(oracle):
    """The complex64 inner solver takes the same steps as the binary64
    BiCGStab (Section 7 with the Hermitian inner product): on a well
    conditioned damped FD box with a complex right-hand side, its first ten
    recursive residuals agree with or_bicgstab's to 1e-5 relative, the
    binary32 rounding being the only difference.  A dropped conjugate in its
    inner product, a swapped operand or a wrong sign of omega changes the
    very first steps (rho = <r, r> is real only with the conjugate)."""
    A = W.fd_helmholtz_box(8, kh=0.3, damping=1.0)
    b = K.vectors(A.n, 60)[0]
    _, info = oracle.bicgstab(A, b, tol=1e-12, maxit=200)
    _, it, st, h32 = oracle.cbicgstab(A, b.astype(np.complex64), tol=1e-7, maxit=10, history=True)
    assert it == 10 and info.iters > 10
    h64 = info.hist[:11]
    assert h32[0] == 1.0 and h64[0] == 1.0
    assert np.all(np.abs(h32 - h64) <= 1e-5 * h64)


def test_cbicgstab_nonsymmetric_dense_lu(oracle):
    """complex64 BiCGStab on a general (non-symmetric, non-Hermitian)
    complex matrix reaches the dense-LU solution to binary32 accuracy."""
    rng = np.random.default_rng(61)
    n = 60
    D = ((rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2 * n)
         + np.diag(2.0 + 1.0j + 0.5 * rng.standard_normal(n)))
    A = W.CSR.from_scipy(sp.csr_matrix(D))
    b = K.vectors(n, 62)[0]
    x, it, st = oracle.cbicgstab(A, b.astype(np.complex64), tol=1e-6, maxit=200)
    x_lu = np.linalg.solve(D, b)
    assert st == 0 and it < 200
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= 1e-5


def test_mixed_refinement_returns_best_iterate(oracle):
    """Refinement to a tolerance below binary64 rounding (1e-17) cannot
    converge: once a step fails to reduce the outer residual the refinement
    stops and returns the iterate with the smallest one.  The returned x has
    exactly the reported residual (not the larger one of the last step) and
    is the dense-LU solution to binary64 accuracy."""
    A, b, _ = W.c1_small_fd()
    S = A.to_scipy()
    x, d = oracle.refine_mixed(A, b, tol=1e-17, max_outer=30)
    assert d["status"] == 4 and 2 <= d["outer"] < 30
    r = np.linalg.norm(b - S @ x) / np.linalg.norm(b)
    assert abs(r - d["relres"]) <= 1e-6 * r and r < 1e-12
    x_lu = np.linalg.solve(S.toarray(), b)
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= 1e-10
    # a right-hand side the inner solve cannot improve returns x0 = 0
    rng = np.random.default_rng(63)
    n = 40
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    D = Q1 @ np.diag(np.logspace(0, -8, n)) @ Q2.conj().T
    Ad = W.CSR.from_scipy(sp.csr_matrix(D))
    bd = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xd, dd = oracle.refine_mixed(Ad, bd, tol=1e-12, max_outer=30)
    assert dd["status"] == 4 and dd["relres"] == 1.0 and not xd.any()


# --------------------------------------------------------------------------- adjoint
def test_adjoint_oracle_gradient(oracle):
    """Oracle chain (solve, adjoint solve, outer product on the pattern) against
    the dense-LU gradient and central differences of the loss."""
    m = 6
    A = W.fd_helmholtz_box(m, kh=0.5, damping=0.05)
    n = A.n
    b = K.vectors(n, 50)[0]
    idx = np.arange(0, n, 7)
    d = K.vectors(idx.size, 51)[0]
    S = A.to_scipy().toarray()

    def loss_dense(Sm):
        x = np.linalg.solve(Sm, b)
        return float(np.sum(np.abs(x[idx] - d) ** 2)), x

    L0, x_lu = loss_dense(S)
    x, _ = oracle.bicgstab(A, b, tol=1e-13, maxit=5000)
    g = np.zeros(n, dtype=np.complex128)
    g[idx] = 2 * (x[idx] - d)
    mu, info = oracle.bicgstab(A, np.conj(g), tol=1e-13, maxit=5000)
    grad_val = oracle.outer_on_pattern(A, mu, x)
    lam = np.linalg.solve(S.conj().T, g)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    grad_lu = -lam[rows] * np.conj(x_lu[A.col])
    assert np.linalg.norm(grad_val - grad_lu) <= 1e-8 * np.linalg.norm(grad_lu)
    # central differences along random directions on the stored entries
    rng = np.random.default_rng(52)
    eps = 1e-4   # the directional derivatives here are ~1e-5 of the loss: keep FD round-off small
    for _ in range(3):
        v = rng.standard_normal(A.nnz) + 1j * rng.standard_normal(A.nnz)
        dA = sp.csr_matrix((v, A.col, A.rowptr), shape=(n, n)).toarray()
        fd = (loss_dense(S + eps * dA)[0] - loss_dense(S - eps * dA)[0]) / (2 * eps)
        an = float(np.real(np.vdot(grad_val, v)))
        assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-12)   # FD round-off ~ eps_mach L / eps


def test_openmp_oracle_is_thread_count_invariant(oracle):
    """The all-cores CPU baseline runs the oracle built with OpenMP.  Its
    reductions sum fixed chunks of 8192 elements and add the chunk totals in
    order, so any thread count gives the same iterates bit for bit.  Its
    solution is the plain build's up to the rounding of the chunked sums:
    both reach the tolerance, and the solutions agree to 1e-8 relative (the
    two differ by at most about 2 cond(A) tol).  13,824 unknowns span two
    chunks."""
    A = W.fd_helmholtz_box(24, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 7)[0]
    runs = [oracle.bicgstab_omp(A, b, tol=1e-10, maxit=2000, threads=t) for t in (1, 3, 4)]
    for x, info in runs:
        assert info.status == 0 and info.relres_true <= 1e-10
        assert np.array_equal(x, runs[0][0]) and info.iters == runs[0][1].iters
    xs, info_s = oracle.bicgstab(A, b, tol=1e-10, maxit=2000)[:2]
    assert info_s.status == 0 and info_s.relres_true <= 1e-10
    assert np.linalg.norm(xs - runs[0][0]) <= 1e-8 * np.linalg.norm(xs)
