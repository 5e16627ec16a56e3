"""GPU parity: TFQMR (Section 7's P-TFQMR, preconditioner-free or Jacobi)
through the C ABI, against the CPU oracle and dense LU.  Both sides stop on
the quasi-residual bound sqrt(m+1) tau_m <= tol ||b|| tested once per
iteration, and record that bound as the history."""

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import workloads as W
from tests import _cases as K

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(a).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def true_relres(oracle, A, x, b):
    return oracle.dznrm2(b - oracle.zspmv(A, x)) / oracle.dznrm2(b)


@pytest.mark.parametrize("ff", [False, True])
def test_tfqmr_fd_box_vs_oracle_and_lu(hz, oracle, ff):
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 1001)[0]
    M = hz.Matrix.from_csr(A, ff=ff)
    hist = torch.zeros(2001, dtype=torch.float64, device="cuda")
    x, info = hz.zsolve(M, dev(b), tol=1e-11, maxit=2000, method="tfqmr", hist=hist)
    xo, io = oracle.tfqmr(A, b, tol=1e-11, maxit=2000)
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    assert info.converged and io.status == 0, (info, io.iters)
    assert abs(info.iters - io.iters) <= max(3, 0.1 * io.iters), (info, io.iters)
    xg = host(x)
    assert true_relres(oracle, A, xg, b) <= 1e-11
    assert np.linalg.norm(xg - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
    h = host(hist)
    assert h[0] == 1.0
    assert np.all(np.abs(h[1:6] - io.hist[1:6]) <= 1e-9 * io.hist[1:6])


@pytest.mark.parametrize("variant", [("csr", 4), ("ffflat", 0), ("fftma", 0), ("sell", 0)])
def test_tfqmr_cylinder_variants(hz, oracle, variant):
    A, b = K.small_cylinder()
    M = hz.Matrix.from_csr(A, sell=True, ff=True)
    M.set_spmv(*variant)
    x, info = hz.zsolve(M, dev(b), tol=1e-10, maxit=3000, method="tfqmr")
    xo, io = oracle.tfqmr(A, b, tol=1e-10, maxit=3000)
    assert info.status == io.status == 0
    assert true_relres(oracle, A, host(x), b) <= 1e-10
    assert np.linalg.norm(host(x) - xo) / np.linalg.norm(xo) <= 1e-7


def test_tfqmr_jacobi_and_manufactured(hz, oracle):
    rng = np.random.default_rng(61)
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    As = W.CSR.from_scipy((A.to_scipy() @ sp.diags(rng.uniform(0.01, 100, A.n))).tocsr())
    b = K.vectors(A.n, 62)[0]
    M = hz.Matrix.from_csr(As, ff=True)
    x, info = hz.zsolve(M, dev(b), tol=1e-10, maxit=3000, method="tfqmr", precond="jacobi")
    x_lu = np.linalg.solve(As.to_scipy().toarray(), b)
    assert info.converged and np.linalg.norm(host(x) - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
    A, _, xs = W.c1_small_fd()
    M = hz.Matrix.from_csr(A)
    x, info = hz.zsolve(M, dev(A.to_scipy() @ xs), tol=1e-12, maxit=3000, method="tfqmr")
    assert info.converged and np.linalg.norm(host(x) - xs) <= 1e-8 * np.linalg.norm(xs)


def test_tfqmr_edge_cases(hz, oracle):
    A, b, _ = W.c1_small_fd()
    M = hz.Matrix.from_csr(A, ff=True)
    x, info = hz.zsolve(M, torch.zeros(A.n, dtype=torch.complex128, device="cuda"),
                        x=dev(np.ones(A.n, np.complex128)), method="tfqmr")
    assert info.converged and info.iters == 0 and not host(x).any()
    x, info = hz.zsolve(M, dev(b), maxit=0, method="tfqmr")
    assert info.status == 4 and info.iters == 0 and not host(x).any()
    bn = b.copy()
    bn[0] = np.nan
    assert hz.zsolve(M, dev(bn), method="tfqmr")[1].status == 6
    I = W.CSR.from_scipy(sp.identity(300, dtype=np.complex128, format="csr"))
    bi = K.vectors(300, 63)[0]
    x, info = hz.zsolve(hz.Matrix.from_csr(I, ff=True), dev(bi), tol=1e-10, method="tfqmr")
    assert info.converged and info.iters == 1
    assert np.allclose(host(x), bi, rtol=0, atol=1e-14)
    lam = np.repeat(np.array([1.0 + 0.5j, 3.0 - 1j, 7.0 + 2j]), 40)
    D = W.CSR.from_scipy(sp.diags(lam, format="csr"))
    bd = K.vectors(120, 64)[0]
    x, info = hz.zsolve(hz.Matrix.from_csr(D), dev(bd), tol=1e-13, maxit=50, method="tfqmr")
    assert info.converged and info.iters <= 3
    assert np.linalg.norm(host(x) - bd / lam) <= 1e-12 * np.linalg.norm(bd / lam)
    with pytest.raises(hz.HzError):
        hz.zsolve(M, dev(b), method="tfqmr", mode="mixed")


def test_tfqmr_range_guard_c2(hz, oracle):
    """On the C2 cylinder TFQMR stagnates and its squared-BiCG vectors u, v
    grow geometrically against w.  The binary64 run follows the oracle's
    history; the double-float run follows it too, past the point where its
    vectors leave the binary32 range without the power-of-two rescaling
    (about 70 iterations), and ends cleanly (no NaN) once the spread between
    u and w exceeds what binary32 exponents can hold."""
    A, b = W.c2_cylinder()
    _, io = oracle.tfqmr(A, b, tol=1e-10, maxit=40)
    hists, infos = {}, {}
    for ff, kind in ((False, "csr"), (True, "ffflat")):
        M = hz.Matrix.from_csr(A, ff=ff)
        M.set_spmv(kind, 4)
        hist = torch.zeros(151, dtype=torch.float64, device="cuda")
        x, info = hz.zsolve(M, dev(b), tol=1e-10, maxit=150, method="tfqmr", hist=hist)
        assert info.status in (4, 5) and np.isfinite(info.relres_true) and np.isfinite(host(x)).all(), (kind, info)
        hists[kind], infos[kind] = host(hist), info
        M.close()
    assert infos["csr"].status == 4 and infos["csr"].iters == 150
    assert np.allclose(hists["csr"][:41], io.hist[:41], rtol=1e-9, atol=0)
    k = infos["ffflat"].iters
    assert k > 75
    assert np.allclose(hists["ffflat"][:k + 1], hists["csr"][:k + 1], rtol=1e-6, atol=0)
