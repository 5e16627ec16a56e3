"""GPU parity: BiCGStab(l) (Section 7's P-BiCGSTAB(l), preconditioner-free
or Jacobi) through the C ABI, against the CPU oracle (modified Gram-Schmidt
minimal-residual step; the GPU solves the Gram normal equations) and dense
LU.  Iterations are counted in BiCG steps on both sides."""

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


@pytest.mark.parametrize("ell", [1, 2, 4, 8])
@pytest.mark.parametrize("ff", [False, True])
def test_bicgstabl_fd_box_vs_oracle_and_lu(hz, oracle, ell, ff):
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 1001)[0]
    M = hz.Matrix.from_csr(A, ff=ff)
    hist = torch.zeros(2000 + ell, dtype=torch.float64, device="cuda")
    x, info = hz.zsolve(M, dev(b), tol=1e-11, maxit=1999, method="bicgstabl", ell=ell, hist=hist)
    xo, io = oracle.bicgstabl(A, b, ell=ell, tol=1e-11, maxit=1999)
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    assert info.converged and io.status == 0, (info, io.iters, io.status)
    assert abs(info.iters - io.iters) <= max(2 * ell, 0.1 * io.iters), (info, io.iters)
    xg = host(x)
    assert true_relres(oracle, A, xg, b) <= 1e-11
    assert np.linalg.norm(xg - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
    h = host(hist)
    assert h[0] == 1.0
    k = min(5, io.iters - 1)
    assert np.all(np.abs(h[1:k + 1] - io.hist[1:k + 1]) <= 1e-9 * io.hist[1:k + 1])


def test_bicgstabl_ell1_matches_bicgstab(hz, oracle):
    """BiCGStab(1) is BiCGStab: its GPU history follows the oracle's BiCGStab."""
    A, b, _ = W.c1_small_fd()
    M = hz.Matrix.from_csr(A, ff=True)
    hist = torch.zeros(2001, dtype=torch.float64, device="cuda")
    x, info = hz.zsolve(M, dev(b), tol=1e-10, maxit=2000, method="bicgstabl", ell=1, hist=hist)
    _, io = oracle.bicgstab(A, b, tol=1e-10, maxit=2000)
    assert info.converged
    assert np.all(np.abs(host(hist)[1:11] - io.hist[1:11]) <= 1e-9 * io.hist[1:11])


@pytest.mark.parametrize("variant", [("csr", 4), ("ffflat", 0), ("fftma", 0), ("sell", 0), ("sellff", 0)])
def test_bicgstabl_cylinder_variants(hz, oracle, variant):
    A, b = K.small_cylinder()
    M = hz.Matrix.from_csr(A, sell=True, ff=True)
    M.set_spmv(*variant)
    x, info = hz.zsolve(M, dev(b), tol=1e-10, maxit=3000, method="bicgstabl", ell=4)
    xo, io = oracle.bicgstabl(A, b, ell=4, tol=1e-10, maxit=3000)
    assert info.status == io.status == 0
    assert true_relres(oracle, A, host(x), b) <= 1e-10
    assert np.linalg.norm(host(x) - xo) / np.linalg.norm(xo) <= 1e-7
    # fewer BiCG steps than BiCGStab needs iterations on this system
    _, i0 = hz.zsolve(M, dev(b), tol=1e-10, maxit=3000)
    assert info.iters < i0.iters


def test_bicgstabl_jacobi(hz, oracle):
    rng = np.random.default_rng(51)
    A = W.fd_helmholtz_box(8, kh=0.5, damping=0.05)
    sc = rng.uniform(0.01, 100, A.n)
    As = W.CSR.from_scipy((A.to_scipy() @ sp.diags(sc)).tocsr())
    b = K.vectors(A.n, 52)[0]
    M = hz.Matrix.from_csr(As, ff=True)
    x, info = hz.zsolve(M, dev(b), tol=1e-10, maxit=3000, method="bicgstabl", ell=2, precond="jacobi")
    x_lu = np.linalg.solve(As.to_scipy().toarray(), b)
    assert info.converged and np.linalg.norm(host(x) - x_lu) <= 1e-8 * np.linalg.norm(x_lu)


def test_bicgstabl_edge_cases(hz, oracle):
    A, b, _ = W.c1_small_fd()
    M = hz.Matrix.from_csr(A, ff=True)
    x, info = hz.zsolve(M, torch.zeros(A.n, dtype=torch.complex128, device="cuda"), x=dev(np.ones(A.n, np.complex128)),
                        method="bicgstabl", ell=4)
    assert info.converged and info.iters == 0 and not host(x).any()
    x, info = hz.zsolve(M, dev(b), maxit=0, method="bicgstabl", ell=4)
    assert info.status == 4 and info.iters == 0 and not host(x).any()
    bn = b.copy()
    bn[0] = np.nan
    assert hz.zsolve(M, dev(bn), method="bicgstabl", ell=2)[1].status == 6
    # A = I: one BiCG step, x = b
    I = W.CSR.from_scipy(sp.identity(300, dtype=np.complex128, format="csr"))
    bi = K.vectors(300, 53)[0]
    MI = hz.Matrix.from_csr(I, ff=True)
    x, info = hz.zsolve(MI, dev(bi), tol=1e-10, method="bicgstabl", ell=4)
    assert info.converged and info.iters == 1
    assert np.allclose(host(x), bi, rtol=0, atol=1e-14)
    with pytest.raises(hz.HzError):
        hz.zsolve(M, dev(b), method="bicgstabl", ell=9)
    with pytest.raises(hz.HzError):
        hz.zsolve(M, dev(b), method="bicgstabl", ell=2, mode="mixed")
    # the BiCGStab solver on the same handle is unaffected
    x, info = hz.zsolve(M, dev(b), tol=1e-10)
    assert info.converged
