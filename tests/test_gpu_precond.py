"""GPU parity: the element-wise product (Section 5) and Jacobi right
preconditioning of BiCGStab (Section 7's "P-" solver) through the C ABI,
against the CPU oracle (which applies z = D^-1 p explicitly, while the GPU
runs on the column-scaled operator A D^-1) and dense LU."""

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


def test_zmul_elementwise(hz, oracle):
    rng = np.random.default_rng(41)
    n = 100_003
    xi = rng.integers(-9, 10, n) + 1j * rng.integers(-9, 10, n)
    yi = rng.integers(-9, 10, n) + 1j * rng.integers(-9, 10, n)
    assert np.array_equal(host(hz.zmul_elementwise(dev(xi), dev(yi))), oracle.zmul_elementwise(xi, yi))
    x, y = K.vectors(n, 42)[:2]
    z = host(hz.zmul_elementwise(dev(x), dev(y)))
    ref = oracle.zmul_elementwise(x, y)
    assert np.all(np.abs(z - ref) <= 1e-15 * np.abs(x) * np.abs(y))
    xd = dev(x)
    hz.zmul_elementwise(xd, dev(y), xd)          # in place
    assert np.all(np.abs(host(xd) - ref) <= 1e-15 * np.abs(x) * np.abs(y))
    assert hz.zmul_elementwise(dev(x[:0]), dev(y[:0])).numel() == 0


def scaled_columns(A, seed):
    rng = np.random.default_rng(seed)
    sc = rng.uniform(0.01, 100, A.n) * np.exp(1j * rng.uniform(0, 2 * np.pi, A.n))
    return W.CSR.from_scipy((A.to_scipy() @ sp.diags(sc)).tocsr())


@pytest.mark.parametrize("ff", [False, True])
def test_jacobi_fd_box_vs_oracle_and_lu(hz, oracle, ff):
    A = scaled_columns(W.fd_helmholtz_box(8, kh=0.5, damping=0.05), 43)
    b = K.vectors(A.n, 44)[0]
    M = hz.Matrix.from_csr(A, ff=ff)
    hist = torch.zeros(3001, dtype=torch.float64, device="cuda")
    x, info = hz.zsolve(M, dev(b), tol=1e-11, maxit=3000, precond="jacobi", hist=hist)
    xo, io = oracle.bicgstab(A, b, tol=1e-11, maxit=3000, precond="jacobi")
    x_lu = np.linalg.solve(A.to_scipy().toarray(), b)
    assert info.converged and io.status == 0
    assert abs(info.iters - io.iters) <= max(5, 0.1 * io.iters)
    xg = host(x)
    assert true_relres(oracle, A, xg, b) <= 1e-11
    assert np.linalg.norm(xg - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
    h = host(hist)
    assert h[0] == 1.0
    assert np.all(np.abs(h[1:6] - io.hist[1:6]) <= 1e-10 * io.hist[1:6])
    # the same system without the preconditioner: the scaling costs iterations
    _, i0 = hz.zsolve(M, dev(b), tol=1e-11, maxit=3000)
    assert i0.iters > 2 * info.iters


@pytest.mark.parametrize("variant", [("csr", 4), ("ff", 4), ("ffflat", 0), ("fftma", 0), ("sell", 0)])
def test_jacobi_cylinder_variants(hz, oracle, variant):
    A, b = K.small_cylinder()
    M = hz.Matrix.from_csr(A, sell=True, ff=True)
    M.set_spmv(*variant)
    x, info = hz.zsolve(M, dev(b), tol=1e-10, maxit=3000, precond="jacobi")
    xo, io = oracle.bicgstab(A, b, tol=1e-10, maxit=3000, precond="jacobi")
    assert info.status == io.status
    if io.status == 0:
        assert true_relres(oracle, A, host(x), b) <= 1e-10
        assert np.linalg.norm(host(x) - xo) / np.linalg.norm(xo) <= 1e-7
    M.check()


def test_jacobi_start_and_refresh(hz, oracle):
    """x0 enters through y0 = D x0: starting from the solution ends at once;
    new values (refresh / set_diag) rebuild the scaled operator."""
    A = scaled_columns(W.fd_helmholtz_box(6, kh=0.5, damping=0.05), 45)
    b = K.vectors(A.n, 46)[0]
    M = hz.Matrix.from_csr(A, ff=True)
    xs, _ = oracle.bicgstab(A, b, tol=1e-13, maxit=3000, precond="jacobi")
    x, info = hz.zsolve(M, dev(b), x=dev(xs), tol=1e-10, precond="jacobi")
    assert info.converged and info.iters == 0
    assert np.linalg.norm(host(x) - xs) <= 1e-12 * np.linalg.norm(xs)
    # change the values in place (scale the whole matrix by 2) and refresh
    M.val.mul_(2.0)
    M.refresh_values()
    A2 = W.CSR(A.n, A.rowptr, A.col, 2.0 * A.val)
    x2, info2 = hz.zsolve(M, dev(b), tol=1e-10, precond="jacobi")
    assert info2.converged
    assert true_relres(oracle, A2, host(x2), b) <= 1e-10
    assert np.linalg.norm(host(x2) - xs / 2) <= 1e-8 * np.linalg.norm(xs / 2)


def test_jacobi_mixed_and_edge_cases(hz, oracle):
    A = W.fd_helmholtz_box(12, kh=0.5, damping=0.05)
    b = K.vectors(A.n, 47)[0]
    M = hz.Matrix.from_csr(A, c64=True)
    x, info = hz.zsolve(M, dev(b), tol=1e-10, mode="mixed", precond="jacobi")
    assert info.converged and true_relres(oracle, A, host(x), b) <= 1e-10
    # b = 0 and maxit = 0 behave as without a preconditioner
    x, info = hz.zsolve(M, torch.zeros(A.n, dtype=torch.complex128, device="cuda"), precond="jacobi")
    assert info.converged and info.iters == 0 and not host(x).any()
    x, info = hz.zsolve(M, dev(b), maxit=0, precond="jacobi")
    assert info.status == 4 and info.iters == 0
    with pytest.raises(ValueError):
        hz.zsolve(M, dev(b), precond="ilu")
