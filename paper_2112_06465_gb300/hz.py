"""Python binding of libhz (argument marshalling only).

Every function takes CUDA tensors (torch.complex128 vectors, int32 CSR
indices), passes their device pointers and the current CUDA stream to the C
ABI of include/hz.h, and returns CUDA tensors.  All arithmetic happens in the
library's kernels; nothing here computes on the CPU and there is no fallback.
PyTorch provides device memory and streams only.
"""

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import (HZ_FLAG_AUTOTUNE, HZ_FLAG_C64, HZ_FLAG_SELL, HZ_FLAG_VALIDATE,  # noqa: F401
                   HZ_MODE_FP64, HZ_MODE_MIXED, HzError, check, hz_info, hz_mat_props,
                   hz_solve_opts, hz_z)

_L = _lib.load()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _vec(t, dtype=torch.complex128, name="vector"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Matrix:
    """CSR matrix handle (Section 3.2 storage: values, column indices, row pointers).

    The handle borrows the three tensors (index_base 0), so they are kept
    referenced here for its lifetime.
    """

    def __init__(self, rowptr, col, val, index_base=0, sell=False, c64=False, autotune=False,
                 validate=False, ff=False):
        self.rowptr = _vec(rowptr, torch.int32, "rowptr")
        self.col = _vec(col, torch.int32, "col")
        self.val = _vec(val, torch.complex128, "val")
        self.n = rowptr.numel() - 1
        self.nnz = col.numel()
        flags = ((HZ_FLAG_SELL if sell else 0) | (HZ_FLAG_C64 if c64 else 0)
                 | (HZ_FLAG_AUTOTUNE if autotune else 0) | (HZ_FLAG_VALIDATE if validate else 0)
                 | (_lib.HZ_FLAG_FF if ff else 0))
        h = C.c_void_p()
        check(_L.hz_csr_create(C.byref(h), self.n, self.nnz, _ptr(self.rowptr), _ptr(self.col),
                               _ptr(self.val), int(index_base), flags, _stream()))
        self._h = h

    @classmethod
    def from_csr(cls, csr, device="cuda", **kw):
        """From a host CSR object with numpy fields n, rowptr, col, val."""
        rp = torch.as_tensor(csr.rowptr, dtype=torch.int32).to(device)
        cl = torch.as_tensor(csr.col, dtype=torch.int32).to(device)
        vl = torch.as_tensor(csr.val, dtype=torch.complex128).to(device)
        return cls(rp, cl, vl, **kw)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("matrix handle is closed")
        return self._h

    def props(self) -> dict:
        p = hz_mat_props()
        check(_L.hz_mat_query(self.handle, C.byref(p)))
        return {f: getattr(p, f) for f, _ in p._fields_}

    def set_spmv(self, kind="csr", group=4):
        """Force the SpMV variant: ("csr" | "ff", lanes per row) or ("flat64p" | "flat64" |
        "sell" | "sellff" | "ffflat" | "fftma", ignored)."""
        k = {"sell": _lib.HZ_SPMV_SELL, "ff": _lib.HZ_SPMV_FF, "sellff": _lib.HZ_SPMV_SELL_FF,
             "ffflat": _lib.HZ_SPMV_FF_FLAT, "fftma": _lib.HZ_SPMV_FF_TMA,
             "flat64": _lib.HZ_SPMV_FLAT64, "flat64p": _lib.HZ_SPMV_FLAT64P}.get(kind, _lib.HZ_SPMV_CSR_VECTOR)
        check(_L.hz_mat_set_spmv(self.handle, k, int(group)))

    def check(self):
        """Synchronise the current stream and raise HzError(ERR_TIMEOUT) if a bounded
        wait of an asynchronous SpMV on this handle expired."""
        check(_L.hz_mat_check(self.handle, _stream()))

    def refresh_values(self):
        check(_L.hz_mat_refresh_values(self.handle, _stream()))

    def close(self):
        if getattr(self, "_h", None) is not None:
            _L.hz_mat_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # conveniences
    def __matmul__(self, x):
        return zspmv(self, x)

    def solve(self, b, **kw):
        return zsolve(self, b, **kw)


def zspmv(A: Matrix, x, y=None):
    """y = A x (complex128)."""
    x = _vec(x, name="x")
    if y is None:
        y = torch.empty(A.n, dtype=torch.complex128, device=x.device)
    check(_L.hz_zspmv(A.handle, _ptr(x), _ptr(_vec(y, name="y")), _stream()))
    return y


def cspmv(A: Matrix, x, y=None):
    """y = A32 x with the handle's complex64 copy (binary32 sums)."""
    x = _vec(x, torch.complex64, "x")
    if y is None:
        y = torch.empty(A.n, dtype=torch.complex64, device=x.device)
    check(_L.hz_cspmv(A.handle, _ptr(x), _ptr(_vec(y, torch.complex64, "y")), _stream()))
    return y


def _pair(x, y):
    x, y = _vec(x, name="x"), _vec(y, name="y")
    if x.numel() != y.numel():
        raise ValueError("length mismatch")
    return x, y


def zdotc(x, y, out=None):
    """sum conj(x_i) y_i, returned as a 1-element device tensor."""
    x, y = _pair(x, y)
    out = torch.empty(1, dtype=torch.complex128, device=x.device) if out is None else out
    check(_L.hz_zdotc(x.numel(), _ptr(x), _ptr(y), _ptr(out), _stream()))
    return out


def zdotu(x, y, out=None):
    """sum x_i y_i, returned as a 1-element device tensor."""
    x, y = _pair(x, y)
    out = torch.empty(1, dtype=torch.complex128, device=x.device) if out is None else out
    check(_L.hz_zdotu(x.numel(), _ptr(x), _ptr(y), _ptr(out), _stream()))
    return out


def dznrm2(x, out=None):
    """sqrt(sum |x_i|^2), returned as a 1-element float64 device tensor."""
    x = _vec(x, name="x")
    out = torch.empty(1, dtype=torch.float64, device=x.device) if out is None else out
    check(_L.hz_dznrm2(x.numel(), _ptr(x), _ptr(out), _stream()))
    return out


def _scalar(alpha, device):
    if isinstance(alpha, torch.Tensor):
        return _vec(alpha.reshape(1), name="alpha")
    return torch.tensor([complex(alpha)], dtype=torch.complex128, device=device)


def zaxpy(alpha, x, y):
    """y = alpha x + y in place; alpha is a number or a 1-element device tensor."""
    x, y = _pair(x, y)
    a = _scalar(alpha, x.device)
    check(_L.hz_zaxpy(x.numel(), _ptr(a), _ptr(x), _ptr(y), _stream()))
    return y


def zscal(alpha, x):
    """x = alpha x in place."""
    x = _vec(x, name="x")
    a = _scalar(alpha, x.device)
    check(_L.hz_zscal(x.numel(), _ptr(a), _ptr(x), _stream()))
    return x


def zcopy(x, y=None):
    """y = x."""
    x = _vec(x, name="x")
    y = torch.empty_like(x) if y is None else y
    x, y = _pair(x, y)
    check(_L.hz_zcopy(x.numel(), _ptr(x), _ptr(y), _stream()))
    return y


def zmul_elementwise(x, y, z=None):
    """z_i = x_i y_i (z may be x or y)."""
    x, y = _pair(x, y)
    z = torch.empty_like(x) if z is None else _vec(z, name="z")
    check(_L.hz_zmul_elementwise(x.numel(), _ptr(x), _ptr(y), _ptr(z), _stream()))
    return z


def zconj(x, y=None):
    """y = conj(x) (y may be x)."""
    x = _vec(x, name="x")
    y = torch.empty_like(x) if y is None else y
    check(_L.hz_zconj(x.numel(), _ptr(x), _ptr(_vec(y, name="y")), _stream()))
    return y


@dataclass
class SolveInfo:
    iters: int
    status: int
    restarts: int
    outer: int
    relres_rec: float
    relres_true: float

    @property
    def status_name(self):
        return _lib.STATUS_NAMES.get(self.status, str(self.status))

    @property
    def converged(self):
        return self.status == _lib.HZ_OK


def _info(i: hz_info) -> SolveInfo:
    return SolveInfo(i.iters, i.status, i.restarts, i.outer, i.relres_rec, i.relres_true)


def zsolve(A: Matrix, b, x=None, tol=1e-10, maxit=2000, mode="fp64", hist=None,
           inner_tol=1e-5, inner_maxit=1000, max_outer=50, precond="none", method="bicgstab", ell=4,
           x0_zero=None):
    """Solve A x = b with BiCGStab on the device; returns (x, SolveInfo).

    x (optional) holds x0 and receives the solution (x0_zero=True: start
    from x0 = 0 whatever x holds; the default is x0 = 0 only without x); mode is "fp64" or
    "mixed"; precond is "none" or "jacobi" (right preconditioning by the
    inverse diagonal); method is "bicgstab", "bicgstabl" (BiCGStab(ell),
    iterations counted in BiCG steps) or "tfqmr" (stopping on the
    quasi-residual bound, hist holding that bound); hist (optional float64 device tensor
    of maxit+1 entries, maxit+ell for BiCGStab(ell)) receives the residual
    history.  Non-convergence is reported in the info, not raised.
    """
    if method not in ("bicgstab", "bicgstabl", "tfqmr"):
        raise ValueError("method must be 'bicgstab', 'bicgstabl' or 'tfqmr'")
    if precond not in ("none", "jacobi"):
        raise ValueError("precond must be 'none' or 'jacobi'")
    b = _vec(b, name="b")
    if x0_zero is None:
        x0_zero = x is None
    if x is None:
        x = torch.empty_like(b)
    x = _vec(x, name="x")
    o = hz_solve_opts()
    o.tol = float(tol)
    o.maxit = int(maxit)
    o.mode = HZ_MODE_MIXED if mode == "mixed" else HZ_MODE_FP64
    o.inner_tol = float(inner_tol)
    o.inner_maxit = int(inner_maxit)
    o.max_outer = int(max_outer)
    o.x0_is_zero = 1 if x0_zero else 0
    o.d_hist = hist.data_ptr() if hist is not None else None
    o.precond = _lib.HZ_PRECOND_JACOBI if precond == "jacobi" else _lib.HZ_PRECOND_NONE
    o.method = {"bicgstab": _lib.HZ_METHOD_BICGSTAB, "bicgstabl": _lib.HZ_METHOD_BICGSTABL,
                "tfqmr": _lib.HZ_METHOD_TFQMR}[method]
    o.ell = int(ell)
    need = maxit + (int(ell) if method == "bicgstabl" else 1)
    if hist is not None and (hist.dtype != torch.float64 or hist.numel() < need):
        raise ValueError(f"hist must be a float64 device tensor with {need} entries")
    info = hz_info()
    check(_L.hz_zsolve_opts(A.handle, _ptr(b), _ptr(x), C.byref(o), C.byref(info), _stream()),
          allow=_lib.SOLVE_OUTCOMES)
    return x, _info(info)


def zsolve_batched(mats, bs, xs=None, tol=1e-10, maxit=2000, mode="fp64"):
    """Solve A[s] x[s] = b[s] for every s in one persistent launch.

    xs (optional) hold the starting guesses (zero if omitted) and receive the
    solutions; mode "fp64" (BiCGStab) or "mixed" (complex64 inner BiCGStab
    with binary64 refinement per system; maxit caps each system's inner
    iterations in total).  Returns (xs, [SolveInfo])."""
    ns = len(mats)
    if xs is None:
        xs = [torch.zeros_like(b) for b in bs]
    arrA = (C.c_void_p * ns)(*[m.handle.value for m in mats])
    arrB = (C.c_void_p * ns)(*[_vec(b, name="b").data_ptr() for b in bs])
    arrX = (C.c_void_p * ns)(*[_vec(x, name="x").data_ptr() for x in xs])
    infos = (hz_info * ns)()
    if mode not in ("fp64", "mixed"):
        raise ValueError("mode must be 'fp64' or 'mixed'")
    md = HZ_MODE_MIXED if mode == "mixed" else HZ_MODE_FP64
    check(_L.hz_zsolve_batched(ns, arrA, arrB, arrX, float(tol), int(maxit), md, infos,
                               _stream()), allow=_lib.SOLVE_OUTCOMES)
    return xs, [_info(i) for i in infos]


def outer_on_pattern(A: Matrix, mu, x, out=None):
    """grad[k] = -conj(mu_i x_j) for every stored entry k = (i, j)."""
    mu, x = _pair(mu, x)
    out = torch.empty(A.nnz, dtype=torch.complex128, device=x.device) if out is None else out
    check(_L.hz_outer_on_pattern(A.handle, _ptr(mu), _ptr(x), _ptr(out), _stream()))
    return out


def mat_set_diag(A: Matrix, base, scale, theta):
    """A_ii = base_i + scale * theta_i written into A's value tensor."""
    base, theta = _pair(base, theta)
    s = complex(scale)
    check(_L.hz_mat_set_diag(A.handle, _ptr(base), hz_z(s.real, s.imag), _ptr(theta), _stream()))


def diag_grad(A: Matrix, mu, x, scale, out=None):
    """grad_theta_i = conj(scale) * (-conj(mu_i x_i))."""
    mu, x = _pair(mu, x)
    out = torch.empty_like(x) if out is None else out
    s = complex(scale)
    check(_L.hz_diag_grad(A.handle, _ptr(mu), _ptr(x), hz_z(s.real, s.imag), _ptr(out), _stream()))
    return out


def version() -> int:
    return int(_L.hz_version())
