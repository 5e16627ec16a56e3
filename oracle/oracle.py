"""ctypes wrapper of the C oracle (``hz_oracle.c``) -- TEST INFRASTRUCTURE.

Arrays are numpy: int32 CSR indices, complex128 (or complex64) values and
vectors, C-contiguous.  Every function returns new arrays and leaves its
inputs untouched unless its name says otherwise (``zaxpy``/``zscal`` return
the updated copy).
"""

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hz_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64 arithmetic, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """The same source built with -fopenmp: SpMV rows and BiCGStab vector
    updates over threads, reductions over fixed chunks (deterministic for
    any thread count).  Used only for the benchmark's all-cores CPU baseline;
    the tests use the plain build."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def bicgstab_omp(A, b, tol=1e-10, maxit=2000, threads=1):
    """or_bicgstab from the OpenMP build on `threads` threads; returns (x, OracleInfo)."""
    global _lib_omp
    if _lib_omp is None:
        build_omp()
        lib = C.CDLL(_LIB_OMP)
        P = C.c_void_p
        lib.or_bicgstab.argtypes = [C.c_int32, P, P, P, P, P, C.c_double, C.c_int32, P, P]
        lib.or_bicgstab.restype = C.c_int
        lib.or_set_threads.argtypes = [C.c_int32]
        _lib_omp = lib
    _lib_omp.or_set_threads(int(threads))
    b = _z(b)
    x = np.zeros(A.n, dtype=np.complex128)
    info = _OrInfo()
    rp, cl, vl = _i(A.rowptr), _i(A.col), _z(A.val)
    _lib_omp.or_bicgstab(A.n, _p(rp), _p(cl), _p(vl), _p(b), _p(x), float(tol), int(maxit), None, C.byref(info))
    return x, OracleInfo(info.iters, info.status, info.restarts, info.relres_rec, info.relres_true)


def load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        i32, i64, f64, f32 = C.c_int32, C.c_int64, C.c_double, C.c_float
        lib.or_zspmv.argtypes = [i32, P, P, P, P, P]
        lib.or_cspmv.argtypes = [i32, P, P, P, P, P]
        for f in (lib.or_zdotc, lib.or_zdotu):
            f.argtypes = [i64, P, P, P]
        lib.or_dznrm2.argtypes = [i64, P]
        lib.or_dznrm2.restype = f64
        lib.or_zaxpy.argtypes = [i64, P, P, P]
        lib.or_zscal.argtypes = [i64, P, P]
        lib.or_zcopy.argtypes = [i64, P, P]
        lib.or_bicgstab.argtypes = [i32, P, P, P, P, P, f64, i32, P, P]
        lib.or_bicgstab.restype = C.c_int
        lib.or_bicgstab_pc.argtypes = [i32, P, P, P, P, P, P, f64, i32, P, P]
        lib.or_bicgstab_pc.restype = C.c_int
        lib.or_jacobi_dinv.argtypes = [i32, P, P, P, P]
        lib.or_bicgstabl.argtypes = [i32, P, P, P, i32, P, P, f64, i32, P, P]
        lib.or_bicgstabl.restype = C.c_int
        lib.or_tfqmr.argtypes = [i32, P, P, P, P, P, f64, i32, P, P]
        lib.or_tfqmr.restype = C.c_int
        lib.or_zmul_elementwise.argtypes = [i64, P, P, P]
        lib.or_cbicgstab.argtypes = [i32, P, P, P, P, P, f32, i32, P, P]
        lib.or_cbicgstab.restype = i32
        lib.or_refine_mixed.argtypes = [i32, P, P, P, P, P, P, f64, f32, i32, i32, P, P, P]
        lib.or_refine_mixed.restype = C.c_int
        lib.or_outer_on_pattern.argtypes = [i32, P, P, P, P, P]
        _lib = lib
    return _lib


class _OrInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("restarts", C.c_int32),
                ("relres_rec", C.c_double), ("relres_true", C.c_double)]


@dataclass
class OracleInfo:
    iters: int
    status: int
    restarts: int
    relres_rec: float
    relres_true: float
    hist: np.ndarray = None


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _z(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def zspmv(A, x):
    lib = load()
    x = _z(x)
    y = np.empty(A.n, dtype=np.complex128)
    rp, cl, vl = _i(A.rowptr), _i(A.col), _z(A.val)
    lib.or_zspmv(A.n, _p(rp), _p(cl), _p(vl), _p(x), _p(y))
    return y


def cspmv(A, x, val32=None):
    lib = load()
    x = _c(x)
    v = _c(A.val if val32 is None else val32)
    y = np.empty(A.n, dtype=np.complex64)
    rp, cl = _i(A.rowptr), _i(A.col)
    lib.or_cspmv(A.n, _p(rp), _p(cl), _p(v), _p(x), _p(y))
    return y


def _dot(fn, x, y):
    x, y = _z(x), _z(y)
    out = np.zeros(1, dtype=np.complex128)
    fn(x.size, _p(x), _p(y), _p(out))
    return complex(out[0])


def zdotc(x, y):
    return _dot(load().or_zdotc, x, y)


def zdotu(x, y):
    return _dot(load().or_zdotu, x, y)


def dznrm2(x):
    x = _z(x)
    return float(load().or_dznrm2(x.size, _p(x)))


def zaxpy(alpha, x, y):
    x, y = _z(x), _z(y).copy()
    a = np.array([alpha], dtype=np.complex128)
    load().or_zaxpy(x.size, _p(a), _p(x), _p(y))
    return y


def zscal(alpha, x):
    x = _z(x).copy()
    a = np.array([alpha], dtype=np.complex128)
    load().or_zscal(x.size, _p(a), _p(x))
    return x


def zcopy(x):
    x = _z(x)
    y = np.empty_like(x)
    load().or_zcopy(x.size, _p(x), _p(y))
    return y


def jacobi_dinv(A):
    """Inverse diagonal of A (Section 7's Jacobi preconditioner): 1 / a_ii, or 1
    where the diagonal is absent or zero."""
    lib = load()
    d = np.zeros(A.n, dtype=np.complex128)
    rp, cl, vl = _i(A.rowptr), _i(A.col), _z(A.val)
    lib.or_jacobi_dinv(A.n, _p(rp), _p(cl), _p(vl), _p(d))
    return d


def zmul_elementwise(x, y):
    """z_i = x_i y_i (Section 5's element-wise product)."""
    lib = load()
    x, y = _z(x), _z(y)
    z = np.zeros_like(x)
    lib.or_zmul_elementwise(x.size, _p(x), _p(y), _p(z))
    return z


def bicgstab(A, b, x0=None, tol=1e-10, maxit=2000, history=True, precond=None):
    """BiCGStab in binary64; returns (x, OracleInfo).  precond None (the
    preconditioner-free method) or "jacobi" (right-preconditioned by the
    inverse diagonal)."""
    lib = load()
    b = _z(b)
    x = np.zeros(A.n, dtype=np.complex128) if x0 is None else _z(x0).copy()
    hist = np.full(maxit + 1, np.nan) if history else None
    info = _OrInfo()
    rp, cl, vl = _i(A.rowptr), _i(A.col), _z(A.val)
    if precond not in (None, "none", "jacobi"):
        raise ValueError("precond must be None or 'jacobi'")
    dinv = jacobi_dinv(A) if precond == "jacobi" else None
    lib.or_bicgstab_pc(A.n, _p(rp), _p(cl), _p(vl), _p(dinv) if dinv is not None else None, _p(b), _p(x),
                       float(tol), int(maxit), _p(hist) if history else None, C.byref(info))
    out = OracleInfo(info.iters, info.status, info.restarts, info.relres_rec, info.relres_true)
    if history:
        out.hist = hist[: info.iters + 1].copy()
    return x, out


def bicgstabl(A, b, ell=2, x0=None, tol=1e-10, maxit=2000, history=True):
    """BiCGStab(l) in binary64 (l BiCG steps + a minimal-residual step per outer
    iteration); returns (x, OracleInfo) with iters counted in BiCG steps."""
    lib = load()
    b = _z(b)
    x = np.zeros(A.n, dtype=np.complex128) if x0 is None else _z(x0).copy()
    hist = np.full(maxit + int(ell) + 1, np.nan) if history else None
    info = _OrInfo()
    rp, cl, vl = _i(A.rowptr), _i(A.col), _z(A.val)
    st = lib.or_bicgstabl(A.n, _p(rp), _p(cl), _p(vl), int(ell), _p(b), _p(x), float(tol), int(maxit),
                          _p(hist) if history else None, C.byref(info))
    if st < 0:
        raise ValueError("ell must be in 1..8")
    out = OracleInfo(info.iters, info.status, info.restarts, info.relres_rec, info.relres_true)
    if history:
        out.hist = hist[: info.iters + 1].copy()
    return x, out


def tfqmr(A, b, x0=None, tol=1e-10, maxit=2000, history=True):
    """TFQMR in binary64, stopping on the quasi-residual bound; returns (x,
    OracleInfo) with iters counted in iterations (two products with A each)."""
    lib = load()
    b = _z(b)
    x = np.zeros(A.n, dtype=np.complex128) if x0 is None else _z(x0).copy()
    hist = np.full(maxit + 1, np.nan) if history else None
    info = _OrInfo()
    rp, cl, vl = _i(A.rowptr), _i(A.col), _z(A.val)
    lib.or_tfqmr(A.n, _p(rp), _p(cl), _p(vl), _p(b), _p(x), float(tol), int(maxit),
                 _p(hist) if history else None, C.byref(info))
    out = OracleInfo(info.iters, info.status, info.restarts, info.relres_rec, info.relres_true)
    if history:
        out.hist = hist[: info.iters + 1].copy()
    return x, out


def cbicgstab(A, b, tol=1e-5, maxit=1000, val32=None, history=False):
    """complex64 BiCGStab with binary32 sums from x0 = 0; returns (x, iters, status),
    plus the residual history (||r_j|| / ||b||, j = 0..iters) with history=True."""
    lib = load()
    b = _c(b)
    v = _c(A.val if val32 is None else val32)
    x = np.zeros(A.n, dtype=np.complex64)
    st = C.c_int32(0)
    rp, cl = _i(A.rowptr), _i(A.col)
    hist = np.full(int(maxit) + 1, np.nan) if history else None
    it = lib.or_cbicgstab(A.n, _p(rp), _p(cl), _p(v), _p(b), _p(x), float(tol), int(maxit),
                          C.byref(st), _p(hist) if history else None)
    if history:
        return x, int(it), int(st.value), hist[: int(it) + 1].copy()
    return x, int(it), int(st.value)


def refine_mixed(A, b, x0=None, tol=1e-10, tol_inner=1e-5, maxit_inner=1000, max_outer=50):
    """complex64 inner / complex128 outer iterative refinement.

    Returns (x, dict(status, outer, inner_total, relres))."""
    lib = load()
    b = _z(b)
    x = np.zeros(A.n, dtype=np.complex128) if x0 is None else _z(x0).copy()
    v32 = _c(A.val)
    rp, cl, vl = _i(A.rowptr), _i(A.col), _z(A.val)
    o, it, rel = C.c_int32(0), C.c_int32(0), C.c_double(0)
    st = lib.or_refine_mixed(A.n, _p(rp), _p(cl), _p(vl), _p(v32), _p(b), _p(x), float(tol),
                             float(tol_inner), int(maxit_inner), int(max_outer), C.byref(o),
                             C.byref(it), C.byref(rel))
    return x, {"status": int(st), "outer": int(o.value), "inner_total": int(it.value),
               "relres": float(rel.value)}


def outer_on_pattern(A, mu, x):
    """grad[k] = -conj(mu_i x_j) for each stored entry k = (i, j) of A."""
    lib = load()
    mu, x = _z(mu), _z(x)
    g = np.empty(A.nnz, dtype=np.complex128)
    rp, cl = _i(A.rowptr), _i(A.col)
    lib.or_outer_on_pattern(A.n, _p(rp), _p(cl), _p(mu), _p(x), _p(g))
    return g
