"""ctypes loader of libhz.so, with argument types for every C-ABI entry point.

There is no fallback: if the library has not been built, importing the
package's compute API raises ImportError.  Build it with
``python -c "import __graft_entry__ as g; g.build()"`` or
``python paper_2112_06465_gb300/build.py``.
"""

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhz.so")

HZ_OK, HZ_ERR_ARG, HZ_ERR_CUDA, HZ_ERR_ALLOC = 0, 1, 2, 3
HZ_NOT_CONVERGED, HZ_BREAKDOWN, HZ_ERR_NAN, HZ_ERR_TIMEOUT = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_ALLOC", 4: "NOT_CONVERGED",
                5: "BREAKDOWN", 6: "ERR_NAN", 7: "ERR_TIMEOUT"}
SOLVE_OUTCOMES = (HZ_OK, HZ_NOT_CONVERGED, HZ_BREAKDOWN, HZ_ERR_NAN)

HZ_FLAG_VALIDATE, HZ_FLAG_SELL, HZ_FLAG_C64, HZ_FLAG_AUTOTUNE, HZ_FLAG_FF = 1, 2, 4, 8, 16
HZ_MODE_FP64, HZ_MODE_MIXED = 0, 1
HZ_PRECOND_NONE, HZ_PRECOND_JACOBI = 0, 1
HZ_METHOD_BICGSTAB, HZ_METHOD_BICGSTABL, HZ_METHOD_TFQMR = 0, 1, 2
(HZ_SPMV_CSR_VECTOR, HZ_SPMV_SELL, HZ_SPMV_FF, HZ_SPMV_SELL_FF, HZ_SPMV_FF_FLAT, HZ_SPMV_FF_TMA,
 HZ_SPMV_FLAT64, HZ_SPMV_FLAT64P) = 0, 1, 2, 3, 4, 5, 6, 7

# every symbol include/hz.h declares
EXPORTS = (
    "hz_csr_create", "hz_mat_destroy", "hz_mat_query", "hz_mat_set_spmv", "hz_mat_refresh_values",
    "hz_zspmv",
    "hz_cspmv", "hz_zdotc", "hz_zdotu", "hz_dznrm2", "hz_zaxpy", "hz_zscal", "hz_zcopy",
    "hz_zconj", "hz_zsolve", "hz_zsolve_opts", "hz_zsolve_batched", "hz_outer_on_pattern",
    "hz_mat_set_diag", "hz_diag_grad", "hz_last_error", "hz_version", "hz_zdotc_noalloc",
    "hz_mat_check", "hz_zmul_elementwise",
)


class hz_z(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class hz_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("restarts", C.c_int32),
                ("outer", C.c_int32), ("relres_rec", C.c_double), ("relres_true", C.c_double)]


class hz_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int32), ("mode", C.c_uint32),
                ("inner_tol", C.c_float), ("inner_maxit", C.c_int32), ("max_outer", C.c_int32),
                ("x0_is_zero", C.c_int32), ("d_hist", C.c_void_p), ("precond", C.c_uint32),
                ("method", C.c_uint32), ("ell", C.c_int32)]


class hz_mat_props(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("max_row", C.c_int32),
                ("min_row", C.c_int32), ("mean_row", C.c_double), ("spmv_kind", C.c_int32),
                ("group", C.c_int32), ("sell_slots", C.c_int64), ("sell_sigma", C.c_int32),
                ("has_c64", C.c_int32)]


class HzError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libhz.so and declare its signatures (raises ImportError if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhz.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    P, i32, i64, u32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
    sig = {
        "hz_csr_create": [C.POINTER(C.c_void_p), i32, i32, P, P, P, i32, u32, P],
        "hz_mat_destroy": [P],
        "hz_mat_query": [P, C.POINTER(hz_mat_props)],
        "hz_mat_check": [P, P],
        "hz_zmul_elementwise": [i64, P, P, P, P],
        "hz_mat_set_spmv": [P, i32, i32],
        "hz_mat_refresh_values": [P, P],
        "hz_zspmv": [P, P, P, P],
        "hz_cspmv": [P, P, P, P],
        "hz_zdotc": [i64, P, P, P, P],
        "hz_zdotu": [i64, P, P, P, P],
        "hz_zdotc_noalloc": [i64, P, P, P, P],
        "hz_dznrm2": [i64, P, P, P],
        "hz_zaxpy": [i64, P, P, P, P],
        "hz_zscal": [i64, P, P, P],
        "hz_zcopy": [i64, P, P, P],
        "hz_zconj": [i64, P, P, P],
        "hz_zsolve": [P, P, P, f64, i32, u32, C.POINTER(hz_info), P],
        "hz_zsolve_opts": [P, P, P, C.POINTER(hz_solve_opts), C.POINTER(hz_info), P],
        "hz_zsolve_batched": [i32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                              C.POINTER(C.c_void_p), f64, i32, u32, C.POINTER(hz_info), P],
        "hz_outer_on_pattern": [P, P, P, P, P],
        "hz_mat_set_diag": [P, P, hz_z, P, P],
        "hz_diag_grad": [P, P, P, hz_z, P, P],
        "hz_last_error": [],
        "hz_version": [],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.hz_last_error.restype = C.c_char_p
    lib.hz_version.restype = C.c_int32
    _lib = lib
    return lib


def check(status: int, allow=(HZ_OK,)):
    """Raise HzError unless status is in `allow`; returns the status."""
    if status not in allow:
        raise HzError(status, load().hz_last_error().decode(errors="replace"))
    return status
