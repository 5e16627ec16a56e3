"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point include/hz.h declares, and rejects
invalid arguments before touching the device."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    with open(os.path.join(ROOT, "include", "hz.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"HZ_API\s+[\w\s\*]+?\b(hz_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    from paper_2112_06465_gb300 import _lib
    return _lib.load()


def test_header_declares_the_paper_calls():
    syms = header_symbols()
    for name in ("hz_zspmv", "hz_zdotc", "hz_zdotu", "hz_dznrm2", "hz_zaxpy", "hz_zscal", "hz_zcopy",
                 "hz_zsolve", "hz_zsolve_batched", "hz_csr_create", "hz_outer_on_pattern"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    from paper_2112_06465_gb300 import _lib
    syms = header_symbols()
    assert sorted(_lib.EXPORTS) == syms
    for name in syms:
        assert hasattr(lib, name), name


def test_only_declared_symbols_are_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only",
                          os.path.join(ROOT, "paper_2112_06465_gb300", "libhz.so")],
                         capture_output=True, text=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T " in ln})
    assert exported == header_symbols()


def test_version_and_error_string(lib):
    assert lib.hz_version() == 100
    assert isinstance(lib.hz_last_error(), bytes)


def test_argument_errors_without_device(lib):
    from paper_2112_06465_gb300 import _lib
    out = C.c_void_p()
    # index_base must be 0 or 1; sizes must be non-negative
    assert lib.hz_csr_create(C.byref(out), 4, 4, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), 2, 0,
                             None) == _lib.HZ_ERR_ARG
    assert b"index_base" in lib.hz_last_error()
    assert lib.hz_csr_create(C.byref(out), -1, 0, C.c_void_p(16), None, None, 0, 0, None) == _lib.HZ_ERR_ARG
    assert lib.hz_zdotc(-1, None, None, C.c_void_p(16), None) == _lib.HZ_ERR_ARG
    assert lib.hz_dznrm2(5, None, C.c_void_p(16), None) == _lib.HZ_ERR_ARG
    assert lib.hz_zaxpy(5, None, None, None, None) == _lib.HZ_ERR_ARG
    assert lib.hz_zsolve(None, None, None, 1e-10, 10, 0, None, None) == _lib.HZ_ERR_ARG
    assert lib.hz_zsolve_batched(2, None, None, None, 1e-10, 10, 1, None, None) == _lib.HZ_ERR_ARG
    assert lib.hz_mat_set_spmv(None, 0, 4) == _lib.HZ_ERR_ARG


def test_build_targets_sm103a_only():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_b", os.path.join(ROOT, "paper_2112_06465_gb300", "build.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    assert m.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
