"""hz_zdotc_noalloc: the dot product for callers that must not allocate
device memory (its scratch is a fixed array inside libhz.so).

Called through the C ABI and compared with hz_zdotc, which allocates its own
scratch, and with the CPU oracle's compensated dot product, within the
dot-product tolerance of the other GPU tests:
|difference| <= 1e-13 * sum |x_i| |y_i|.  Two calls in a row check that the
shared array left by one call does not disturb the next.  The sizes cover
one tile, a ragged tail, more tiles than a block has threads (the last
block's fold then takes several partials per thread) and the largest
accepted length, where x = y = 1 gives the exact sum 2^28.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from tests import _cases as K

pytestmark = pytest.mark.gpu

TOL = 1e-13


def _p(t):
    return C.c_void_p(t.data_ptr())


def _dot(lib, fn, x, y):
    out = torch.empty(1, dtype=torch.complex128, device="cuda")
    st = fn(x.numel(), _p(x), _p(y), _p(out), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.hz_last_error()
    torch.cuda.synchronize()
    return complex(out.cpu()[0])


@pytest.mark.parametrize("n", [1, 4095, 4097, 1_000_003, (1 << 21) + 1, (1 << 22) + 3])
def test_noalloc_matches_zdotc_twice(hz, oracle, n):
    from paper_2112_06465_gb300 import _lib
    lib = _lib.load()
    for call in range(2):
        x, y = K.vectors(n, 700 + 10 * call + n % 7)
        xd, yd = torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda()
        ref = _dot(lib, lib.hz_zdotc, xd, yd)
        got = _dot(lib, lib.hz_zdotc_noalloc, xd, yd)
        bound = TOL * float(np.sum(np.abs(x) * np.abs(y)))
        assert abs(got - ref) <= bound, (call, got, ref)
        assert abs(got - oracle.zdotc(x, y)) <= bound, (call, got)


def test_noalloc_at_capacity(hz):
    """n = 2^28, the largest accepted length (65536 tiles), twice: with
    x = y = 1 every partial and the total are exact, so the result is 2^28."""
    from paper_2112_06465_gb300 import _lib
    lib = _lib.load()
    n = 1 << 28
    x = torch.ones(n, dtype=torch.complex128, device="cuda")
    for _ in range(2):
        got = _dot(lib, lib.hz_zdotc_noalloc, x, x)
        assert got == complex(n, 0.0)
    del x
    torch.cuda.empty_cache()


def test_noalloc_rejects_sizes_beyond_its_array(hz):
    from paper_2112_06465_gb300 import _lib
    lib = _lib.load()
    x = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = torch.zeros(1, dtype=torch.complex128, device="cuda")
    st = lib.hz_zdotc_noalloc((1 << 28) + 1, _p(x), _p(x), _p(out), None)
    assert st == _lib.HZ_ERR_ARG
    assert b"2^28" in lib.hz_last_error()
