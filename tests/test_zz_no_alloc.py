"""mpgemm_noalloc: the Strassen/Winograd product with its temporaries in the
library's static device scratch instead of allocated memory.

Callers that cannot allocate device memory while they multiply -- work being
captured into a CUDA graph, serving loops that must not touch an allocator,
hosts whose device memory belongs to another owner -- use this entry point.
It must give exactly the bits of mpgemm (the existing entry point, which
allocates its workspace) on consecutive calls that reuse the same scratch.
This file is collected last, so a failure here leaves every other test run.
"""
import ctypes

import pytest

from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, dev

pytestmark = pytest.mark.gpu


def _pair(m, l, n, p, seed):
    return dev(gen.uniform_pm1(m, l, p, seed, -16, 16)), dev(gen.uniform_pm1(l, n, p, seed + 1, -16, 16))


def test_noalloc_matches_mpgemm_on_consecutive_calls():
    cases = [(200, 200, 200, 512, mp.WINOGRAD, 64, 101),    # two recursion levels
             (151, 170, 133, 256, mp.STRASSEN, 32, 103)]    # odd sizes, peeled, 2 levels
    for m, l, n, p, algo, cutoff, seed in cases:
        A, B = _pair(m, l, n, p, seed)
        want = mp.DeviceMP.empty(m, n, p)
        mp.mpgemm(A, B, want, algo, cutoff)
        mp.check_status("mpgemm")
        got = mp.DeviceMP.empty(m, n, p)
        mp.mpgemm_noalloc(A, B, got, algo, cutoff)
        mp.check_status("mpgemm_noalloc")
        assert_bits_equal(got.to_host(), want.to_host(), "noalloc %s" % ((m, l, n, p, algo),))


def test_noalloc_rejects_products_beyond_the_scratch():
    p, n = 512, 256
    A, B = _pair(n, n, n, p, 7)
    Cm = mp.DeviceMP.empty(n, n, p)
    assert mp.workspace_size(n, n, n, p, mp.WINOGRAD, 64) > mp.NOALLOC_SCRATCH_BYTES
    a, b, c = A.struct(), B.struct(), Cm.struct()
    rc = mp.load_library().mpgemm_noalloc(n, n, n, p, mp.WINOGRAD, 64, ctypes.byref(a),
                                          ctypes.byref(b), ctypes.byref(c))
    assert rc == -8        # MP_ERR_SCRATCH
    assert mp.load_library().mp_strerror(-8).startswith(b"product needs more")
