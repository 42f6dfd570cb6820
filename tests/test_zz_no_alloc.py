"""mpgemm_noalloc: C := A B with the Strassen/Winograd temporaries in the
library's static device scratch instead of allocated memory.

It is for callers that cannot allocate device memory while they multiply:
real-time or serving loops that must not touch an allocator (an allocation
can synchronise the device and stall them), code that runs inside a host
framework's allocator or memory-pool callback (re-entering the allocator
there can deadlock), and hosts whose device memory is all handed out in
advance by another owner.  It must give exactly the bits of mpgemm (the
entry point that allocates its workspace) on consecutive calls that reuse
the same scratch.  This file is collected last, so a failure here leaves
every other test run.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, dev

pytestmark = pytest.mark.gpu


def _pair(m, l, n, p, seed):
    A = gen.uniform_pm1(m, l, p, seed, -16, 16)
    B = gen.uniform_pm1(l, n, p, seed + 1, -16, 16)
    return A, B, dev(A), dev(B)


def _raw(m, l, n, p, algo, cutoff, A, B, Cm):
    a, b, c = A.struct(), B.struct(), Cm.struct()
    return mp.load_library().mpgemm_noalloc(m, l, n, p, algo, cutoff, ctypes.byref(a),
                                            ctypes.byref(b), ctypes.byref(c))


@pytest.mark.parametrize("m,l,n,p,algo,cutoff,seed", [
    (200, 200, 200, 512, mp.WINOGRAD, 64, 101),    # two recursion levels
    (151, 170, 133, 256, mp.STRASSEN, 32, 103),    # odd sizes, peeled, two levels
    (70, 45, 90, 1024, mp.SIMPLE, 64, 105),        # no scratch needed
    (64, 97, 33, 128, mp.BLOCK, 64, 107),
])
def test_noalloc_matches_mpgemm_on_consecutive_calls(m, l, n, p, algo, cutoff, seed):
    """Two calls in a row (the second one finds the first one's temporaries
    in the scratch) give mpgemm's bits, and every output equals the oracle
    running the same algorithm."""
    Ah, Bh, A, B = _pair(m, l, n, p, seed)
    want = mp.DeviceMP.empty(m, n, p)
    mp.mpgemm(A, B, want, algo, cutoff)
    mp.check_status("mpgemm")
    want_h = want.to_host()
    for call in range(2):
        got = mp.DeviceMP.empty(m, n, p)
        mp.mpgemm_noalloc(A, B, got, algo, cutoff)
        mp.check_status("mpgemm_noalloc")
        got_h = got.to_host()
        assert_bits_equal(got_h, want_h, "noalloc call %d %s" % (call, (m, l, n, p, algo)))
    assert_bits_equal(got_h, orc.gemm(algo, Ah, Bh, cutoff=cutoff), "noalloc vs oracle")


def test_noalloc_empty_inner_dimension_gives_zeros():
    p, m, n = 256, 9, 14
    A = mp.DeviceMP.empty(m, 0, p)
    B = mp.DeviceMP.empty(0, n, p)
    Cm = dev(gen.uniform_pm1(m, n, p, 5))
    for _ in range(2):
        mp.mpgemm_noalloc(A, B, Cm, mp.WINOGRAD, 64)
        mp.check_status("noalloc l = 0")
        got = Cm.to_host()
        assert np.all(got.exp == gen.EXP_ZERO) and not got.limb.any() and not got.sign.any()


def test_noalloc_rejects_products_beyond_the_scratch():
    p, n = 512, 256
    _, _, A, B = _pair(n, n, n, p, 7)
    Cm = mp.DeviceMP.empty(n, n, p)
    assert mp.workspace_size(n, n, n, p, mp.WINOGRAD, 64) > mp.NOALLOC_SCRATCH_BYTES
    assert _raw(n, n, n, p, mp.WINOGRAD, 64, A, B, Cm) == -8        # MP_ERR_SCRATCH
    assert mp.load_library().mp_strerror(-8).startswith(b"product needs more")


def test_noalloc_refuses_exact_and_split_forms():
    p, m, l, n = 256, 8, 8, 8
    _, _, A, B = _pair(m, l, n, p, 9)
    Cm = mp.DeviceMP.empty(m, n, p)
    for algo in (mp.EXACT, mp.SPLIT):
        assert _raw(m, l, n, p, algo, 64, A, B, Cm) == -7           # MP_ERR_UNSUPPORTED
    assert _raw(m, l, n, p, 17, 64, A, B, Cm) == -1                 # MP_ERR_ARG


def test_noalloc_reports_range_overflow():
    """An exponent overflow inside a no-alloc product reaches mp_sync_status
    through the entry point's own static status word, as it would for
    mpgemm; the status is cleared once read."""
    p, m, l, n = 128, 4, 3, 5
    Ah = gen.uniform_pm1(m, l, p, 11)
    Bh = gen.uniform_pm1(l, n, p, 12)
    Ah.exp[:] = (1 << 61) + 5
    Bh.exp[:] = (1 << 61) + 5
    Cm = mp.DeviceMP.empty(m, n, p)
    mp.mpgemm_noalloc(dev(Ah), dev(Bh), Cm, mp.SIMPLE, 64)
    assert mp.sync_status() == -6                                    # MP_ERR_RANGE
    assert mp.sync_status() == 0
