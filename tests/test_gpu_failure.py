"""Failure detection on the device without a fault: the library's bounded
mbarrier wait (the one the split form's slice kernel and the TMA-staged
Block kernel use) is made to run out on a barrier that nothing completes;
the timeout comes back as MP_ERR_TIMEOUT through the status word, and the
device stays usable: the next product matches the oracle bit for bit."""
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, gemm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cycles", [1, 100_000, 20_000_000])
def test_bounded_wait_reports_timeout(cycles):
    assert mp.wait_selftest(cycles) == -4                 # MP_ERR_TIMEOUT
    assert mp.sync_status() == 0                          # reported once, then cleared


def test_device_usable_after_timeout():
    assert mp.wait_selftest(1_000_000) == -4
    A = gen.uniform_pm1(70, 66, 512, 91, -16, 16)
    B = gen.uniform_pm1(66, 98, 512, 92, -16, 16)
    assert_bits_equal(gemm(A, B, mp.WINOGRAD, 16), orc.gemm(mp.WINOGRAD, A, B, cutoff=16), "after timeout")


def test_selftest_limit_range():
    lib = mp.load_library()
    assert lib.mp_wait_selftest(0) == -1
    assert lib.mp_wait_selftest((1 << 32) + 1) == -1
