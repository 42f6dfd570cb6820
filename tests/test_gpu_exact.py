"""MP_EXACT: every c_ij the exact dot product rounded once, against the
oracle's correctly rounded exact dot product (bit for bit)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, gemm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [53, 128, 200, 256, 512, 1024, 2048])
@pytest.mark.parametrize("spread", [0, 16, 40])
def test_exact_matches_oracle(p, spread):
    m, l, n = (19, 37, 23) if p >= 1024 else (41, 77, 35)
    A = gen.uniform_pm1(m, l, p, 61, -spread, spread)
    B = gen.uniform_pm1(l, n, p, 62, -spread, spread)
    want = orc.dot_exact(A, B)
    assert_bits_equal(gemm(A, B, mp.EXACT), want, "exact p=%d spread=%d" % (p, spread))


def test_exact_cancellation_and_zero():
    p = 256
    A = gen.from_ints([[3, -3, 5, -5, 0], [1, 2, 3, 4, 5]], p)
    B = gen.from_ints([[7], [7], [1], [1], [9]], p)
    got = gemm(A, B, mp.EXACT)
    want = orc.dot_exact(A, B)
    assert_bits_equal(got, want, "cancellation")
    assert got.exp[0, 0] == gen.EXP_ZERO and got.sign[0, 0] == 0
