"""The Section 4 benchmark matrices on the GPU: results bit-exact against
the oracle running the same algorithm, and the maximum relative errors at
n = 2048 against the values the paper prints
(tests/golden/sqrt_matrix_errors.txt): Block and Strassen within a factor
of 10, Strassen above Block.  Winograd is the exception: with
b_ij = sqrt(3)(n-i+1) as printed, the columns of B are all alike, so
S5 = B12 - B11 and S8 = S6 - B21 are exact zeros at every level, M5 = M7 = 0,
and Winograd's error drops to the Block level -- far below the 2.25e-35
(128 bits) and 3.92e-305 (1024 bits) the paper prints.  The test checks
that consequence of the printed formulas instead."""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, dev, rel_errors_vs_rows

pytestmark = pytest.mark.gpu

ALGOS = {"block": mp.BLOCK, "strassen": mp.STRASSEN, "winograd": mp.WINOGRAD}
ORC_ALGO = {mp.SIMPLE: orc.SIMPLE, mp.BLOCK: orc.BLOCK, mp.STRASSEN: orc.STRASSEN, mp.WINOGRAD: orc.WINOGRAD}


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "sqrt_matrix_errors.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        bits, algo, which, v = line.split()
        out[(int(bits), algo, which)] = float(v)
    return out


@pytest.fixture
def mixed_policy():
    mp.set_odd_policy(mp.MIXED)
    yield
    mp.set_odd_policy(mp.PEEL)


@pytest.mark.parametrize("p", [128, 1024])
@pytest.mark.parametrize("algo", [mp.SIMPLE, mp.BLOCK, mp.STRASSEN, mp.WINOGRAD])
@pytest.mark.parametrize("dims", [(70, 70, 70), (65, 63, 67), (40, 100, 33)])
def test_sqrt_matrices_bit_exact(p, algo, dims, mixed_policy):
    m, l, n = dims
    A, B = gen.sqrt_matrices(m, l, n, p)
    dA, dB = dev(A), dev(B)
    dC = mp.DeviceMP.empty(m, n, p)
    mp.mpgemm(dA, dB, dC, algo, 16)
    mp.check_status("gemm")
    want = orc.gemm(ORC_ALGO[algo], A, B, cutoff=16, policy=orc.MIXED)
    assert_bits_equal(dC.to_host(), want, "sqrt matrices %s algo %d p %d" % (dims, algo, p))


def test_error_routine_matches_oracle(mixed_policy):
    """The device-side error reading equals the oracle's exact errors."""
    m = l = n = 40
    A, B = gen.sqrt_matrices(m, l, n, 128)
    dC = mp.DeviceMP.empty(m, n, 128)
    mp.mpgemm(dev(A), dev(B), dC, mp.WINOGRAD, 8)
    mp.check_status("gemm")
    got = rel_errors_vs_rows(dC, orc.sqrt_product_rows(m, l, n, 256))
    want = orc.sqrt_rel_errors(dC.to_host(), m, l, n)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=0)


@pytest.mark.parametrize("p", [128, 1024])
def test_errors_match_the_paper(p, mixed_policy):
    n = 2048
    gold = _golden()
    A, B = gen.sqrt_matrices(n, n, n, p)
    dA, dB = dev(A), dev(B)
    R = orc.sqrt_product_rows(n, n, n, 2 * p)
    got = {}
    for name, algo in ALGOS.items():
        dC = mp.DeviceMP.empty(n, n, p)
        mp.mpgemm(dA, dB, dC, algo, 32)
        mp.check_status(name)
        e = rel_errors_vs_rows(dC, R)
        got[name] = (float(e.max()), float(e.min()))
    u = 2.0 ** -p
    for name in ("block", "strassen"):
        want = gold.get((p, name, "max"))
        if want is not None:
            # same order of magnitude: the paper rounds sqrt(5) before scaling
            # by (i+j-1) and its n is not stated
            assert want / 10 <= got[name][0] <= want * 10, (p, name, got[name][0], want)
    assert 0 < got["block"][1] <= got["block"][0] < got["strassen"][0]
    # Winograd with M5 = M7 = 0: an order of magnitude below Strassen, within
    # a few dozen units in the last place like Block
    assert got["winograd"][0] <= got["strassen"][0] / 10, got
    assert got["winograd"][0] <= 64 * u and got["block"][0] <= 64 * u, got
