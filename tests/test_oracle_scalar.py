"""Pins of the oracle's scalar arithmetic (round to nearest, ties to even,
after every operation; arXiv 1410.1599 Sec. 1/Sec. 3, MPFR semantics).

References that are not the oracle itself:
  * IEEE 754 binary64 hardware arithmetic: at p = 53 the oracle must
    reproduce numpy float64 +, -, *, / bit for bit (both are correctly
    rounded to nearest-even; exponents stay far from the double range);
  * mpmath's libmpf (mpf_add/mpf_mul/mpf_div at precision p, round_nearest)
    at p in {128, 200, 256, 512, 1024, 2048};
  * hand-built tie, carry-out and cancellation cases with closed-form answers.
"""
import random

import mpmath
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300.inputs import EXP_ZERO, HostMP, from_exact_ints
from tests.mpref import (entry_mpf, exact, from_mpf_list, man_exp, mp_add, mp_div, mp_mul,
                         mp_sub, put_mpf, rn)

OPS = {"add": mp_add, "sub": mp_sub, "mul": mp_mul, "div": mp_div}


def _doubles_to_hostmp(vals, p=53):
    return from_mpf_list([exact(mpmath.libmp.from_float(float(v))) for v in vals], p, (1, len(vals)))


@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_p53_matches_ieee_double(op):
    rng = np.random.default_rng(11)
    n = 3000
    # mixed magnitudes: exponent gaps 0..60 and exact cancellations
    a = rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))
    b = rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))
    b[:200] = -a[:200]                    # x - x and x + (-x)
    b[200:400] = a[200:400] * (1 + 2.0 ** -52)
    b[400:600] = a[400:600] * 2.0 ** -53  # half-ulp ties for add
    if op == "div":
        b[b == 0] = 1.0
    X, Y = _doubles_to_hostmp(a), _doubles_to_hostmp(b)
    R, rc = orc.scalar(op, X, Y)
    assert rc == 0
    with np.errstate(all="ignore"):
        ref = {"add": a + b, "sub": a - b, "mul": a * b, "div": a / b}[op]
    got = np.array([float(entry_mpf(R, 0, i)) for i in range(n)])
    assert np.array_equal(got, ref), np.nonzero(got != ref)[0][:10]


@pytest.mark.parametrize("p", [128, 200, 256, 512, 1024, 2048, 4000, 8192, 8650, 8704])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_matches_mpmath(op, p):
    rnd = random.Random(p * 7 + len(op))
    n = 300 if p <= 512 else (120 if p <= 2048 else 40)
    xs, ys = [], []
    for i in range(n):
        bx = rnd.randint(1, p)
        x = man_exp(rnd.getrandbits(bx) | 1, rnd.randint(-40, 40) - bx)
        kind = i % 6
        if kind == 0:      # large exponent gap, up to past p + 2
            gap = rnd.randint(0, p + 5)
            y = man_exp(rnd.getrandbits(p) | 1, int(x._mpf_[2]) - gap)
        elif kind == 1:    # near cancellation
            y = exact(mpmath.libmp.mpf_add(mpmath.libmp.mpf_neg(x._mpf_), man_exp(rnd.getrandbits(8) | 1, int(x._mpf_[2]) - rnd.randint(0, 3))._mpf_))
        elif kind == 2:
            y = exact(mpmath.libmp.mpf_neg(x._mpf_))
        else:
            y = man_exp(rnd.getrandbits(rnd.randint(1, p)) | 1, rnd.randint(-40, 40) - p)
        if rnd.random() < 0.5:
            x = exact(mpmath.libmp.mpf_neg(x._mpf_))
        # keep both within p bits
        assert x._mpf_[3] <= p
        if y._mpf_[3] > p:
            y = rn(y, p)
        xs.append(x)
        ys.append(y if not (op == "div" and y._mpf_ == mpmath.libmp.fzero) else man_exp(3, 0))
    X = from_mpf_list(xs, p, (1, n))
    Y = from_mpf_list(ys, p, (1, n))
    R, rc = orc.scalar(op, X, Y)
    assert rc == 0
    for i in range(n):
        ref = OPS[op](xs[i], ys[i], p)
        assert entry_mpf(R, 0, i) == ref, (i, xs[i], ys[i])
    assert orc.range_error() == 0


def _one(p, vals):
    return from_exact_ints(vals, p, (1, len(vals)))


def test_ties_to_even_closed_form():
    p = 128
    # 1 + 2^-p: exactly half an ulp above 1 -> ties to 1 (even)
    # (1 + 2^(1-p)) + 2^-p: halfway between an odd and an even neighbour -> up
    X = _one(p, [(0, 1, 0), (0, (1 << (p - 1)) + 1, p - 1), (0, 1, 0)])
    Y = _one(p, [(0, 1, p), (0, 1, p), (0, 3, p + 1)])   # 3*2^(-p-1) > half ulp
    R, _ = orc.scalar("add", X, Y)
    assert entry_mpf(R, 0, 0) == man_exp(1, 0)
    assert entry_mpf(R, 0, 1) == man_exp((1 << (p - 2)) + 1, 2 - p)
    assert entry_mpf(R, 0, 2) == man_exp((1 << (p - 1)) + 1, 1 - p)


def test_carry_out_renormalises():
    p = 128
    allones = (1 << p) - 1                                   # (2^p - 1) 2^-p
    X = _one(p, [(0, allones, p)])
    Y = _one(p, [(0, 1, p + 1)])                             # half ulp: tie, round up to 1
    R, _ = orc.scalar("add", X, Y)
    assert entry_mpf(R, 0, 0) == man_exp(1, 0)
    assert R.exp[0, 0] == 1 and R.limb[0, 0, 0] == 1 << 63


def test_subtraction_below_power_of_two():
    # x = 1 (a power of two), y tiny: x - y rounds back to 1 when |y| is below
    # a quarter ulp of 1, and to the predecessor 1 - 2^-p when it is above.
    p = 128
    X = _one(p, [(0, 1, 0)] * 3)
    Y = _one(p, [(0, 1, p + 2), (0, 3, p + 2), (0, 1, p + 1)])
    R, _ = orc.scalar("sub", X, Y)
    assert entry_mpf(R, 0, 0) == man_exp(1, 0)
    assert entry_mpf(R, 0, 1) == man_exp((1 << p) - 1, -p)
    # exactly half of the lower spacing: tie between 1 - 2^-p (odd) and 1 (even)
    assert entry_mpf(R, 0, 2) == man_exp(1, 0)


def test_signed_zeros():
    p = 128
    z = HostMP.zeros(1, 4, p)
    z.sign[0, :] = [0, 1, 1, 0]          # +0, -0, -0, +0
    w = HostMP.zeros(1, 4, p)
    w.sign[0, :] = [1, 1, 0, 0]          # -0, -0, +0, +0
    R, _ = orc.scalar("add", z, w)
    assert list(R.sign[0]) == [0, 1, 0, 0]
    assert (R.exp == EXP_ZERO).all()
    x = _one(p, [(0, 5, 1), (1, 5, 1)])
    R, _ = orc.scalar("sub", x, x)
    assert (R.exp == EXP_ZERO).all() and list(R.sign[0]) == [0, 0]   # x - x = +0
    nz = HostMP.zeros(1, 2, p)
    nz.sign[0, :] = [1, 0]
    R, _ = orc.scalar("mul", x, nz)
    assert (R.exp == EXP_ZERO).all() and list(R.sign[0]) == [1, 1]   # sign is the xor


def test_division_by_zero_reported():
    p = 128
    x = _one(p, [(0, 1, 0)])
    R, rc = orc.scalar("div", x, HostMP.zeros(1, 1, p))
    assert rc == -1


def test_convert_roundtrip_and_rounding():
    p = 256
    rnd = random.Random(5)
    vals = [man_exp((rnd.getrandbits(256) | (1 << 255)) * rnd.choice((1, -1)), -256 - rnd.randint(0, 9))
            for _ in range(50)]
    X = from_mpf_list(vals, p, (1, 50))
    W = orc.convert(X, 512)
    assert all(entry_mpf(W, 0, i) == vals[i] for i in range(50))
    N = orc.convert(X, 128)
    for i in range(50):
        assert entry_mpf(N, 0, i) == rn(vals[i], 128)


def test_search_for_disagreements_with_mpmath():
    """A shrinking search (hypothesis) over precisions, mantissa lengths,
    exponent gaps and signs for any disagreement with mpmath's correctly
    rounded add, sub, mul and div."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=400, deadline=None, derandomize=True)
    @hyp.given(st.integers(2, 700), st.integers(1, 700), st.integers(1, 700), st.integers(0, 2 ** 700),
               st.integers(0, 2 ** 700), st.integers(-720, 720), st.booleans(), st.booleans(),
               st.sampled_from(["add", "sub", "mul", "div"]))
    def check(p, bx, by, mx, my, gap, nx, ny, op):
        bx, by = min(bx, p), min(by, p)
        mx = (mx % (1 << bx)) | (1 << (bx - 1))       # exactly bx significant bits
        my = (my % (1 << by)) | (1 << (by - 1))
        x = man_exp(-mx if nx else mx, -bx)
        y = man_exp(-my if ny else my, gap - by)
        X, Y = from_mpf_list([x], p, (1, 1)), from_mpf_list([y], p, (1, 1))
        R, rc = orc.scalar(op, X, Y)
        assert rc == 0
        assert entry_mpf(R, 0, 0) == OPS[op](x, y, p), (p, x, y, op)

    check()
