"""GPU elementwise arithmetic (the add/sub of the recursion's operand sums
and combinations, the multiply and the divide) against the CPU oracle, bit
for bit, and against IEEE double at p = 53."""
import random

import mpmath
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, dev
from tests.mpref import exact, from_mpf_list, man_exp, rn

pytestmark = pytest.mark.gpu

OPS = {"add": mp.OP_ADD, "sub": mp.OP_SUB, "mul": mp.OP_MUL, "div": mp.OP_DIV}


def _edge_pairs(p, n, seed):
    rnd = random.Random(seed)
    xs, ys = [], []
    for i in range(n):
        bx = rnd.randint(1, p)
        x = man_exp(rnd.getrandbits(bx) | 1, rnd.randint(-60, 60) - bx)
        kind = i % 8
        if kind == 0:
            y = man_exp(rnd.getrandbits(p) | 1, int(x._mpf_[2]) - rnd.randint(0, p + 70))
        elif kind == 1:
            y = exact(mpmath.libmp.mpf_add(mpmath.libmp.mpf_neg(x._mpf_),
                                           man_exp(rnd.getrandbits(8) | 1, int(x._mpf_[2]) - rnd.randint(0, 3))._mpf_))
        elif kind == 2:
            y = exact(mpmath.libmp.mpf_neg(x._mpf_))
        elif kind == 3:
            y = x
        elif kind == 4:   # ties: y is exactly half an ulp of x, or 1.5 ulp
            ex = int(x._mpf_[2]) + int(x._mpf_[3])
            y = man_exp(rnd.choice([1, 3]), ex - p - 1)
        elif kind == 5:
            y = exact(mpmath.libmp.fzero)
        else:
            y = man_exp(rnd.getrandbits(rnd.randint(1, p)) | 1, rnd.randint(-60, 60) - p)
        if rnd.random() < 0.5:
            x = exact(mpmath.libmp.mpf_neg(x._mpf_))
        if y._mpf_[3] > p:
            y = rn(y, p)
        xs.append(x)
        ys.append(y)
    X = from_mpf_list(xs, p, (1, n))
    Y = from_mpf_list(ys, p, (1, n))
    # a few signed zeros on both sides
    X.sign[0, :4] = [0, 1, 1, 0]
    X.exp[0, :4] = gen.EXP_ZERO
    X.limb[:, 0, :4] = 0
    Y.exp[0, :4] = gen.EXP_ZERO
    Y.limb[:, 0, :4] = 0
    Y.sign[0, :4] = [1, 1, 0, 0]
    return X, Y


@pytest.mark.parametrize("p", [2, 53, 64, 127, 128, 200, 256, 300, 512, 1000, 1024, 2048,
                               2049, 4000, 8192, 8650, 8704])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_elementwise_matches_oracle(op, p):
    n = 2000 if p <= 1024 else (600 if p <= 2048 else 150)
    X, Y = _edge_pairs(p, n, p * 13 + len(op))
    if op == "div":
        z = Y.exp == gen.EXP_ZERO
        Y.exp[z] = 1
        Y.limb[0][z] = np.uint64(1 << 63)
    # plus a block of generator values with a wide exponent spread
    U = gen.uniform_pm1(1, 500, p, 5, -40, 40)
    V = gen.uniform_pm1(1, 500, p, 6, -40, 40)
    if op == "div":                      # small p draws exact zeros often
        z = V.exp == gen.EXP_ZERO
        V.exp[z] = 3
        V.limb[0][z] = np.uint64(1 << 63)
    for A, B in ((X, Y), (U, V)):
        want, rc = orc.scalar(op, A, B)
        assert rc == 0
        dR = mp.DeviceMP.empty(1, A.shape[1], p)
        mp.elementwise(OPS[op], dev(A), dev(B), dR)
        mp.check_status(op)
        assert_bits_equal(dR.to_host(), want, "%s p=%d" % (op, p))


@pytest.mark.parametrize("p", [2, 53, 64, 127, 128, 200, 256, 300, 512, 1000, 1024])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_warp_elementwise_matches_oracle(op, p):
    """ops 4..7: the warp-cooperative add, subtract, multiply and divide of
    the LU solves (one warp per element, lane = word) on the same edge-case
    pairs (ties, carries, cancellation, exponent gaps, zeros) and wide
    exponent spreads; every bit equals the oracle's."""
    X, Y = _edge_pairs(p, 700, p * 17 + len(op))
    if op == "div":
        z = Y.exp == gen.EXP_ZERO
        Y.exp[z] = 1
        Y.limb[0][z] = np.uint64(1 << 63)
    U = gen.uniform_pm1(1, 300, p, 7, -40, 40)
    V = gen.uniform_pm1(1, 300, p, 8, -40, 40)
    if op == "div":
        z = V.exp == gen.EXP_ZERO
        V.exp[z] = 3
        V.limb[0][z] = np.uint64(1 << 63)
    for A, B in ((X, Y), (U, V)):
        want, rc = orc.scalar(op, A, B)
        assert rc == 0
        dR = mp.DeviceMP.empty(1, A.shape[1], p)
        mp.elementwise(OPS[op] + 4, dev(A), dev(B), dR)
        mp.check_status(op)
        assert_bits_equal(dR.to_host(), want, "warp %s p=%d" % (op, p))


def test_warp_elementwise_rejects_wide():
    A = gen.uniform_pm1(1, 4, 2048, 1)
    dR = mp.DeviceMP.empty(1, 4, 2048)
    with pytest.raises(mp.MPError) as e:
        mp.elementwise(4, dev(A), dev(A), dR)
    assert e.value.code == -7


@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_p53_matches_ieee_double(op):
    rng = np.random.default_rng(17)
    n = 4096
    a = rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, n))
    b = rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, n))
    b[:300] = -a[:300]
    b[300:600] = a[300:600] * 2.0 ** -53
    X = from_mpf_list([exact(mpmath.libmp.from_float(float(v))) for v in a], 53, (1, n))
    Y = from_mpf_list([exact(mpmath.libmp.from_float(float(v))) for v in b], 53, (1, n))
    dR = mp.DeviceMP.empty(1, n, 53)
    mp.elementwise(OPS[op], dev(X), dev(Y), dR)
    mp.check_status(op)
    R = dR.to_host()
    ref = {"add": a + b, "sub": a - b, "mul": a * b, "div": a / b}[op]
    got = np.array([float(gen.entry_fraction(R, 0, i)) for i in range(n)])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("pf,pt", [(256, 512), (512, 256), (2048, 128), (128, 2048), (200, 199),
                                   (8650, 4000), (4000, 8650), (8704, 8192), (1024, 8650)])
def test_convert_matches_oracle(pf, pt):
    X = gen.uniform_pm1(7, 33, pf, 9, -30, 30)
    want = orc.convert(X, pt)
    dR = mp.DeviceMP.empty(7, 33, pt)
    mp.convert(dev(X), dR)
    mp.check_status("convert")
    assert_bits_equal(dR.to_host(), want, "convert")


def test_division_by_zero_is_reported():
    X = gen.uniform_pm1(1, 8, 256, 1)
    Y = gen.HostMP.zeros(1, 8, 256)
    dR = mp.DeviceMP.empty(1, 8, 256)
    mp.elementwise(mp.OP_DIV, dev(X), dev(Y), dR)
    assert mp.sync_status() == -1
    assert mp.sync_status() == 0        # the status is cleared once read


def test_range_overflow_is_reported():
    p = 128
    X = gen.uniform_pm1(1, 4, p, 1)
    X.exp[:] = (1 << 61) + 5
    dR = mp.DeviceMP.empty(1, 4, p)
    mp.elementwise(mp.OP_MUL, dev(X), dev(X), dR)
    assert mp.sync_status() == -6
    want, _ = orc.scalar("mul", X, X)
    assert orc.range_error() == 1


def _words_number(words_le, p, e, sign=0):
    """Interchange entry from little-endian 32-bit words (mantissa of 32*len bits)."""
    N = 0
    for i, w in enumerate(words_le):
        N |= (w & 0xFFFFFFFF) << (32 * i)
    bl = N.bit_length()
    return (sign, N, bl - e)     # value N * 2^(e - bl): fraction N/2^bl times 2^e


@pytest.mark.parametrize("p", [128, 256, 512])
def test_mul_truncation_boundaries(p):
    """Products whose truncated partial sum cannot decide the rounding: the
    word under the mantissa sits just below the round bit, exactly on a tie,
    or just above it, with and without a nonzero tail.  a and b have only
    their top and bottom 32-bit words set, so the omitted partial product is
    a0*b0 alone."""
    W = p // 32
    cases = []
    for s_top, a0, b0 in [(0xFFFFFFFF, 0x40000000, 0x40000001),   # w = 0x7fffffff, tail != 0
                          (0xFFFFFFFF, 0x80000000, 0x00000000),   # w = 0x80000000, no tail: tie
                          (0xFFFFFFFF, 0x7FFFFFFF, 0x00000001),   # w = 0x80000000 after carry
                          (0xFFFFFFFF, 0x00000003, 0x7FFFFFF0),
                          (0x80000000, 0x80000000, 0x00000000),   # product < 1/2: shifted case
                          (0x80000001, 0x3FFFFFFF, 0x40000001)]:
        a = [a0] + [0] * (W - 2) + [s_top]
        b = [b0] + [0] * (W - 2) + [s_top]
        cases.append((a, b))
    xs = [_words_number(a, p, 1) for a, b in cases]
    ys = [_words_number(b, p, -3, 1) for a, b in cases]
    X = gen.from_exact_ints(xs, p, (1, len(xs)))
    Y = gen.from_exact_ints(ys, p, (1, len(ys)))
    want, rc = orc.scalar("mul", X, Y)
    dR = mp.DeviceMP.empty(1, len(xs), p)
    mp.elementwise(mp.OP_MUL, dev(X), dev(Y), dR)
    mp.check_status("mul boundaries")
    assert_bits_equal(dR.to_host(), want, "mul boundaries p=%d" % p)
