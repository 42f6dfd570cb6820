"""The Section 4 benchmark matrices (a_ij = sqrt(5)(i+j-1), b_ij =
sqrt(3)(n-i+1)), the closed form of their exact product, and the oracle's
exact relative errors, each pinned to something other than itself."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import inputs as gen

mpmath = pytest.importorskip("mpmath")


def _value(sg, M, s):
    v = Fraction(M) / Fraction(2) ** s
    return -v if sg else v


def _half_ulp(M, s, p):
    # ulp of a p-bit value M 2^-s whose top bit is bit p-1 of M
    return Fraction(2) ** (M.bit_length() - p) / Fraction(2) ** s / 2


@pytest.mark.parametrize("p", [2, 3, 8, 53, 128, 1024])
def test_rn_sqrt_brackets_the_root(p):
    """RN_p(sqrt N): the exact root lies within half an ulp of the result
    (checked by squaring), and squares come out exact."""
    Ns = [1, 2, 3, 4, 5, 15, 20, 45, 63, 64, 65, 255, 4 ** 9 - 1, 5 * 2047 ** 2, 3 * 2049 ** 2, 10 ** 30 + 7]
    for N in Ns:
        sg, M, s = gen.rn_sqrt(N, p)
        assert sg == 0 and 0 < M < 2 ** p
        v, h = _value(0, M, s), _half_ulp(M, s, p)
        assert (v - h) ** 2 <= N <= (v + h) ** 2, (N, p)
        r = math.isqrt(N)
        if r * r == N and r.bit_length() <= p:
            assert v == r


@pytest.mark.parametrize("p", [64, 128, 256, 1024])
def test_rn_sqrt_matches_mpmath(p):
    """Second opinion: mpmath's correctly rounded square root at p bits."""
    with mpmath.workprec(p):
        for k in list(range(1, 40)) + [1023, 2048, 4097]:
            for c in (3, 5):
                sg, M, s = gen.rn_sqrt(c * k * k, p)
                want = mpmath.sqrt(mpmath.mpf(c * k * k))
                man, exp = want.man_exp
                assert Fraction(M) / Fraction(2) ** s == Fraction(int(man)) * Fraction(2) ** int(exp)


def test_sqrt_matrices_entries():
    """a_ij = RN(sqrt(5)(i+j-1)), b_ij = RN(sqrt(3)(n-i+1)) with 1-based
    indices and the literal n; b is constant along its rows; b = 0 and
    negative entries where l > n."""
    p = 128
    A, B = gen.sqrt_matrices(4, 9, 7, p)
    assert A.shape == (4, 9) and B.shape == (9, 7)
    for i in range(4):
        for j in range(9):
            want = _value(*gen.rn_sqrt(5 * (i + j + 1) ** 2, p))
            assert gen.entry_fraction(A, i, j) == want
    for i in range(9):
        k = 7 - (i + 1) + 1
        for j in range(7):
            got = gen.entry_fraction(B, i, j)
            if k == 0:
                assert got == 0 and B.exp[i, j] == gen.EXP_ZERO
            else:
                mag = _value(*gen.rn_sqrt(3 * k * k, p))
                assert got == (mag if k > 0 else -mag)
    # the magnitudes: sqrt(5) and sqrt(3) to double precision
    assert abs(float(gen.entry_fraction(A, 0, 0)) - math.sqrt(5)) < 1e-15
    assert abs(float(gen.entry_fraction(B, 6, 0)) - math.sqrt(3)) < 1e-15


@pytest.mark.parametrize("m,l,n", [(1, 1, 1), (5, 7, 6), (12, 64, 12), (3, 10, 4), (30, 65, 1024)])
def test_product_S_closed_form(m, l, n):
    """S_i = sum_k (i+k-1)(n-k+1) against the polynomial
    (i-1)(l(n+1) - l(l+1)/2) + (n+1) l(l+1)/2 - l(l+1)(2l+1)/6."""
    S = orc.sqrt_product_S(m, l, n)
    for i in range(1, m + 1):
        poly = (i - 1) * (l * (n + 1) - l * (l + 1) // 2) + (n + 1) * l * (l + 1) // 2 \
            - l * (l + 1) * (2 * l + 1) // 6
        assert S[i - 1] == poly


@pytest.mark.parametrize("q", [64, 128, 512, 2048])
def test_product_rows_rounded_once(q):
    """RN_q(sqrt(15) S_i): within half an ulp of the exact value (squared
    comparison), and mpmath agrees."""
    m, l, n = 6, 9, 8
    S = orc.sqrt_product_S(m, l, n)
    R = orc.sqrt_product_rows(m, l, n, q)
    for i in range(m):
        v = gen.entry_fraction(R, i, 0)
        L = R.limb.shape[0]
        M = 0
        for k in range(L):
            M = (M << 64) | int(R.limb[k, i, 0])
        M >>= 64 * L - q
        h = Fraction(2) ** (int(R.exp[i, 0]) - q) / 2
        assert (abs(v) - h) ** 2 <= 15 * S[i] ** 2 <= (abs(v) + h) ** 2
        with mpmath.workprec(q):
            want = mpmath.sqrt(mpmath.mpf(15 * S[i] ** 2))
            man, exp = want.man_exp
            assert v == Fraction(int(man)) * Fraction(2) ** int(exp)


def test_rel_errors_pinned():
    """The exact-error routine on constructed results: the correctly rounded
    product has error <= 2^-p (and > 0: sqrt(15) is irrational); one ulp
    more adds 2^(1-p)-ish; a wrong sign gives 1 + |x|/sqrt(15) = 2; mpmath
    at 600 bits gives the same numbers to double precision."""
    m, l, n, p = 4, 5, 3, 128
    R = orc.sqrt_product_rows(m, l, n, p)
    C = orc.OMat(np.repeat(R.limb, n, axis=2), np.repeat(R.exp, n, axis=1), np.repeat(R.sign, n, axis=1), p)
    e = orc.sqrt_rel_errors(C, m, l, n)
    assert (e > 0).all() and (e <= 2.0 ** -p).all()
    # one ulp up in entry (1, 2), sign flipped in entry (2, 0)
    L = C.limb.shape[0]
    C.limb[L - 1, 1, 2] += np.uint64(1 << (64 * L - p))
    C.sign[2, 0] = 1
    e2 = orc.sqrt_rel_errors(C, m, l, n)
    S = orc.sqrt_product_S(m, l, n)
    with mpmath.workprec(600):
        for (i, j) in [(1, 2), (0, 0), (3, 1)]:
            x = mpmath.mpf(0)
            for k in range(L):
                x = x * 2 ** 64 + int(C.limb[k, i, j])
            x = x / mpmath.mpf(2) ** (64 * L) * mpmath.mpf(2) ** int(C.exp[i, j])
            true = mpmath.sqrt(15) * S[i]
            want = float(abs(x - true) / true)
            assert e2[i, j] == pytest.approx(want, rel=1e-12)
    assert e2[1, 2] > 2.0 ** -p
    assert e2[2, 0] == pytest.approx(2.0, rel=1e-15)


@pytest.mark.parametrize("n", [24, 33])
def test_oracle_errors_on_sqrt_matrices(n):
    """Simple/Block on the Section 4 matrices: all terms positive, so the
    relative error obeys the summation bound gamma_{l+2} = (l+2)u/(1-(l+2)u),
    u = 2^-p (inputs rounded once, one rounding per multiply and per add);
    Block reproduces Simple bit for bit.  Strassen and Winograd (mixed odd
    policy, n_min = 8) stay below the same bound times the growth of their
    operand sums (a loose factor 2^10 here)."""
    p = 128
    A, B = gen.sqrt_matrices(n, n, n, p)
    u = 2.0 ** -p
    g = (n + 2) * u / (1 - (n + 2) * u)
    Cs = orc.gemm(orc.SIMPLE, A, B)
    es = orc.sqrt_rel_errors(Cs, n, n, n)
    assert es.max() <= g and es.max() > 0
    Cb = orc.gemm(orc.BLOCK, A, B, nb=8)
    assert np.array_equal(Cb.limb, Cs.limb) and np.array_equal(Cb.exp, Cs.exp)
    for algo in (orc.STRASSEN, orc.WINOGRAD):
        C = orc.gemm(algo, A, B, cutoff=8, policy=orc.MIXED)
        e = orc.sqrt_rel_errors(C, n, n, n)
        assert 0 < e.max() <= 1024 * g
