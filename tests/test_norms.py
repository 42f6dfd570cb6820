"""The log-space matrix norms used for Sec. 4's condition numbers, pinned on
matrices whose norms are known exactly: the inverse of the Hilbert matrix
(integer entries (-1)^(i+j) (i+j-1) C(n+i-1, n-j) C(n+j-1, n-i) C(i+j-2, i-1)^2,
1-based), checked against H H^-1 = I in exact rationals, and matrices with
zeros and exponents far outside double range."""
from fractions import Fraction
from math import comb, log2

import numpy as np

from paper_1410_1599_gb300 import inputs as gen
from paper_1410_1599_gb300 import norms


def hilbert_inverse(n):
    return [[(-1) ** (i + j) * (i + j - 1) * comb(n + i - 1, n - j) * comb(n + j - 1, n - i)
             * comb(i + j - 2, i - 1) ** 2 for j in range(1, n + 1)] for i in range(1, n + 1)]


def test_hilbert_inverse_is_the_inverse():
    n = 7
    Hi = hilbert_inverse(n)
    for i in range(n):
        for k in range(n):
            s = sum(Fraction(1, i + j + 1) * Hi[j][k] for j in range(n))
            assert s == (1 if i == k else 0)


def test_norm1_of_hilbert_inverse():
    for n, p in ((6, 128), (12, 256), (18, 512)):
        Hi = hilbert_inverse(n)
        M = gen.from_ints(Hi, p)
        exact = max(sum(abs(Hi[i][j]) for i in range(n)) for j in range(n))
        exact_inf = max(sum(abs(x) for x in row) for row in Hi)
        assert abs(norms.norm1_log2(M) - log2(exact)) < 1e-12 * max(1.0, log2(exact))
        assert abs(norms.norm_inf_log2(M) - log2(exact_inf)) < 1e-12 * max(1.0, log2(exact_inf))


def test_norms_with_zeros_and_huge_exponents():
    p = 256
    vals = [(0, 3, 0), (1, 5, 0), (0, 0, 0), (0, 7, -5000), (0, 1, -6000), (1, 1, -6000)]
    M = gen.from_exact_ints(vals, p, (3, 2))
    # columns: {3, 0, 2^6000}, {-5, 7 * 2^5000, -2^6000}
    col0 = log2(3 * 2 ** -6000 + 1) + 6000
    col1 = log2(5 * 2 ** -6000 + 7 * 2 ** -1000 + 1) + 6000
    assert abs(norms.norm1_log2(M) - max(col0, col1)) < 1e-9
    Z = gen.HostMP.zeros(4, 3, p)
    assert norms.norm1_log2(Z) == -np.inf


def test_regrouped_hilbert_inverse():
    """The oracle's form G_ij = (-1)^(i+j) a_i a_j / (i+j-1),
    a_i = (n+i-1)! / ((n-i)! ((i-1)!)^2), equals the binomial closed form."""
    from math import factorial
    for n in (1, 2, 5, 9):
        Hi = hilbert_inverse(n)
        a = [0] + [factorial(n + i - 1) // (factorial(n - i) * factorial(i - 1) ** 2) for i in range(1, n + 1)]
        for i in range(1, n + 1):
            for j in range(1, n + 1):
                assert Fraction((-1) ** (i + j) * a[i] * a[j], i + j - 1) == Hi[i - 1][j - 1]


def _exact_inverse(M):
    n = len(M)
    a = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for k in range(n):
        piv = next(i for i in range(k, n) if a[i][k] != 0)
        a[k], a[piv] = a[piv], a[k]
        inv = 1 / a[k][k]
        a[k] = [v * inv for v in a[k]]
        for i in range(n):
            if i != k and a[i][k] != 0:
                f = a[i][k]
                a[i] = [vi - f * vk for vi, vk in zip(a[i], a[k])]
    return [row[n:] for row in a]


def test_oracle_lotkin_condition_number():
    """The oracle's exact ||A||_1 and ||A^-1||_1 of the Lotkin matrix (Sec. 4)
    equal those of the inverse found by Gauss-Jordan elimination in exact
    rationals, and the golden values were written by the committed script."""
    import os
    from oracle import oracle as orc
    for n in (1, 2, 3, 6, 10, 14):
        A = [[Fraction(1)] * n] + [[Fraction(1, i + j + 1) for j in range(n)] for i in range(1, n)]
        Ai = _exact_inverse(A)
        n1 = lambda M: max(sum(abs(M[i][j]) for i in range(n)) for j in range(n))
        la, li = orc.lotkin_norm1_log2(n)
        assert abs(la - log2(n1(A))) < 1e-12 and abs(li - log2(n1(Ai))) < 1e-12 * max(1.0, li)
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lotkin_cond1.txt")
    rows = [ln.split() for ln in open(here) if not ln.startswith("#")]
    n, la10, li10, lc10 = rows[0]
    la, li = orc.lotkin_norm1_log2(int(n))
    assert abs(float(lc10) - (la + li) * 0.30102999566398120) < 1e-6
