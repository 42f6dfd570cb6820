"""The seeded generators: valid interchange encodings, reproducible, and
with the value distributions the workloads state."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1410_1599_gb300 import inputs as gen


def _valid(M):
    L = M.limb.shape[0]
    nz = M.exp != gen.EXP_ZERO
    top = (M.limb[0] >> np.uint64(63)) == 1
    assert (top | ~nz).all()
    assert (M.limb[:, ~nz] == 0).all()
    drop = 64 * L - M.p
    if drop:
        low = M.limb[L - 1] & np.uint64((1 << drop) - 1)
        assert (low == 0).all()


@pytest.mark.parametrize("p", [128, 200, 256, 512, 1024, 2048])
def test_uniform_valid_and_in_range(p):
    A = gen.uniform_pm1(40, 50, p, 7)
    _valid(A)
    fr = A.to_fractions()
    vals = [x for row in fr for x in row]
    assert all(-1 <= x < 1 for x in vals)
    grid = Fraction(1, 2 ** (p - 1))
    assert all((x / grid).denominator == 1 for x in vals)
    assert abs(float(sum(vals)) / len(vals)) < 0.05
    B = gen.uniform_pm1(40, 50, p, 7)
    assert A.equal(B)
    assert not A.equal(gen.uniform_pm1(40, 50, p, 8))


def test_uniform_scaled_exponents():
    A = gen.uniform_pm1(64, 64, 512, 3, -16, 16)
    _valid(A)
    scale = A.exp.astype(np.int64)
    assert scale.min() >= -16 - 40 and scale.max() <= 17


def test_extremes_reachable():
    # -1 is on the grid and encodes as mantissa 1/2, exponent 1, negative
    p = 128
    M = gen.from_exact_ints([(1, 1, 0)], p, (1, 1))
    assert gen.entry_fraction(M, 0, 0) == -1 and M.exp[0, 0] == 1


def test_well_conditioned_and_lotkin():
    n, p = 24, 256
    A = gen.well_conditioned(n, p, 5)
    _valid(A)
    fr = A.to_fractions()
    for i in range(n):
        assert n - 1 <= fr[i][i] < n + 1
        assert sum(abs(fr[j][i]) for j in range(n) if j != i) < abs(fr[i][i])  # column dominant
    L = gen.lotkin(n, p)
    _valid(L)
    fl = L.to_fractions()
    assert all(x == 1 for x in fl[0])
    for i in range(1, n):
        for j in range(n):
            exact = Fraction(1, i + j + 1)
            assert abs(fl[i][j] - exact) <= exact / 2 ** p


@pytest.mark.parametrize("rows,cols,p", [(70, 130, 256), (3, 5000, 64), (41, 211, 1024), (9, 1000, 53)])
def test_uniform_generator_is_independent_of_chunking(monkeypatch, rows, cols, p):
    """The generator works through the entries in chunks; entry t always takes
    the draws t(L+1)+1 .. t(L+1)+L+1, so the matrix is the same for any chunk
    size (one pass, the default, and a tiny one)."""
    ref = None
    for chunk in (1 << 30, gen._CHUNK, 97):
        monkeypatch.setattr(gen, "_CHUNK", chunk)
        M = gen.uniform_pm1(rows, cols, p, 123, -16, 16)
        if ref is None:
            ref = M
        else:
            assert M.equal(ref), chunk
