"""Pins of the oracle's GEMM algorithms (arXiv 1410.1599 Sec. 2).

What pins them, other than the oracle itself:
  * Table 1 of the paper (tests/golden/table1.txt): the operation-count
    ratios at n_min = 32, reproduced by the oracle's instrumented counters
    (through the count model, which is first checked against the counters);
  * mathematics: with small integer entries every intermediate is exact, so
    Strassen and Winograd must equal Simple bit for bit; A I = A and I B = B
    exactly for Simple/Block; Block == Simple (same k-ascending sequence);
  * an exact rational product for dyadic inputs;
  * an independent replay of the printed formulas with mpmath scalar
    operations on tiny matrices (odd sizes, padding and peeling);
  * the error bound of recursive multiplication (Higham) on random inputs.
"""
import os

import mpmath
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import inputs as gen
from tests.mpref import entry_mpf, mp_add, mp_mul, mp_sub

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def _table1():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, a, b, c, d = line.split()
        rows.append((int(n), float(a), float(b), float(c), float(d)))
    return rows


@pytest.mark.parametrize("algo", [orc.STRASSEN, orc.WINOGRAD])
@pytest.mark.parametrize("policy", [orc.PEEL, orc.MIXED])
@pytest.mark.parametrize("dims,cutoff", [((33, 33, 33), 8), ((40, 27, 35), 6), ((64, 64, 64), 16),
                                         ((31, 45, 19), 4), ((50, 50, 50), 7)])
def test_counters_equal_count_model(algo, policy, dims, cutoff):
    m, l, n = dims
    A = gen.uniform_pm1(m, l, 128, 21)
    B = gen.uniform_pm1(l, n, 128, 22)
    _, mul, add = orc.gemm_counted(algo, A, B, cutoff=cutoff, policy=policy)
    assert (mul, add) == orc.count_model(algo, m, l, n, cutoff, policy)


def test_table1_reproduced():
    """All 48 printed ratios, with the header read as (Mul, Add&Sub)."""
    hits = 0
    for n, s_mul, s_add, w_mul, w_add in _table1():
        base = n ** 3
        sm, sa = orc.count_model(orc.STRASSEN, n, n, n, 32, orc.MIXED)
        wm, wa = orc.count_model(orc.WINOGRAD, n, n, n, 32, orc.MIXED)
        for got, want in ((sm, s_mul), (sa, s_add), (wm, w_mul), (wa, w_add)):
            assert round(got / base, 3) == pytest.approx(want, abs=1e-12), (n, got / base, want)
            hits += 1
    assert hits == 48


def test_table1_not_reproduced_by_peel_only():
    # the padding half of the mixed rule matters: peel-only misses some rows
    misses = 0
    for n, s_mul, s_add, w_mul, w_add in _table1():
        sm, sa = orc.count_model(orc.STRASSEN, n, n, n, 32, orc.PEEL)
        misses += round(sm / n ** 3, 3) != s_mul or round(sa / n ** 3, 3) != s_add
    assert misses > 0


@pytest.mark.parametrize("algo", [orc.STRASSEN, orc.WINOGRAD])
@pytest.mark.parametrize("policy", [orc.PEEL, orc.MIXED])
@pytest.mark.parametrize("dims,cutoff", [((1, 1, 1), 1), ((2, 3, 5), 1), ((17, 17, 17), 4),
                                         ((37, 23, 41), 5), ((64, 64, 64), 8), ((65, 63, 66), 8),
                                         ((130, 97, 71), 16)])
def test_integer_inputs_reproduce_simple(algo, policy, dims, cutoff):
    m, l, n = dims
    A = gen.small_ints(m, l, 256, 31, bits=20)
    B = gen.small_ints(l, n, 256, 32, bits=20)
    S = orc.gemm(orc.SIMPLE, A, B)
    R = orc.gemm(algo, A, B, cutoff=cutoff, policy=policy)
    assert np.array_equal(S.limb, R.limb) and np.array_equal(S.exp, R.exp)
    assert np.array_equal(S.sign, R.sign)


@pytest.mark.parametrize("p", [4000, 8650])
def test_wide_precision_integer_and_replay(p):
    """Above 2048 bits: Strassen and Winograd reproduce Simple on integer
    inputs, and an mpmath replay of Winograd's printed formulas on random
    p-bit inputs gives the same bits."""
    A = gen.small_ints(9, 11, p, 33, bits=20)
    B = gen.small_ints(11, 10, p, 34, bits=20)
    S = orc.gemm(orc.SIMPLE, A, B)
    for algo in (orc.STRASSEN, orc.WINOGRAD):
        R = orc.gemm(algo, A, B, cutoff=2, policy=orc.MIXED)
        assert np.array_equal(S.limb, R.limb) and np.array_equal(S.exp, R.exp)
    X = gen.uniform_pm1(5, 7, p, 35, -8, 8)
    Y = gen.uniform_pm1(7, 6, p, 36, -8, 8)
    for algo in (orc.SIMPLE, orc.WINOGRAD):
        R = orc.gemm(algo, X, Y, cutoff=2, policy=orc.PEEL)
        ref = _simple(_mat(X), _mat(Y), p) if algo == orc.SIMPLE else \
            _rec(_mat(X), _mat(Y), p, algo, 2, orc.PEEL, 5, 7, 6)
        for i in range(5):
            for j in range(6):
                assert entry_mpf(R, i, j) == ref[i][j], (algo, i, j)


def test_block_equals_simple_and_identity():
    p = 256
    A = gen.uniform_pm1(45, 37, p, 41, -16, 16)
    B = gen.uniform_pm1(37, 29, p, 42, -16, 16)
    S = orc.gemm(orc.SIMPLE, A, B)
    for nb in (1, 7, 16, 32, 64):
        Bl = orc.gemm(orc.BLOCK, A, B, nb=nb)
        assert np.array_equal(S.limb, Bl.limb) and np.array_equal(S.exp, Bl.exp)
        assert np.array_equal(S.sign, Bl.sign)
    I37, I45 = gen.identity(37, p), gen.identity(45, p)
    for algo in (orc.SIMPLE, orc.BLOCK):
        AI = orc.gemm(algo, A, I37)
        IA = orc.gemm(algo, I45, A)
        for R in (AI, IA):
            assert np.array_equal(R.limb, A.limb) and np.array_equal(R.exp, A.exp)
            nz = A.exp != gen.EXP_ZERO
            assert np.array_equal(R.sign[nz], A.sign[nz])


def test_exact_rational_product():
    # dyadic entries with 6 significant bits: every sum and product is exact at 256 bits
    rng = np.random.default_rng(3)
    m, l, n = 7, 9, 5
    a = rng.integers(-63, 64, (m, l))
    b = rng.integers(-63, 64, (l, n))
    sa, sb = rng.integers(0, 9, (m, l)), rng.integers(0, 9, (l, n))
    A = gen.from_exact_ints([(int(x < 0), abs(int(x)), int(s)) for x, s in zip(a.ravel(), sa.ravel())], 256, (m, l))
    B = gen.from_exact_ints([(int(x < 0), abs(int(x)), int(s)) for x, s in zip(b.ravel(), sb.ravel())], 256, (l, n))
    FA, FB = A.to_fractions(), B.to_fractions()
    for algo in (orc.SIMPLE, orc.STRASSEN, orc.WINOGRAD):
        R = orc.gemm(algo, A, B, cutoff=1)
        for i in range(m):
            for j in range(n):
                ref = sum(FA[i][k] * FB[k][j] for k in range(l))
                assert gen.entry_fraction(R, i, j) == ref


def test_empty_and_degenerate_shapes():
    p = 128
    A = gen.uniform_pm1(3, 0, p, 1)
    B = gen.uniform_pm1(0, 4, p, 2)
    for algo in (orc.SIMPLE, orc.BLOCK, orc.STRASSEN, orc.WINOGRAD):
        R = orc.gemm(algo, A, B, cutoff=1)
        assert (R.exp == gen.EXP_ZERO).all() and (R.sign == 0).all()
    A = gen.uniform_pm1(1, 1, p, 1)
    B = gen.uniform_pm1(1, 1, p, 2)
    R = orc.gemm(orc.WINOGRAD, A, B, cutoff=1)
    assert entry_mpf(R, 0, 0) == mp_mul(entry_mpf(A, 0, 0), entry_mpf(B, 0, 0), p)


# ---------------------------------------------------------------------------
# independent replay of the printed formulas with mpmath scalar arithmetic
# ---------------------------------------------------------------------------
def _mat(M):
    return [[entry_mpf(M, i, j) for j in range(M.shape[1])] for i in range(M.shape[0])]


def _addm(X, Y, p, s=1):
    f = mp_add if s > 0 else mp_sub
    return [[f(x, y, p) for x, y in zip(rx, ry)] for rx, ry in zip(X, Y)]


def _simple(X, Y, p):
    m, l, n = len(X), len(Y), len(Y[0]) if Y else 0
    out = []
    for i in range(m):
        row = []
        for j in range(n):
            c = mpmath.mpf(0)
            for k in range(l):
                c = mp_add(c, mp_mul(X[i][k], Y[k][j], p), p)
            row.append(c)
        out.append(row)
    return out


def _rec(X, Y, p, algo, cutoff, policy, m, l, n):
    if not (m > cutoff and l > cutoff and n > cutoff):
        return _simple(X, Y, p)

    def ev(x):
        if x % 2 == 0:
            return x
        return x + 1 if (policy == orc.MIXED and x % 4 == 3) else x - 1

    M, K, N = ev(m), ev(l), ev(n)
    z = mpmath.mpf(0)
    get = lambda Z, i, j, R, Cc: Z[i][j] if i < R and j < Cc else z
    h, k, w = M // 2, K // 2, N // 2
    q = lambda Z, R, Cc, r0, c0, rr, cc: [[get(Z, r0 + i, c0 + j, R, Cc) for j in range(cc)] for i in range(rr)]
    A11, A12 = q(X, m, l, 0, 0, h, k), q(X, m, l, 0, k, h, k)
    A21, A22 = q(X, m, l, h, 0, h, k), q(X, m, l, h, k, h, k)
    B11, B12 = q(Y, l, n, 0, 0, k, w), q(Y, l, n, 0, w, k, w)
    B21, B22 = q(Y, l, n, k, 0, k, w), q(Y, l, n, k, w, k, w)
    mul = lambda U, V: _rec(U, V, p, algo, cutoff, policy, h, k, w)
    if algo == orc.STRASSEN:
        P1 = mul(_addm(A11, A22, p), _addm(B11, B22, p))
        P2 = mul(_addm(A21, A22, p), B11)
        P3 = mul(A11, _addm(B12, B22, p, -1))
        P4 = mul(A22, _addm(B21, B11, p, -1))
        P5 = mul(_addm(A11, A12, p), B22)
        P6 = mul(_addm(A21, A11, p, -1), _addm(B11, B12, p))
        P7 = mul(_addm(A12, A22, p, -1), _addm(B21, B22, p))
        C11 = _addm(_addm(_addm(P1, P4, p), P5, p, -1), P7, p)
        C12 = _addm(P3, P5, p)
        C21 = _addm(P2, P4, p)
        C22 = _addm(_addm(_addm(P1, P3, p), P2, p, -1), P6, p)
    else:
        S1 = _addm(A21, A22, p); S2 = _addm(S1, A11, p, -1)
        S3 = _addm(A11, A21, p, -1); S4 = _addm(A12, S2, p, -1)
        S5 = _addm(B12, B11, p, -1); S6 = _addm(B22, S5, p, -1)
        S7 = _addm(B22, B12, p, -1); S8 = _addm(S6, B21, p, -1)
        M1, M2, M3 = mul(S2, S6), mul(A11, B11), mul(A12, B21)
        M4, M5, M6, M7 = mul(S3, S7), mul(S1, S5), mul(S4, B22), mul(A22, S8)
        T1 = _addm(M1, M2, p); T2 = _addm(T1, M4, p)
        C11 = _addm(M2, M3, p); C12 = _addm(_addm(T1, M5, p), M6, p)
        C21 = _addm(T2, M7, p, -1); C22 = _addm(T2, M5, p)
    C = [[None] * n for _ in range(m)]
    quads = [[C11, C12], [C21, C22]]
    mr, nr = min(M, m), min(N, n)
    for i in range(mr):
        for j in range(nr):
            C[i][j] = quads[i // h][j // w][i % h][j % w]
            if K < l:
                C[i][j] = mp_add(C[i][j], mp_mul(X[i][l - 1], Y[l - 1][j], p), p)
    full = _simple([X[m - 1]], Y, p)[0] if M < m else None
    if M < m:
        C[m - 1] = full
    if N < n:
        col = _simple(X[:mr], [[Y[t][n - 1]] for t in range(l)], p)
        for i in range(mr):
            C[i][n - 1] = col[i][0]
    return C


@pytest.mark.parametrize("algo", [orc.SIMPLE, orc.STRASSEN, orc.WINOGRAD])
@pytest.mark.parametrize("policy", [orc.PEEL, orc.MIXED])
@pytest.mark.parametrize("dims,cutoff", [((5, 7, 6), 2), ((8, 8, 8), 1), ((11, 9, 7), 2), ((7, 7, 7), 1)])
def test_replay_with_mpmath(algo, policy, dims, cutoff):
    p = 128
    m, l, n = dims
    A = gen.uniform_pm1(m, l, p, 51, -8, 8)
    B = gen.uniform_pm1(l, n, p, 52, -8, 8)
    R = orc.gemm(algo, A, B, cutoff=cutoff, policy=policy)
    ref = _rec(_mat(A), _mat(B), p, algo, cutoff, policy, m, l, n) if algo != orc.SIMPLE \
        else _simple(_mat(A), _mat(B), p)
    for i in range(m):
        for j in range(n):
            assert entry_mpf(R, i, j) == ref[i][j], (i, j)


# ---------------------------------------------------------------------------
# sampled recursion == full recursion
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("algo", [orc.STRASSEN, orc.WINOGRAD])
@pytest.mark.parametrize("policy", [orc.PEEL, orc.MIXED])
@pytest.mark.parametrize("dims,cutoff,seeds", [((67, 61, 70), 8, [(0, 0), (66, 69), (33, 12)]),
                                               ((64, 64, 64), 8, [(5, 9), (63, 63)]),
                                               ((45, 50, 39), 5, [(44, 38), (20, 3)])])
def test_sampled_equals_full(algo, policy, dims, cutoff, seeds):
    m, l, n = dims
    p = 192
    A = gen.uniform_pm1(m, l, p, 61, -16, 16)
    B = gen.uniform_pm1(l, n, p, 62, -16, 16)
    full = orc.gemm(algo, A, B, cutoff=cutoff, policy=policy)
    for i0, j0 in seeds:
        rows = orc.sample_set(0, algo, m, l, n, cutoff, policy, i0)
        cols = orc.sample_set(1, algo, m, l, n, cutoff, policy, j0)
        assert i0 in rows and j0 in cols
        S = orc.gemm_sampled(algo, A, B, rows, cols, cutoff=cutoff, policy=policy)
        ref = full.limb[:, rows[:, None], cols[None, :]]
        assert np.array_equal(S.limb, ref)
        assert np.array_equal(S.exp, full.exp[rows[:, None], cols[None, :]])
        assert np.array_equal(S.sign, full.sign[rows[:, None], cols[None, :]])


def test_sample_set_size_is_two_to_the_depth():
    rows = orc.sample_set(0, orc.WINOGRAD, 2048, 2048, 2048, 64, orc.PEEL, 5)
    assert len(rows) == 32 and all(r % 64 == 5 for r in rows)


# ---------------------------------------------------------------------------
# error against the exact product
# ---------------------------------------------------------------------------
def test_error_bounds_and_ordering():
    """Normwise error |C^ - C| / (|A||B|) against the exact product: Simple is
    within l*u (u = 2^-p); Strassen/Winograd within Higham's recursive bound
    (Accuracy and Stability, Thm 23.3/23.4 form: growth 12^d and 18^d level
    constants); their errors are larger than Simple's (stated, not hidden)."""
    p, n, cutoff = 128, 96, 12
    A = gen.uniform_pm1(n, n, p, 71)
    B = gen.uniform_pm1(n, n, p, 72)
    exact = orc.dot_exact(A, B, p_out=4 * p)
    Fabs = np.abs(orc.to_double(A)) @ np.abs(orc.to_double(B))
    errs = {}
    u = 2.0 ** -p
    for algo in (orc.SIMPLE, orc.STRASSEN, orc.WINOGRAD):
        R = orc.gemm(algo, A, B, cutoff=cutoff)
        wide = orc.convert(R, 4 * p)
        diff, _ = orc.scalar("sub", wide, exact)
        e = np.abs(orc.to_double(diff)) / Fabs
        errs[algo] = e.max() / u
    d = 3  # 96 -> 48 -> 24 -> 12
    assert errs[orc.SIMPLE] <= n
    assert errs[orc.STRASSEN] <= (12 ** d) * (cutoff ** 2 + 5 * cutoff)
    assert errs[orc.WINOGRAD] <= (18 ** d) * (cutoff ** 2 + 6 * cutoff)
    assert errs[orc.STRASSEN] > errs[orc.SIMPLE] and errs[orc.WINOGRAD] > errs[orc.SIMPLE]


def test_search_shapes_against_the_replay():
    """A shrinking search (hypothesis) over shapes 1..13, cutoffs 1..4, both
    odd-size policies, both recursions and exponent ranges, for any
    disagreement between the oracle and the mpmath replay of the printed
    formulas."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=150, deadline=None, derandomize=True)
    @hyp.given(st.integers(1, 13), st.integers(1, 13), st.integers(1, 13), st.integers(1, 4),
               st.sampled_from([orc.PEEL, orc.MIXED]), st.sampled_from([orc.STRASSEN, orc.WINOGRAD]),
               st.integers(0, 20), st.integers(0, 10 ** 6))
    def check(m, l, n, cutoff, policy, algo, spread, seed):
        p = 96
        A = gen.uniform_pm1(m, l, p, seed, -spread, spread)
        B = gen.uniform_pm1(l, n, p, seed + 1, -spread, spread)
        R = orc.gemm(algo, A, B, cutoff=cutoff, policy=policy)
        ref = _rec(_mat(A), _mat(B), p, algo, cutoff, policy, m, l, n)
        for i in range(m):
            for j in range(n):
                assert entry_mpf(R, i, j) == ref[i][j], (m, l, n, cutoff, policy, algo, i, j)

    check()
