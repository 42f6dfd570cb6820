"""GPU blocked LU with partial pivoting and the solves (arXiv 1410.1599
Sec. 4) against the CPU oracle: factors, pivots and solution bit for bit."""
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, dev

pytestmark = pytest.mark.gpu


def gpu_lu(A, b, panel, algo, cutoff, pivoting=True):
    n = A.shape[0]
    dA = dev(A)
    db = dev(b)
    dx = mp.DeviceMP.empty(n, 1, A.p)
    piv = torch.zeros(n, dtype=torch.int64, device="cuda")
    mp.set_lu(panel, algo, cutoff)
    mp.set_lu_pivoting(pivoting)
    try:
        mp.mplu(dA, piv, db, dx)
        rc = mp.sync_status()
    finally:
        mp.set_lu(128, mp.SIMPLE, 64)
        mp.set_lu_pivoting(True)
    return dA.to_host(), piv.cpu().numpy(), dx.to_host(), rc


def b_of(A):
    """b = A * ones by the Simple product (both sides use the same b)."""
    n = A.shape[0]
    return orc.gemm(orc.SIMPLE, A, gen.ones(n, 1, A.p))


def check(A, panel, algo, cutoff, pivoting=True):
    b = b_of(A)
    bB = gen.HostMP(b.limb, b.exp, b.sign, b.p)
    F, piv, x, rc = gpu_lu(A, bB, panel, algo, cutoff, pivoting)
    assert rc == 0
    Fo, pivo, rco = orc.lu(A, panel=panel, algo=algo, cutoff=cutoff, pivoting=pivoting)
    assert rco == 0
    assert list(piv) == list(pivo)
    assert_bits_equal(F, Fo, "factors")
    xo = orc.lu_solve(Fo, pivo, b)
    assert_bits_equal(x, xo, "solution")
    return x


@pytest.mark.parametrize("panel", [1, 3, 8, 128])
@pytest.mark.parametrize("algo,cutoff", [(mp.SIMPLE, 64), (mp.BLOCK, 64), (mp.STRASSEN, 2), (mp.WINOGRAD, 2)])
def test_small_random_pivoting(panel, algo, cutoff):
    A = gen.uniform_pm1(23, 23, 256, 7, -4, 4)
    check(A, panel, algo, cutoff)


@pytest.mark.parametrize("p", [128, 256, 300, 512, 1024])
@pytest.mark.parametrize("algo,cutoff", [(mp.SIMPLE, 64), (mp.WINOGRAD, 16)])
def test_well_conditioned_ragged_panels(p, algo, cutoff):
    n = 75 if p == 1024 else 150
    A = gen.well_conditioned(n, p, 5)
    x = check(A, 32, algo, cutoff)
    # x is close to ones
    err = max(abs(float(gen.entry_fraction(x, i, 0)) - 1.0) for i in range(n))
    assert err < 1e-20


def test_pivot_ties():
    """Tied pivot magnitudes (opposite signs) at two elimination steps: the
    first row of largest |a_ik| is taken, as in the oracle."""
    rows = [[2, 1, 3, -1, 5, 7], [-2, 3, 1, 4, -2, 1], [2, -3, 2, 1, 3, -4],
            [1, 3, -5, 2, 1, 2], [-1, 2, 4, -3, 2, 6], [1, -1, 2, 5, -6, 3]]
    for p in (128, 1024):
        check(gen.from_ints(rows, p), 2, mp.SIMPLE, 64)


def test_lotkin_ill_conditioned():
    A = gen.lotkin(48, 256)
    check(A, 16, mp.WINOGRAD, 8)


def test_singular_reported():
    p = 128
    A = gen.uniform_pm1(12, 12, p, 9)
    A.exp[:, 5] = gen.EXP_ZERO
    A.limb[:, :, 5] = 0
    b = gen.uniform_pm1(12, 1, p, 10)
    _, _, _, rc = gpu_lu(A, b, 4, mp.SIMPLE, 64)
    assert rc == -3
    assert mp.load_library().mp_singular_column() == 5


@pytest.mark.parametrize("p,n", [(256, 90), (1024, 70), (2048, 40), (8650, 24)])
@pytest.mark.parametrize("panel", [1, 8, 128])
def test_unpivoted_paper_lu(p, n, panel):
    """The paper's LU without pivoting (Sec. 4) on a random matrix, where
    partial pivoting would exchange rows: factors, piv = identity and the
    solution bit for bit (fused column steps up to 1024 bits, separate
    pivot / divide / rank-1 launches at 2048)."""
    A = gen.uniform_pm1(n, n, p, 31)
    check(A, panel, mp.WINOGRAD, 8, pivoting=False)


def test_unpivoted_zero_pivot_reported():
    p = 256
    A = gen.uniform_pm1(10, 10, p, 32)
    A.exp[0, 0] = gen.EXP_ZERO                   # a_11 = 0: regular, but no pivot without exchanges
    A.limb[:, 0, 0] = 0
    b = gen.uniform_pm1(10, 1, p, 33)
    _, _, _, rc = gpu_lu(A, b, 4, mp.SIMPLE, 64, pivoting=False)
    assert rc == -3
    assert mp.load_library().mp_singular_column() == 0
    _, _, _, rc = gpu_lu(A, b, 4, mp.SIMPLE, 64, pivoting=True)
    assert rc == 0


@pytest.mark.parametrize("p", [8192, 8650])
@pytest.mark.parametrize("pivoting", [False, True])
def test_lotkin_wide_precision(p, pivoting):
    """The paper's ill-conditioned case at its own precisions (Sec. 4: 8192
    and 8650 bits): Lotkin matrix, blocked LU with Winograd trailing
    products, factors and solution bit for bit against the oracle."""
    A = gen.lotkin(32, p)
    check(A, 8, mp.WINOGRAD, 4, pivoting=pivoting)


def _first_max_abs_row(A, col):
    """Index of the first entry of largest magnitude in column col (exact)."""
    mags = [abs(gen.entry_fraction(A, i, col)) for i in range(A.shape[0])]
    best = max(mags)
    return mags.index(best)


def _log2abs(M):
    """log2 |x| of every entry (-inf for zeros), from the top limb and the exponent."""
    f = np.asarray(M.limb[0], dtype=np.float64) * 2.0 ** -64
    with np.errstate(divide="ignore"):
        out = np.log2(f) + np.asarray(M.exp, dtype=np.float64)
    return np.where(np.asarray(M.exp) == gen.EXP_ZERO, -np.inf, out)


@pytest.mark.parametrize("n,p,kind", [(1024, 256, "well"), (1024, 1024, "lotkin"),
                                      (2048, 256, "lotkin"), (2048, 1024, "well")])
def test_full_size_properties(n, p, kind):
    """The LU workload at its full sizes (n = 1024 and 2048 at 256 and 1024
    bits, U[-1,1) + nI and Lotkin, panel 128, Winograd trailing products,
    cutoff 64: the launch configuration bench.py times), checked where the
    oracle reaches one entry at a time and by properties that hold at any
    size (Sec. 4 and partial pivoting):
      - the first pivot is the first row of largest |a_i1|; row 1 of U is that
        row of A, bit for bit; every multiplier of column 1 is the oracle's
        RN(a_i1 / u_11) of the finally permuted row, bit for bit;
      - piv is a sequence of exchanges (piv[k] >= k), the identity for the
        diagonally dominant matrix; every multiplier has |l_ik| <= 1;
      - sampled rows of the residual b - A x~, formed exactly by the
        oracle, stay below n 2^-p (||A|| ||x~|| + ||b||)."""
    A = gen.well_conditioned(n, p, 5) if kind == "well" else gen.lotkin(n, p)
    b = gen.uniform_pm1(n, 1, p, 61)
    F, piv, x, rc = gpu_lu(A, b, 128, mp.WINOGRAD, 64)
    assert rc == 0
    assert np.all(piv >= np.arange(n)) and np.all(piv < n)
    if kind == "well":
        assert np.array_equal(piv, np.arange(n))
    sigma = np.arange(n)
    for k in range(n):
        sigma[[k, piv[k]]] = sigma[[piv[k], k]]
    # column 1: pivot, first row of U, multipliers
    assert sigma[0] == _first_max_abs_row(A, 0)
    assert_bits_equal(F.sub([0], np.arange(n)), A.sub([sigma[0]], np.arange(n)), "first row of U")
    q, _ = orc.scalar("div", A.sub(sigma[1:], [0]), A.sub(np.full(n - 1, sigma[0]), [0]))
    assert_bits_equal(F.sub(np.arange(1, n), [0]), q, "multipliers of column 1")
    # |l_ik| <= 1 below the diagonal: exponent <= 0, or exactly 1 (exponent 1, mantissa 1/2)
    low = np.tril(np.ones((n, n), bool), -1)
    e = np.asarray(F.exp)
    zero = e == gen.EXP_ZERO
    half = (np.asarray(F.limb[0]) == np.uint64(1 << 63)) & ~np.asarray(F.limb[1:]).any(axis=0)
    assert np.all((zero | (e <= 0) | ((e == 1) & half))[low]), "a multiplier exceeds 1 in magnitude"
    # residual of sampled rows, exact: [a_i, b_i] . [x~; -1] rounded once
    rng = np.random.default_rng(n + p)
    rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 14)]))
    Ar, br = A.sub(rows, np.arange(n)), b.sub(rows, [0])
    Aaug = gen.HostMP(np.concatenate([Ar.limb, br.limb], axis=2), np.concatenate([Ar.exp, br.exp], axis=1),
                      np.concatenate([Ar.sign, br.sign], axis=1), p)
    m1 = gen.from_ints([[-1]], p)
    Xaug = gen.HostMP(np.concatenate([x.limb, m1.limb], axis=1), np.concatenate([x.exp, m1.exp], axis=0),
                      np.concatenate([x.sign, m1.sign], axis=0), p)
    r = orc.dot_exact(Aaug, Xaug)
    l_r = float(_log2abs(r).max())
    l_a = float(np.log2(np.exp2(_log2abs(A)).sum(axis=1).max()))
    l_x, l_b = float(_log2abs(x).max()), float(_log2abs(b).max())
    l_den = max(l_a + l_x, l_b) + 1.0          # >= log2(||A|| ||x~|| + ||b||)
    assert l_r <= l_den + np.log2(n) - p, "residual 2^%.1f above n 2^-p scale 2^%.1f" % (l_r, l_den + np.log2(n) - p)


@pytest.mark.parametrize("p", [256, 1024])
def test_strided_views(p):
    """A, b and x as sub-blocks of larger matrices (ld > cols, offsets):
    factors, pivots and solution equal the oracle's, and the parents keep
    every entry outside the views."""
    n = 40
    A = gen.uniform_pm1(n, n, p, 95)
    Big = gen.uniform_pm1(n + 7, n + 10, p, 96)
    Big.limb[:, 3:3 + n, 6:6 + n] = A.limb
    Big.exp[3:3 + n, 6:6 + n] = A.exp
    Big.sign[3:3 + n, 6:6 + n] = A.sign
    b = b_of(A)
    Bb = gen.uniform_pm1(n + 4, 3, p, 97)
    Bb.limb[:, 2:2 + n, 1] = b.limb[:, :, 0]
    Bb.exp[2:2 + n, 1] = b.exp[:, 0]
    Bb.sign[2:2 + n, 1] = b.sign[:, 0]
    Xb = gen.uniform_pm1(n + 2, 4, p, 98)
    dBig, dBb, dXb = dev(Big), dev(Bb), dev(Xb)
    piv = torch.zeros(n, dtype=torch.int64, device="cuda")
    mp.set_lu(16, mp.WINOGRAD, 8)
    try:
        mp.mplu(dBig.view(3, 6, n, n), piv, dBb.view(2, 1, n, 1), dXb.view(1, 2, n, 1))
        assert mp.sync_status() == 0
    finally:
        mp.set_lu(128, mp.SIMPLE, 64)
    Fo, pivo, rco = orc.lu(A, panel=16, algo=mp.WINOGRAD, cutoff=8)
    assert rco == 0 and list(piv.cpu().numpy()) == list(pivo)
    got = dBig.to_host()
    assert_bits_equal(got.sub(np.arange(3, 3 + n), np.arange(6, 6 + n)), Fo, "strided factors")
    xo = orc.lu_solve(Fo, pivo, b)
    gx = dXb.to_host()
    assert_bits_equal(gx.sub(np.arange(1, 1 + n), [2]), xo, "strided solution")
    for H, M, (r0, c0, r, c) in ((got, Big, (3, 6, n, n)), (gx, Xb, (1, 2, n, 1)),
                                 (dBb.to_host(), Bb, (0, 0, 0, 0))):
        keep = np.ones(M.shape, bool)
        keep[r0:r0 + r, c0:c0 + c] = False
        assert np.array_equal(H.exp[keep], M.exp[keep]) and np.array_equal(H.limb[:, keep], M.limb[:, keep])


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("p", [128, 1024, 8650])
def test_tiny_systems(n, p):
    """n = 1, 2, 3 (one pivot, one exchange, a one-column trailing product)."""
    A = gen.uniform_pm1(n, n, p, 60 + n)
    check(A, 2, mp.WINOGRAD, 1)


@pytest.mark.parametrize("n", [256, 384])
@pytest.mark.parametrize("p", [128, 256, 512, 1024])
@pytest.mark.parametrize("kind", ["well", "lotkin", "uniform"])
def test_config_lu_bit_exact(n, p, kind):
    """The LU workload's own setup (Sec. 4 steps 1-3 with partial pivoting:
    panel 128, trailing products by Winograd with cutoff 64) over two and
    three panels, so that several trailing products recurse one level and
    the multi-CTA column steps, U12 solves and row exchanges all run, at
    every register class of the fused panel (128 to 1024 bits):
    factors, piv and x bit for bit against the oracle.  U[-1,1) + nI
    (no exchanges), the Lotkin matrix and plain U[-1,1) (exchanges at most
    steps)."""
    if kind == "well":
        A = gen.well_conditioned(n, p, 5)
    elif kind == "lotkin":
        A = gen.lotkin(n, p)
    else:
        A = gen.uniform_pm1(n, n, p, 71)
    check(A, 128, mp.WINOGRAD, 64)


@pytest.mark.parametrize("kind", ["well", "lotkin"])
def test_config_lu_bit_exact_n1024(kind):
    """One full-size LU of the workload (n = 1024 at 256 bits, panel 128,
    Winograd cutoff 64: eight panels, the configuration bench.py times):
    every entry of the factors, the pivots and the solution bit for bit
    against the oracle (about half a minute of oracle time on 16 cores)."""
    A = gen.well_conditioned(1024, 256, 5) if kind == "well" else gen.lotkin(1024, 256)
    check(A, 128, mp.WINOGRAD, 64)


@pytest.mark.parametrize("p,n,nrhs", [(256, 40, 7), (1024, 33, 5), (8650, 14, 3)])
def test_multi_rhs_solve_matches_single(p, n, nrhs):
    """mplu_solve on the factors mplu left: column c of X equals, bit for
    bit, mplu's own solution for b = column c of B, and the oracle's solve
    with its factors (Sec. 4; the wide class at 8650 bits)."""
    A = gen.uniform_pm1(n, n, p, 110 + n)
    B = gen.uniform_pm1(n, nrhs, p, 120 + n)
    F, piv, x0, rc = gpu_lu(A, B.sub(np.arange(n), [0]), 8, mp.WINOGRAD, 4)
    assert rc == 0
    dF, dB = dev(F), dev(B)
    dX = mp.DeviceMP.empty(n, nrhs, p)
    dpiv = torch.as_tensor(piv, device="cuda")
    mp.mplu_solve(dF, dpiv, dB, dX)
    assert mp.sync_status() == 0
    X = dX.to_host()
    assert_bits_equal(X.sub(np.arange(n), [0]), x0, "column 0 vs mplu's own solve")
    Fo, pivo, rco = orc.lu(A, panel=8, algo=mp.WINOGRAD, cutoff=4)
    assert rco == 0 and list(piv) == list(pivo)
    for c in range(nrhs):
        xo = orc.lu_solve(Fo, pivo, B.sub(np.arange(n), [c]))
        assert_bits_equal(X.sub(np.arange(n), [c]), xo, "column %d vs the oracle" % c)


def _exact_inverse(M):
    """Gauss-Jordan in exact rationals."""
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


def test_lotkin_condition_number_small():
    """cond_1 = ||A||_1 ||A^-1||_1 of a small Lotkin matrix (Sec. 4's
    ill-conditioned case) from the GPU inverse (mplu, then mplu_solve with
    B = I) agrees with the exact rational value to 12 digits."""
    from fractions import Fraction as Fr
    from paper_1410_1599_gb300 import norms

    n, p = 12, 256
    A = gen.lotkin(n, p)
    F, piv, _, rc = gpu_lu(A, gen.ones(n, 1, p), 4, mp.WINOGRAD, 2)
    assert rc == 0
    dX = mp.DeviceMP.empty(n, n, p)
    mp.mplu_solve(dev(F), torch.as_tensor(piv, device="cuda"), dev(gen.identity(n, p)), dX)
    assert mp.sync_status() == 0
    X = dX.to_host()
    got = norms.norm1_log2(A) + norms.norm1_log2(X)
    exact_A = [[Fr(1)] * n] + [[Fr(1, i + j + 1) for j in range(n)] for i in range(1, n)]
    Ai = _exact_inverse(exact_A)
    n1 = lambda M: max(sum(abs(M[i][j]) for i in range(n)) for j in range(n))
    import math
    want = math.log2(n1(exact_A)) + math.log2(n1(Ai))
    assert abs(got - want) < 1e-12 * want


@pytest.mark.parametrize("n,p", [(64, 512), (256, 1536)])
def test_lotkin_condition_number_exact(n, p):
    """||A||_1 ||A^-1||_1 of the Lotkin matrix from the GPU inverse (mplu,
    then mplu_solve with B = I) equals the oracle's exact value (the integer
    Hilbert inverse and the Sherman-Morrison update) to 10 digits of its
    logarithm: cond_1 = 10^96.04 at n = 64, 10^389.82 at n = 256."""
    from paper_1410_1599_gb300 import norms

    A = gen.lotkin(n, p)
    F, piv, _, rc = gpu_lu(A, gen.ones(n, 1, p), 32, mp.WINOGRAD, 16)
    assert rc == 0
    dX = mp.DeviceMP.empty(n, n, p)
    mp.mplu_solve(dev(F), torch.as_tensor(piv, device="cuda"), dev(gen.identity(n, p)), dX)
    assert mp.sync_status() == 0
    la, li = orc.lotkin_norm1_log2(n)
    got_a, got_i = norms.norm1_log2(A), norms.norm1_log2(dX.to_host())
    assert abs(got_a - la) < 1e-10 and abs(got_i - li) < 1e-10 * li
