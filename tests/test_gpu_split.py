"""The split form (MP_SPLIT): rows of A / columns of B aligned and cut into
signed 8-bit digits, digit products on tensor cores, exact recombination and
one rounding -- bit for bit the oracle's correctly rounded exact dot product,
including rows/columns beyond the 64-bit spread budget (limb fallback)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, gemm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [53, 128, 200, 256, 512, 1024, 2048])
def test_split_matches_exact_oracle(p):
    m, l, n = (37, 70, 45) if p >= 1024 else (70, 131, 66)
    A = gen.uniform_pm1(m, l, p, 71, -16, 16)
    B = gen.uniform_pm1(l, n, p, 72, -16, 16)
    want = orc.dot_exact(A, B)
    assert_bits_equal(gemm(A, B, mp.SPLIT), want, "split p=%d" % p)


def test_split_wide_rows_and_columns_fall_back():
    p, m, l, n = 256, 40, 64, 33
    A = gen.uniform_pm1(m, l, p, 73, -8, 8)
    B = gen.uniform_pm1(l, n, p, 74, -8, 8)
    A.exp[3, 5] -= 200          # row 3 spreads over 200 bits
    B.exp[7, 11] += 150         # column 11 too
    A.exp[10, :] = gen.EXP_ZERO # an all-zero row
    A.limb[:, 10, :] = 0
    want = orc.dot_exact(A, B)
    assert_bits_equal(gemm(A, B, mp.SPLIT), want, "split with wide rows/cols")


def test_split_cancellation_to_zero_and_long_k():
    p = 128
    A = gen.from_ints([[3, -3, 5, -5], [1, 1, 1, 1]], p)
    B = gen.from_ints([[7], [7], [1], [1]], p)
    got = gemm(A, B, mp.SPLIT)
    assert_bits_equal(got, orc.dot_exact(A, B), "cancellation")
    assert got.exp[0, 0] == gen.EXP_ZERO
    # k beyond one fp32 chunk
    A = gen.uniform_pm1(9, 1500, 512, 75, -4, 4)
    B = gen.uniform_pm1(1500, 7, 512, 76, -4, 4)
    assert_bits_equal(gemm(A, B, mp.SPLIT), orc.dot_exact(A, B), "long k")


def test_split_equals_exact_kernel_larger():
    p, n = 1024, 256
    A = gen.uniform_pm1(n, n, p, 77, -16, 16)
    B = gen.uniform_pm1(n, n, p, 78, -16, 16)
    s = gemm(A, B, mp.SPLIT)
    e = gemm(A, B, mp.EXACT)
    assert_bits_equal(s, e, "split vs exact kernel")
    rows, cols = np.arange(0, n, 37), np.arange(5, n, 41)
    assert_bits_equal(s.sub(rows, cols), orc.dot_exact(A, B, rows=rows, cols=cols), "oracle sample")


def test_split_many_chunks_per_diagonal():
    """l = 2048 at 1024 bits: the middle weight diagonal gathers 137 pairs x
    2048 k-terms = 548 exact fp32 chunks of 512, more than one int32 register
    sum can take (255 chunks), so the int64 partial sums are built in steps."""
    p, m, l, n = 1024, 20, 2048, 24
    A = gen.uniform_pm1(m, l, p, 79, -6, 6)
    B = gen.uniform_pm1(l, n, p, 80, -6, 6)
    s = gemm(A, B, mp.SPLIT)
    assert_bits_equal(s, gemm(A, B, mp.EXACT), "split vs exact kernel, long k")
    rows, cols = np.array([0, 7, 19]), np.array([0, 11, 23])
    assert_bits_equal(s.sub(rows, cols), orc.dot_exact(A, B, rows=rows, cols=cols), "oracle sample, long k")


def _split(A, B, truncate):
    mp.set_split_truncation(truncate)
    try:
        out = gemm(A, B, mp.SPLIT)
        fb = mp.split_fallbacks()
    finally:
        mp.set_split_truncation(True)
    return out, fb


@pytest.mark.parametrize("p", [53, 128, 512, 1024, 2048])
def test_truncated_equals_full_split(p):
    """Skipping the low diagonals changes no bit: truncated and full split
    forms agree everywhere, and on these inputs (exponents in [-16, 16]) no
    output needs the exact fallback."""
    m, l, n = (70, 200, 90) if p >= 1024 else (150, 300, 140)
    A = gen.uniform_pm1(m, l, p, 81, -16, 16)
    B = gen.uniform_pm1(l, n, p, 82, -16, 16)
    full, fb0 = _split(A, B, False)
    trunc, fb1 = _split(A, B, True)
    assert fb0 == 0 and fb1 == 0
    assert_bits_equal(trunc, full, "truncated vs full split p=%d" % p)
    rows, cols = np.arange(0, m, 7), np.arange(3, n, 11)
    assert_bits_equal(trunc.sub(rows, cols), orc.dot_exact(A, B, rows=rows, cols=cols), "oracle sample")


def _cancelling(m, h, n, p, seed, rows_cancel):
    """A = [X, X'] with X' = X on the rows in rows_cancel, B = [Y; -(1 - 2^-100) Y]
    with small integers Y: on those rows the exact sum is 2^-100 sum_k x_ik y_kj,
    about 100 bits under the products' own size (and every exponent spread
    stays within the 64-bit budget); other rows take an independent X'."""
    X = gen.uniform_pm1(m, h, p, seed)
    X2 = gen.uniform_pm1(m, h, p, seed + 1)
    Y = gen.small_ints(h, n, p, seed + 2, 20)
    A = gen.HostMP.zeros(m, 2 * h, p)
    A.limb[:, :, :h], A.exp[:, :h], A.sign[:, :h] = X.limb, X.exp, X.sign
    A.limb[:, :, h:], A.exp[:, h:], A.sign[:, h:] = X2.limb, X2.exp, X2.sign
    for i in rows_cancel:
        A.limb[:, i, h:], A.exp[i, h:], A.sign[i, h:] = X.limb[:, i], X.exp[i], X.sign[i]
    vals = []
    for k in range(h):
        for j in range(n):
            y = int(gen.entry_fraction(Y, k, j))
            vals.append((0 if y <= 0 else 1, abs(y) * ((1 << 100) - 1), 100))
    Yn = gen.from_exact_ints(vals, p, (h, n))
    B = gen.HostMP.zeros(2 * h, n, p)
    B.limb[:, :h], B.exp[:h], B.sign[:h] = Y.limb, Y.exp, Y.sign
    B.limb[:, h:], B.exp[h:], B.sign[h:] = Yn.limb, Yn.exp, Yn.sign
    return A, B


@pytest.mark.parametrize("p", [128, 1024])
def test_truncation_falls_back_on_cancellation(p):
    """Outputs whose exact value cancels to ~2^-100 of the products are left
    undecided by the truncated sum and recomputed by the exact kernel: the
    fallback count is exactly those outputs, and every bit still equals the
    oracle's exact dot product (and the full split form's)."""
    m, h, n = 24, 40, 19
    cancel = list(range(0, m, 2))
    A, B = _cancelling(m, h, n, p, 90, cancel)
    got, fb = _split(A, B, True)
    assert fb == len(cancel) * n
    want = orc.dot_exact(A, B)
    assert_bits_equal(got, want, "truncated split with cancellation")
    full, fb0 = _split(A, B, False)
    assert fb0 == 0
    assert_bits_equal(full, want, "full split with cancellation")


def test_split_full_size_sampled():
    """The split-form workload at its full size: 4096^3 at 1024 bits, entries
    U[-1,1) * 2^e with e uniform in [-16, 16] (the inputs of bench.py --split),
    truncated form (the default), the launch configuration that run times.
    Sampled outputs, corners included, equal the oracle's correctly rounded
    exact dot product computed one output at a time."""
    import torch

    p, n = 1024, 4096
    A = gen.uniform_pm1(n, n, p, 13, -16, 16)
    B = gen.uniform_pm1(n, n, p, 14, -16, 16)
    dA, dB = mp.DeviceMP.from_host(A), mp.DeviceMP.from_host(B)
    dC = mp.DeviceMP.empty(n, n, p)
    mp.set_split_truncation(True)
    mp.mpgemm(dA, dB, dC, mp.SPLIT, 64)
    mp.check_status("split 4096")
    torch.cuda.synchronize()
    rng = np.random.default_rng(4096)
    rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 10)]))
    cols = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 10)]))
    r, c = torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")
    got = gen.HostMP(dC.limb[:, r][:, :, c].cpu().numpy().view(np.uint64),
                     dC.exp[r][:, c].cpu().numpy(), dC.sign[r][:, c].cpu().numpy(), p)
    del dA, dB, dC
    torch.cuda.empty_cache()
    want = orc.dot_exact(A, B, rows=rows, cols=cols)
    assert_bits_equal(got, want, "split 4096^3 sample")


# ---------------------------------------------------------------------------
# Worst-case digit magnitudes.  The exactness argument of the split form is
# tight here: a digit product reaches 2^14 only when both digits are -128 or
# both +128, an fp32 chunk of 512 such products reaches 2^23, and an int32
# register of 255 chunks reaches 255 * 2^23 < 2^31.  Entries are built from
# byte patterns whose balanced digits (byte + carry, minus 256 from 128 up)
# are all -128: the lowest mantissa byte 0x80 (digit -128, carry 1), every
# byte above it 0x7F (0x7F + 1 = 128: digit -128, carry 1), and the top byte
# 0x80 so that the mantissa stays normalised.  "Small" entries keep the top
# byte 0x80 and take their other bytes from {0x00, 0x01, 0xFF}, so their
# digits are in {-1, 0, 1, 2}; one in every 16 consecutive k is small, so
# each K = 16 tensor-core step adds a product of magnitude 1 to 4 to fifteen
# products of 2^14 and an accumulator already near 2^23.
# ---------------------------------------------------------------------------
def _pattern_entries(rows, cols, p, seed, small_every, flip_from=None, axis=1):
    """rows x cols entries of exponent 0 (so every row / column aligns to the
    same e_max), mantissas built from the byte patterns above.  The entry at
    position k along `axis` is small when k % small_every == small_every - 1
    (never when small_every is 0); from k = flip_from on the entries are
    negative (the chunk sums rise towards 2^22 and come back down)."""
    assert p % 8 == 0
    nb = p // 8
    big = 0x80 | sum(0x7F << (8 * t) for t in range(1, nb - 1)) | (0x80 << (8 * (nb - 1)))
    rng = np.random.default_rng(seed)
    vals = []
    for r in range(rows):
        for c in range(cols):
            k = c if axis == 1 else r
            if small_every and k % small_every == small_every - 1:
                low = rng.choice([0x00, 0x01, 0xFF], size=nb - 1)
                M = sum(int(b) << (8 * t) for t, b in enumerate(low)) | (0x80 << (8 * (nb - 1)))
            else:
                M = big
            sg = 1 if (flip_from is not None and k >= flip_from) else 0
            vals.append((sg, M, p))
    return gen.from_exact_ints(vals, p, (rows, cols))


def _digits_of(M_int, p):
    """Balanced base-256 digits of the aligned integer M 2^64 (exponent e_max,
    F = p + 64), by the rule the split form documents: low digit first."""
    S = (p + 64 + 7) // 8 + 1
    x, out, carry = M_int << 64, [], 0
    for u in range(S):
        t = ((x >> (8 * u)) & 0xFF) + carry
        d, carry = (t - 256, 1) if t >= 128 else (t, 0)
        out.append(d)
    return out


def test_worst_case_patterns_have_extreme_digits():
    """The construction does what the tests below rely on: a big entry's
    digits are -128 everywhere inside its mantissa (one -127 and the carry
    digit 1 at the top), a small entry's lie in [-1, 2] below its top byte,
    and the maximal products exceed 2^22 per chunk."""
    p = 512
    A = _pattern_entries(1, 32, p, 5, 16)
    big = _digits_of(gen.entry_int(A, 0, 0) >> (64 * A.L - p), p)
    assert big[:8] == [0] * 8 and big[8:8 + p // 8 - 1] == [-128] * (p // 8 - 1)
    assert big[8 + p // 8 - 1:] == [-127, 1]
    small = _digits_of(gen.entry_int(A, 0, 15) >> (64 * A.L - p), p)
    assert all(-1 <= d <= 2 for d in small[:8 + p // 8 - 1])
    assert 480 * 128 * 128 + 32 > 1 << 22 and 512 * 128 * 128 <= 1 << 23


@pytest.mark.parametrize("truncate", [False, True])
@pytest.mark.parametrize("p,l,small_every,flip", [
    (1024, 512, 16, None),     # chunk sums near 2^23 with their low bits set
    (512, 1000, 16, None),     # ragged l: chunks cross pair boundaries
    (1024, 2048, 0, None),     # every chunk exactly 2^23, 255 chunks per int32 sum
    (1024, 1024, 16, 512),     # the sum rises to ~2^22, then cancels back down
])
def test_split_exact_at_worst_case_digits(p, l, small_every, flip, truncate):
    """Digit products of 2^14 everywhere (the largest a balanced digit pair
    gives), mixed inside each K = 16 tensor-core step with products of
    magnitude 1 to 4: every output of the split form, full and truncated,
    equals the oracle's correctly rounded exact dot product and the exact
    limb kernel's result.  A tensor core that kept fewer than 24 significant
    bits anywhere in its fp32 accumulation would drop the small products."""
    m, n = 12, 20
    A = _pattern_entries(m, l, p, 100 + l, small_every, flip, axis=1)
    B = _pattern_entries(l, n, p, 200 + l, small_every, None, axis=0)
    got, _ = _split(A, B, truncate)
    assert_bits_equal(got, gemm(A, B, mp.EXACT), "split vs exact kernel at worst-case digits")
    assert_bits_equal(got, orc.dot_exact(A, B), "split vs oracle at worst-case digits")


def test_split_refuses_workspace_off_this_device():
    """The split form's digit planes are read by TMA loads multicast inside a
    cluster, so its tensor maps may only cover this GPU's own memory: a
    caller workspace in page-locked host memory is refused with MP_ERR_ARG
    on the host, before anything is launched, and C is left untouched; the
    same product with a device workspace succeeds."""
    import torch

    p, m, l, n = 256, 16, 40, 24
    A = gen.uniform_pm1(m, l, p, 83, -4, 4)
    B = gen.uniform_pm1(l, n, p, 84, -4, 4)
    dA, dB = mp.DeviceMP.from_host(A), mp.DeviceMP.from_host(B)
    dC = mp.DeviceMP.empty(m, n, p)
    before = dC.to_host()
    need = mp.workspace_size(m, l, n, p, mp.SPLIT, 64)
    host = torch.empty(need + 4096, dtype=torch.uint8, pin_memory=True)
    mp.set_workspace(host)
    try:
        with pytest.raises(mp.MPError) as err:
            mp.mpgemm(dA, dB, dC, mp.SPLIT, 64)
        assert err.value.code == -1                     # MP_ERR_ARG
    finally:
        mp.set_workspace(None)
    torch.cuda.synchronize()
    assert_bits_equal(dC.to_host(), before, "C after a refused split call")
    devws = torch.empty(need + 4096, dtype=torch.uint8, device="cuda")
    mp.set_workspace(devws)
    try:
        mp.mpgemm(dA, dB, dC, mp.SPLIT, 64)
        mp.check_status("split with a device workspace")
    finally:
        mp.set_workspace(None)
    assert_bits_equal(dC.to_host(), orc.dot_exact(A, B), "split with a caller workspace")
