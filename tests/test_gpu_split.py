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
