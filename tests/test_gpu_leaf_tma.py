"""The Block kernel with its A/B limb tiles staged by bulk tensor copies
(TMA; mp_set_leaf_tma) against the thread-staged kernel and the CPU oracle:
the same bits (arXiv 1410.1599 Sec. 2, Eq. 2: every c_ij summed over k in
ascending order, rounded after every operation).

The cases cover every capacity class the copies serve (2 to 1024 bits),
precisions whose limb count is below the class's (planes the copies leave
zero), ragged tiles in m, n and the k-slabs, plain Block products, batched
products and Strassen / Winograd leaves read in place from their parents'
quadrants, recursions whose quadrants start at odd columns (the children are
then all written, with even row strides, and staged by TMA), and layouts the
copies cannot address (a caller's odd row stride) and the 2048-bit class,
where the library keeps the threads' loads.  The profiler's launch counts say
which kernel ran."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, dev

pytestmark = pytest.mark.gpu


def run(A, B, algo, cutoff, tma):
    """C = A B with the given staging; (C, TMA-staged launches, thread-staged launches)."""
    dA, dB = dev(A), dev(B)
    dC = mp.DeviceMP.empty(A.shape[0], B.shape[1], A.p)
    mp.set_leaf_tma(tma)
    try:
        mp.profile_enable(True)
        mp.mpgemm(dA, dB, dC, algo, cutoff)
        mp.check_status("gemm")
        prof = mp.profile_read()
    finally:
        mp.profile_enable(False)
        mp.set_leaf_tma(True)
    return dC.to_host(), prof["leaf_tma"][0], prof["leaf_gemm"][0]


@pytest.mark.parametrize("p", [2, 64, 128, 160, 256, 384, 512, 1000, 1024])
def test_block_even_layout_uses_tma(p):
    # ld 70 / 98 and the plane strides even: the copies apply; 66 rows and
    # 98 columns leave ragged tiles, l = 70 a ragged last k-slab
    m, l, n = 66, 70, 98
    A = gen.uniform_pm1(m, l, p, 71, -16, 16)
    B = gen.uniform_pm1(l, n, p, 72, -16, 16)
    want = orc.gemm(orc.SIMPLE, A, B)
    got, n_tma, n_thr = run(A, B, mp.BLOCK, 64, True)
    assert (n_tma, n_thr) == (1, 0)
    assert_bits_equal(got, want, "TMA-staged Block p=%d" % p)
    ref, n_tma, n_thr = run(A, B, mp.BLOCK, 64, False)
    assert (n_tma, n_thr) == (0, 1)
    assert_bits_equal(ref, want, "thread-staged Block p=%d" % p)


@pytest.mark.parametrize("p", [256, 1024])
def test_block_odd_stride_falls_back(p):
    m, l, n = 67, 45, 83                       # ld 45 and 83: no tensor map
    A = gen.uniform_pm1(m, l, p, 73, -16, 16)
    B = gen.uniform_pm1(l, n, p, 74, -16, 16)
    got, n_tma, n_thr = run(A, B, mp.BLOCK, 64, True)
    assert (n_tma, n_thr) == (0, 1)
    assert_bits_equal(got, orc.gemm(orc.SIMPLE, A, B), "fallback p=%d" % p)


@pytest.mark.parametrize("p", [1500, 2048])
def test_2048_bit_class_keeps_thread_staging(p):
    A = gen.uniform_pm1(34, 36, p, 75, -16, 16)
    B = gen.uniform_pm1(36, 40, p, 76, -16, 16)
    got, n_tma, n_thr = run(A, B, mp.BLOCK, 64, True)
    assert (n_tma, n_thr) == (0, 1)
    assert_bits_equal(got, orc.gemm(orc.SIMPLE, A, B), "%d bits" % p)
    A = gen.uniform_pm1(72, 48, p, 77, -16, 16)
    B = gen.uniform_pm1(48, 56, p, 78, -16, 16)
    got, n_tma, n_thr = run(A, B, mp.WINOGRAD, 16, True)
    assert (n_tma, n_thr) == (0, 1)
    assert_bits_equal(got, orc.gemm(mp.WINOGRAD, A, B, cutoff=16, policy=orc.PEEL), "%d-bit leaves" % p)


def test_wide_class_has_no_block_kernel():
    # above 2048 bits the Block product runs the batched Simple kernel
    A = gen.uniform_pm1(10, 12, 4000, 75, -16, 16)
    B = gen.uniform_pm1(12, 14, 4000, 76, -16, 16)
    got, n_tma, n_thr = run(A, B, mp.BLOCK, 64, True)
    assert (n_tma, n_thr) == (0, 1)
    assert_bits_equal(got, orc.gemm(orc.SIMPLE, A, B), "4000 bits")


@pytest.mark.parametrize("algo", [mp.WINOGRAD, mp.STRASSEN])
@pytest.mark.parametrize("p,dims,cutoff", [(512, (128, 128, 128), 16), (256, (96, 160, 64), 16),
                                           (1024, (64, 64, 64), 16), (384, (136, 112, 112), 16)])
def test_recursion_leaves_in_place(algo, p, dims, cutoff):
    m, l, n = dims
    A = gen.uniform_pm1(m, l, p, 77, -16, 16)
    B = gen.uniform_pm1(l, n, p, 78, -16, 16)
    want = orc.gemm(algo, A, B, cutoff=cutoff, policy=orc.PEEL)
    got, n_tma, n_thr = run(A, B, algo, cutoff, True)
    assert n_tma == 1 and n_thr == 0
    assert_bits_equal(got, want, "TMA leaves %s" % (dims,))
    ref, n_tma, n_thr = run(A, B, algo, cutoff, False)
    assert n_tma == 0 and n_thr == 1
    assert_bits_equal(ref, want, "thread-staged leaves %s" % (dims,))


@pytest.mark.parametrize("algo", [mp.WINOGRAD, mp.STRASSEN])
@pytest.mark.parametrize("n,cutoff", [(124, 32), (125, 32), (250, 64)])
def test_odd_leaves_use_materialised_children(algo, n, cutoff):
    # 124 -> 62 -> leaves of 31 (125 peeled, 250 -> 125 -> 62 with an odd
    # parent): the quadrants' odd column offsets rule out in-place leaves,
    # so every child is written, with an even row stride, and staged by TMA
    p = 512
    A = gen.uniform_pm1(n, n, p, 79, -16, 16)
    B = gen.uniform_pm1(n, n, p, 80, -16, 16)
    want = orc.gemm(algo, A, B, cutoff=cutoff, policy=orc.PEEL)
    got, n_tma, n_thr = run(A, B, algo, cutoff, True)
    assert n_tma == 1 and n_thr == 0
    assert_bits_equal(got, want, "odd leaves n=%d" % n)
    ref, n_tma, n_thr = run(A, B, algo, cutoff, False)
    assert n_tma == 0 and n_thr == 1
    assert_bits_equal(ref, want, "odd leaves, thread-staged, n=%d" % n)


def test_user_layout_with_odd_stride_falls_back():
    A = gen.uniform_pm1(21, 35, 1024, 83, -16, 16)          # ld 35: no tensor map
    B = gen.uniform_pm1(35, 19, 1024, 84, -16, 16)
    got, n_tma, n_thr = run(A, B, mp.BLOCK, 64, True)
    assert n_tma == 0 and n_thr == 1
    assert_bits_equal(got, orc.gemm(orc.SIMPLE, A, B), "1024 bits, odd stride")


@pytest.mark.parametrize("algo", [mp.WINOGRAD, mp.STRASSEN])
def test_mixed_policy_padding_uses_tma(algo):
    # 139 = 3 mod 4 is padded to 140 -> 70 -> leaves of 35 (mixed policy):
    # their odd quadrant offsets rule out in-place leaves, so every child is
    # written (even row stride) and staged by TMA
    p, n = 256, 139
    A = gen.uniform_pm1(n, n, p, 85, -16, 16)
    B = gen.uniform_pm1(n, n, p, 86, -16, 16)
    want = orc.gemm(algo, A, B, cutoff=40, policy=orc.MIXED)
    mp.set_odd_policy(mp.MIXED)
    try:
        got, n_tma, n_thr = run(A, B, algo, 40, True)
    finally:
        mp.set_odd_policy(mp.PEEL)
    assert n_tma == 1 and n_thr == 0
    assert_bits_equal(got, want, "mixed policy")


def test_batched_products_use_tma():
    p, m, l, n, batch = 512, 40, 52, 36, 6
    As = [gen.uniform_pm1(m, l, p, 800 + b) for b in range(batch)]
    Bs = [gen.uniform_pm1(l, n, p, 900 + b) for b in range(batch)]
    stack = lambda Ms: gen.HostMP(np.concatenate([M.limb for M in Ms], axis=1),
                                  np.concatenate([M.exp for M in Ms], axis=0),
                                  np.concatenate([M.sign for M in Ms], axis=0), p)
    dA, dB = dev(stack(As)), dev(stack(Bs))
    dC = mp.DeviceMP.empty(batch * m, n, p)
    mp.profile_enable(True)
    try:
        mp.mpgemm_batched(batch, dA, dB, dC, mp.BLOCK)
        mp.check_status("batched")
        prof = mp.profile_read()
    finally:
        mp.profile_enable(False)
    assert prof["leaf_tma"][0] == 1 and prof["leaf_gemm"][0] == 0
    C = dC.to_host()
    for b in range(batch):
        got = C.sub(np.arange(b * m, (b + 1) * m), np.arange(n))
        assert_bits_equal(got, orc.gemm(orc.SIMPLE, As[b], Bs[b]), "batch %d" % b)


def test_full_size_winograd_staging_agrees():
    """The benchmark's launch configuration (Winograd, n = 2048, 512 bits,
    cutoff 64): both stagings give the same bits on every output."""
    p, n = 512, 2048
    A = gen.uniform_pm1(n, n, p, 81, -16, 16)
    B = gen.uniform_pm1(n, n, p, 82, -16, 16)
    got, n_tma, _ = run(A, B, mp.WINOGRAD, 64, True)
    ref, _, n_thr = run(A, B, mp.WINOGRAD, 64, False)
    assert n_tma == 1 and n_thr == 1
    assert_bits_equal(got, ref, "n = 2048 staging")


def test_setting_rejects_other_values():
    lib = mp.load_library()
    assert lib.mp_set_leaf_tma(2) == -1
    assert lib.mp_set_leaf_tma(-1) == -1
    assert lib.mp_set_leaf_tma(1) == 0
