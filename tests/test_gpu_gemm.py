"""GPU MP GEMM against the CPU oracle running the same algorithm, summation
order, cutoff and odd-dimension policy: bit-exact (arXiv 1410.1599 Sec. 2).

Oracle-sized cases span several leaf tiles and ragged tails; the full sizes
of the benchmark (n in {1023, 1024, 2048} at 512 bits, cutoff 64) are
checked on the closed sampled row/column sets the oracle can evaluate
(oracle.orc_sampled.c), which cover every recursion path of those rows."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300 import inputs as gen
from tests.gpu_util import assert_bits_equal, dev, gemm

pytestmark = pytest.mark.gpu

ALGOS = {"simple": mp.SIMPLE, "block": mp.BLOCK, "strassen": mp.STRASSEN, "winograd": mp.WINOGRAD}


def test_config1_simple_64_256bit():
    A = gen.uniform_pm1(64, 64, 256, 1)
    B = gen.uniform_pm1(64, 64, 256, 2)
    want = orc.gemm(orc.SIMPLE, A, B)
    for algo in (mp.SIMPLE, mp.BLOCK):
        assert_bits_equal(gemm(A, B, algo), want, "config1 algo %d" % algo)


@pytest.mark.parametrize("p", [128, 200, 256, 512, 1024, 2048, 4000, 8650])
@pytest.mark.parametrize("algo", ["simple", "block"])
def test_simple_block_ragged(algo, p):
    m, l, n = (67, 45, 83) if p < 1024 else ((37, 29, 45) if p <= 2048 else (19, 13, 37))
    A = gen.uniform_pm1(m, l, p, 11, -16, 16)
    B = gen.uniform_pm1(l, n, p, 12, -16, 16)
    want = orc.gemm(orc.SIMPLE, A, B)
    assert_bits_equal(gemm(A, B, ALGOS[algo]), want, "%s p=%d" % (algo, p))


@pytest.mark.parametrize("policy", [mp.PEEL, mp.MIXED])
@pytest.mark.parametrize("algo", ["strassen", "winograd"])
@pytest.mark.parametrize("dims,cutoff,p", [((130, 97, 71), 16, 256), ((128, 128, 128), 16, 512),
                                           ((67, 99, 35), 8, 128), ((33, 33, 33), 4, 1024),
                                           ((150, 151, 149), 32, 512), ((27, 19, 23), 3, 2048),
                                           ((19, 17, 21), 4, 8192), ((14, 15, 13), 3, 8650)])
def test_recursion_matches_oracle(algo, policy, dims, cutoff, p):
    m, l, n = dims
    A = gen.uniform_pm1(m, l, p, 21, -16, 16)
    B = gen.uniform_pm1(l, n, p, 22, -16, 16)
    want = orc.gemm(ALGOS[algo], A, B, cutoff=cutoff, policy=policy)
    mp.set_odd_policy(policy)
    try:
        got = gemm(A, B, ALGOS[algo], cutoff)
    finally:
        mp.set_odd_policy(mp.PEEL)
    assert_bits_equal(got, want, "%s %s" % (algo, dims))


@pytest.mark.parametrize("algo", list(ALGOS))
def test_degenerate_shapes(algo):
    p = 256
    for m, l, n in ((1, 1, 1), (1, 7, 1), (5, 0, 3), (2, 3, 5), (65, 1, 65), (1, 130, 129)):
        A = gen.uniform_pm1(m, l, p, 31)
        B = gen.uniform_pm1(l, n, p, 32)
        want = orc.gemm(ALGOS[algo], A, B, cutoff=1)
        assert_bits_equal(gemm(A, B, ALGOS[algo], 1), want, "%s %s" % (algo, (m, l, n)))


def test_integer_inputs_all_algorithms_equal():
    A = gen.small_ints(96, 96, 512, 41, bits=20)
    B = gen.small_ints(96, 96, 512, 42, bits=20)
    ref = gemm(A, B, mp.SIMPLE)
    for algo in (mp.BLOCK, mp.STRASSEN, mp.WINOGRAD):
        assert_bits_equal(gemm(A, B, algo, 8), ref, "integers algo %d" % algo)


@pytest.mark.parametrize("n", [1023, 1024, 2048])
@pytest.mark.parametrize("algo", ["winograd", "strassen", "simple"])
def test_full_size_sampled(algo, n):
    """The benchmark workload: 512-bit, entries U[-1,1) * 2^e, e in [-16, 16],
    cutoff 64, odd sizes peeled, in the launch configuration bench.py times."""
    p, cutoff = 512, 64
    A = gen.uniform_pm1(n, n, p, 3, -16, 16)
    B = gen.uniform_pm1(n, n, p, 4, -16, 16)
    got = gemm(A, B, ALGOS[algo], cutoff)
    rng = np.random.default_rng(n)
    seeds = [(0, n - 1), (n - 1, 0), tuple(rng.integers(0, n, 2))]
    for i0, j0 in seeds:
        rows = orc.sample_set(0, ALGOS[algo], n, n, n, cutoff, orc.PEEL, int(i0))
        cols = orc.sample_set(1, ALGOS[algo], n, n, n, cutoff, orc.PEEL, int(j0))
        want = orc.gemm_sampled(ALGOS[algo], A, B, rows, cols, cutoff=cutoff)
        assert_bits_equal(got.sub(rows, cols), want, "%s n=%d sample (%d,%d)" % (algo, n, i0, j0))


def test_batched_equals_individual():
    """Config 1's batch of independent 64^3 products (256-bit) in one launch."""
    p, m, l, n, batch = 256, 64, 64, 64, 24
    As = [gen.uniform_pm1(m, l, p, 500 + b) for b in range(batch)]
    Bs = [gen.uniform_pm1(l, n, p, 600 + b) for b in range(batch)]
    stack = lambda Ms: gen.HostMP(np.concatenate([M.limb for M in Ms], axis=1),
                                  np.concatenate([M.exp for M in Ms], axis=0),
                                  np.concatenate([M.sign for M in Ms], axis=0), p)
    dA, dB = dev(stack(As)), dev(stack(Bs))
    dC = mp.DeviceMP.empty(batch * m, n, p)
    for algo in (mp.SIMPLE, mp.BLOCK):
        mp.mpgemm_batched(batch, dA, dB, dC, algo)
        mp.check_status("batched")
        C = dC.to_host()
        for b in (0, 7, batch - 1):
            want = orc.gemm(orc.SIMPLE, As[b], Bs[b])
            got = C.sub(np.arange(b * m, (b + 1) * m), np.arange(n))
            assert_bits_equal(got, want, "batch %d" % b)


@pytest.mark.parametrize("algo", [mp.EXACT, mp.SPLIT])
def test_exact_and_split_reject_wide_precision(algo):
    """MP_EXACT and MP_SPLIT stop at 2048 bits: MP_ERR_UNSUPPORTED above."""
    A = gen.uniform_pm1(4, 4, 4000, 1)
    dC = mp.DeviceMP.empty(4, 4, 4000)
    with pytest.raises(mp.MPError) as e:
        mp.mpgemm(dev(A), dev(A), dC, algo)
    assert e.value.code == -7


@pytest.mark.parametrize("p,auto", [(512, 64), (2048, 32)])
def test_automatic_cutoff(p, auto):
    """cutoff 0: the library picks the cutoff (64 up to 1024 bits, 32 at
    2048); the bits equal the oracle's Winograd at that cutoff."""
    m = 133 if p == 512 else 70
    A = gen.uniform_pm1(m, m, p, 61, -16, 16)
    B = gen.uniform_pm1(m, m, p, 62, -16, 16)
    want = orc.gemm(orc.WINOGRAD, A, B, cutoff=auto)
    assert_bits_equal(gemm(A, B, mp.WINOGRAD, 0), want, "automatic cutoff p=%d" % p)


@pytest.mark.parametrize("algo", ["simple", "block", "strassen", "winograd", "exact", "split"])
@pytest.mark.parametrize("p", [256, 1024])
def test_strided_views(algo, p):
    """A, B and C as sub-blocks of larger matrices (row stride ld > cols,
    nonzero offsets): the product equals the oracle's on the extracted
    blocks bit for bit, and C's parent keeps every entry outside the view."""
    m, l, n = 70, 45, 53
    BigA = gen.uniform_pm1(m + 9, l + 13, p, 91, -8, 8)
    BigB = gen.uniform_pm1(l + 5, n + 7, p, 92, -8, 8)
    BigC = gen.uniform_pm1(m + 6, n + 11, p, 93)
    dC = dev(BigC)
    code = {"exact": mp.EXACT, "split": mp.SPLIT}.get(algo, ALGOS.get(algo))
    mp.mpgemm(dev(BigA).view(4, 7, m, l), dev(BigB).view(3, 2, l, n), dC.view(5, 3, m, n), code, 16)
    mp.check_status("strided %s" % algo)
    got = dC.to_host()
    A = BigA.sub(np.arange(4, 4 + m), np.arange(7, 7 + l))
    B = BigB.sub(np.arange(3, 3 + l), np.arange(2, 2 + n))
    want = orc.dot_exact(A, B) if algo in ("exact", "split") else orc.gemm(code, A, B, cutoff=16)
    assert_bits_equal(got.sub(np.arange(5, 5 + m), np.arange(3, 3 + n)), want, "strided %s" % algo)
    outside = np.ones(BigC.shape, bool)
    outside[5:5 + m, 3:3 + n] = False
    assert np.array_equal(got.exp[outside], BigC.exp[outside])
    assert np.array_equal(got.sign[outside], BigC.sign[outside])
    assert np.array_equal(got.limb[:, outside], BigC.limb[:, outside])


@pytest.mark.parametrize("algo", ["simple", "block", "strassen", "winograd", "exact", "split"])
def test_empty_outputs(algo):
    """m = 0 or n = 0: nothing to compute; the call succeeds and writes nothing."""
    p = 256
    code = {"exact": mp.EXACT, "split": mp.SPLIT}.get(algo, ALGOS.get(algo))
    for m, l, n in ((0, 5, 4), (4, 5, 0), (0, 0, 0)):
        A = dev(gen.uniform_pm1(m, l, p, 1))
        B = dev(gen.uniform_pm1(l, n, p, 2))
        C = mp.DeviceMP.empty(m, n, p)
        mp.mpgemm(A, B, C, code, 8)
        mp.check_status("empty %s %s" % (algo, (m, l, n)))
        assert C.to_host().exp.shape == (m, n)
