"""GPU blocked LU with partial pivoting and the solves (arXiv 1410.1599
Sec. 4) against the CPU oracle: factors, pivots and solution bit for bit."""
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
