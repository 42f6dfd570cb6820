"""Helpers for the GPU parity tests: move interchange matrices to the device,
run a library call, bring results back, compare bits with the oracle."""
import numpy as np

from paper_1410_1599_gb300 import binding as mp
from paper_1410_1599_gb300.inputs import HostMP


def dev(M: HostMP):
    return mp.DeviceMP.from_host(M)


def assert_bits_equal(got, want, what=""):
    """Every entry's limbs, exponent and sign identical."""
    assert got.exp.shape == want.exp.shape, (what, got.exp.shape, want.exp.shape)
    bad = ((np.asarray(got.limb) != np.asarray(want.limb)).any(axis=0)
           | (np.asarray(got.exp) != np.asarray(want.exp))
           | (np.asarray(got.sign) != np.asarray(want.sign)))
    n = int(bad.sum())
    if n:
        idx = np.argwhere(bad)[:5]
        raise AssertionError("%s: %d of %d entries differ, first at %s" % (what, n, bad.size, idx.tolist()))


def gemm(A: HostMP, B: HostMP, algo, cutoff=64):
    dA, dB = dev(A), dev(B)
    dC = mp.DeviceMP.empty(A.shape[0], B.shape[1], A.p)
    mp.mpgemm(dA, dB, dC, algo, cutoff)
    mp.check_status("gemm")
    return dC.to_host()
