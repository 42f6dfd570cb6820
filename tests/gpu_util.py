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


def rel_errors_vs_rows(C: "mp.DeviceMP", R) -> np.ndarray:
    """|c~_ij - r_i| / |r_i| for a device result C (m x n, p bits) against
    reference rows R (m x 1 at q >= p bits, host): C is widened to q bits
    (exactly) and the difference is taken on the device at q bits, so the
    error is read to ~2^(p-q) relative accuracy from the top limb."""
    import torch

    m, n, q = C.rows, C.cols, R.p
    torch.cuda.synchronize()
    C2 = mp.DeviceMP.empty(m, n, q)
    mp.convert(C, C2)
    dR = mp.DeviceMP.from_host(HostMP(np.asarray(R.limb), np.asarray(R.exp), np.asarray(R.sign), q))
    Rf = mp.DeviceMP(dR.limb.expand(-1, -1, n).contiguous(), dR.exp.expand(-1, n).contiguous(),
                     dR.sign.expand(-1, n).contiguous(), q, m, n)
    torch.cuda.synchronize()
    D = mp.DeviceMP.empty(m, n, q)
    mp.elementwise(mp.OP_SUB, C2, Rf, D)
    mp.check_status("error difference")
    torch.cuda.synchronize()
    top = D.limb[0].cpu().numpy().view(np.uint64).astype(np.float64) * 2.0 ** -64
    e = D.exp.cpu().numpy()
    rtop = np.asarray(R.limb)[0, :, 0].astype(np.float64) * 2.0 ** -64
    re = np.asarray(R.exp)[:, 0]
    zero = e == np.iinfo(np.int64).min
    with np.errstate(divide="ignore", over="ignore"):
        lg = np.log2(np.where(zero, 1.0, top)) + np.where(zero, 0, e).astype(np.float64) \
            - (np.log2(rtop) + re.astype(np.float64))[:, None]
    return np.where(zero, 0.0, np.exp2(lg))
