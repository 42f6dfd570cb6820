"""Test helpers: exact conversions between the interchange format and
mpmath / Fraction values, used to pin the oracle against an independent
arbitrary-precision library (mpmath) and against IEEE double arithmetic."""
from fractions import Fraction

import mpmath
import numpy as np

from paper_1410_1599_gb300.inputs import EXP_ZERO, HostMP, entry_fraction, entry_int

MPF_CTX = mpmath.mp
_lm = mpmath.libmp


def exact(t):
    """mpf from a raw libmpf tuple, without rounding to the context precision."""
    return mpmath.mp.make_mpf(t)


def man_exp(man, e):
    """Exact mpf value man * 2^e (no rounding)."""
    return exact(_lm.from_man_exp(man, e))


def entry_mpf(M, r, c):
    """Exact mpf of entry (r, c) (no rounding: the precision is large enough)."""
    e = int(M.exp[r, c])
    if e == EXP_ZERO:
        return exact(_lm.fzero)
    L = M.limb.shape[0]
    man = entry_int(M, r, c)
    return exact(_lm.from_man_exp(-man if M.sign[r, c] else man, e - 64 * L))


def put_mpf(M, r, c, x, neg_zero=False):
    """Store an mpf that fits in M.p bits (checked)."""
    L = M.limb.shape[0]
    if x._mpf_ == _lm.fzero:
        M.limb[:, r, c] = 0
        M.exp[r, c] = EXP_ZERO
        M.sign[r, c] = 1 if neg_zero else 0
        return
    sgn, man, exp, bc = x._mpf_
    assert bc <= M.p, (bc, M.p)
    mant = int(man) << (64 * L - bc)
    for k in range(L):
        M.limb[k, r, c] = (mant >> (64 * (L - 1 - k))) & 0xFFFFFFFFFFFFFFFF
    M.exp[r, c] = exp + bc
    M.sign[r, c] = sgn


def from_mpf_list(vals, p, shape):
    M = HostMP.zeros(shape[0], shape[1], p)
    for i, x in enumerate(vals):
        put_mpf(M, i // shape[1], i % shape[1], x)
    return M


def rn(x, p):
    """mpmath: x rounded to p bits, nearest-even (library routine)."""
    return exact(_lm.mpf_pos(x._mpf_, p, _lm.round_nearest))


def mp_add(x, y, p):
    return exact(_lm.mpf_add(x._mpf_, y._mpf_, p, _lm.round_nearest))


def mp_sub(x, y, p):
    return exact(_lm.mpf_sub(x._mpf_, y._mpf_, p, _lm.round_nearest))


def mp_mul(x, y, p):
    return exact(_lm.mpf_mul(x._mpf_, y._mpf_, p, _lm.round_nearest))


def mp_div(x, y, p):
    return exact(_lm.mpf_div(x._mpf_, y._mpf_, p, _lm.round_nearest))


def same_value(M, r, c, x):
    """Bits of entry (r, c) equal the p-bit number x (zero sign ignored)."""
    return entry_mpf(M, r, c) == x


def to_fraction(M, r, c):
    return entry_fraction(M, r, c)
