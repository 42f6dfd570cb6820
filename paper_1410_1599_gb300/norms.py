"""Norms of multiple-precision matrices, read in log2 space.

The condition numbers of Sec. 4's ill-conditioned matrices reach
10^1576 (2^5237): far outside double range.  These helpers read each entry
as log2|x| from its top limb and exponent (53 significant bits, plenty for
a norm quoted to a few digits) and sum magnitudes in log space.
"""
from __future__ import annotations

import math

import numpy as np

from .inputs import EXP_ZERO


def log2abs(M) -> np.ndarray:
    """log2 |x| of every entry of an interchange-format matrix (host arrays
    limb[L][rows][cols], exp[rows][cols]); -inf for zeros."""
    top = np.asarray(M.limb[0], dtype=np.uint64).astype(np.float64) * 2.0 ** -64
    e = np.asarray(M.exp)
    zero = e == EXP_ZERO
    with np.errstate(divide="ignore"):
        out = np.log2(np.where(zero, 1.0, top)) + np.where(zero, 0, e).astype(np.float64)
    return np.where(zero, -np.inf, out)


def logsumexp2(v: np.ndarray, axis: int) -> np.ndarray:
    """log2 of the sum of 2^v along axis (-inf for an all -inf slice)."""
    mx = np.max(v, axis=axis, keepdims=True)
    mx = np.where(np.isfinite(mx), mx, 0.0)
    with np.errstate(divide="ignore"):
        s = np.log2(np.sum(np.exp2(v - mx), axis=axis, keepdims=True)) + mx
    return np.squeeze(s, axis=axis)


def norm1_log2(M) -> float:
    """log2 of ||M||_1 = max over columns of sum_i |m_ij|."""
    return float(np.max(logsumexp2(log2abs(M), axis=0)))


def norm_inf_log2(M) -> float:
    """log2 of ||M||_inf = max over rows of sum_j |m_ij|."""
    return float(np.max(logsumexp2(log2abs(M), axis=1)))


def log10_of_log2(v: float) -> float:
    return v * math.log10(2.0)
