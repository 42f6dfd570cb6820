"""ctypes wrapper of the CPU oracle (test infrastructure only).

Only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg use
this module.  Matrices are passed in the interchange format (limb planes,
exponent, sign) as any object with .limb/.exp/.sign/.p attributes and
returned as OMat objects with the same attributes.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from fractions import Fraction

import numpy as np

from . import build as _build

SIMPLE, BLOCK, STRASSEN, WINOGRAD = 0, 1, 2, 3
PEEL, MIXED = 0, 1
EXP_ZERO = np.iinfo(np.int64).min

_lib = None


class OMat:
    """Interchange-format matrix returned by the oracle."""

    def __init__(self, limb, exp, sign, p):
        self.limb, self.exp, self.sign, self.p = limb, exp, sign, p

    @property
    def shape(self):
        return self.exp.shape

    @staticmethod
    def empty(rows, cols, p):
        L = (p + 63) // 64
        return OMat(np.zeros((L, rows, cols), np.uint64),
                    np.full((rows, cols), EXP_ZERO, np.int64),
                    np.zeros((rows, cols), np.int8), p)


def lib():
    """The oracle library: ORACLE_LIB names another build of the same sources
    (the mutation tests load deliberately broken copies this way)."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(os.environ.get("ORACLE_LIB") or _build.build())
        _lib.orc_api_sample_set.restype = C.c_int64
        _lib.orc_api_max_threads.restype = C.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _mat_args(M):
    limb = np.ascontiguousarray(M.limb, dtype=np.uint64)
    exp = np.ascontiguousarray(M.exp, dtype=np.int64)
    sign = np.ascontiguousarray(M.sign, dtype=np.int8)
    rows, cols = exp.shape
    keep = (limb, exp, sign)
    return keep, [_p(limb), _p(exp), _p(sign), C.c_int64(cols), C.c_int64(rows * cols)]


def set_threads(n: int):
    lib().orc_api_set_threads(C.c_int(n))


def max_threads() -> int:
    return lib().orc_api_max_threads()


def range_error() -> int:
    return lib().orc_api_range_error()


def _flat(M):
    """1 x count view of any-shaped interchange arrays."""
    L = M.limb.shape[0]
    return OMat(M.limb.reshape(L, 1, -1), M.exp.reshape(1, -1), M.sign.reshape(1, -1), M.p)


def scalar(op: str, X, Y):
    """Elementwise x op y, op in add/sub/mul/div, arrays of equal shape."""
    code = {"add": 0, "sub": 1, "mul": 2, "div": 3}[op]
    shape = X.exp.shape
    Xf, Yf = _flat(X), _flat(Y)
    count = Xf.exp.shape[1]
    R = OMat.empty(1, count, X.p)
    kx, ax = _mat_args(Xf)
    ky, ay = _mat_args(Yf)
    kr, ar = _mat_args(R)
    rc = lib().orc_api_scalar(C.c_int(code), C.c_int(X.p), C.c_int64(count), *ax, *ay, *ar)
    if rc == -2:
        raise ValueError("invalid operand encoding")
    out = OMat(kr[0].reshape((R.limb.shape[0],) + shape), kr[1].reshape(shape),
               kr[2].reshape(shape), X.p)
    return out, rc


def convert(X, p_to: int):
    shape = X.exp.shape
    Xf = _flat(X)
    count = Xf.exp.shape[1]
    R = OMat.empty(1, count, p_to)
    kx, ax = _mat_args(Xf)
    kr, ar = _mat_args(R)
    rc = lib().orc_api_convert(C.c_int(X.p), C.c_int(p_to), C.c_int64(count), *ax, *ar)
    if rc:
        raise ValueError("invalid operand encoding")
    return OMat(kr[0].reshape((R.limb.shape[0],) + shape), kr[1].reshape(shape),
                kr[2].reshape(shape), p_to)


def to_double(X) -> np.ndarray:
    shape = X.exp.shape
    Xf = _flat(X)
    count = Xf.exp.shape[1]
    out = np.zeros(count, np.float64)
    kx, ax = _mat_args(Xf)
    rc = lib().orc_api_to_double(C.c_int(X.p), C.c_int64(count), *ax, _p(out))
    if rc:
        raise ValueError("invalid operand encoding")
    return out.reshape(shape)


def gemm(algo: int, A, B, cutoff: int = 64, policy: int = PEEL, nb: int = 32):
    m, l = A.exp.shape
    l2, n = B.exp.shape
    assert l == l2 and A.p == B.p
    Cm = OMat.empty(m, n, A.p)
    ka, aa = _mat_args(A)
    kb, ab = _mat_args(B)
    kc, ac = _mat_args(Cm)
    rc = lib().orc_api_gemm(C.c_int(algo), C.c_int(cutoff), C.c_int(policy), C.c_int(nb),
                            C.c_int64(m), C.c_int64(l), C.c_int64(n), C.c_int(A.p),
                            *aa, *ab, *ac)
    if rc:
        raise ValueError("oracle gemm failed: %d" % rc)
    return OMat(*kc, A.p)


def gemm_counted(algo: int, A, B, cutoff: int = 64, policy: int = PEEL, nb: int = 32):
    m, l = A.exp.shape
    n = B.exp.shape[1]
    Cm = OMat.empty(m, n, A.p)
    ka, aa = _mat_args(A)
    kb, ab = _mat_args(B)
    kc, ac = _mat_args(Cm)
    mul, add = C.c_uint64(), C.c_uint64()
    rc = lib().orc_api_gemm_counted(C.c_int(algo), C.c_int(cutoff), C.c_int(policy),
                                    C.c_int(nb), C.c_int64(m), C.c_int64(l), C.c_int64(n),
                                    C.c_int(A.p), *aa, *ab, *ac, C.byref(mul), C.byref(add))
    if rc:
        raise ValueError("oracle gemm failed: %d" % rc)
    return OMat(*kc, A.p), mul.value, add.value


def count_model(algo: int, m: int, l: int, n: int, cutoff: int, policy: int = PEEL):
    mul, add = C.c_uint64(), C.c_uint64()
    lib().orc_api_count_model(C.c_int(algo), C.c_int64(m), C.c_int64(l), C.c_int64(n),
                              C.c_int(cutoff), C.c_int(policy), C.byref(mul), C.byref(add))
    return mul.value, add.value


def sample_set(side: int, algo: int, m: int, l: int, n: int, cutoff: int, policy: int,
               x0: int) -> np.ndarray:
    out = np.zeros(4096, np.int64)
    k = lib().orc_api_sample_set(C.c_int(side), C.c_int(algo), C.c_int64(m), C.c_int64(l),
                                 C.c_int64(n), C.c_int(cutoff), C.c_int(policy),
                                 C.c_int64(x0), _p(out), C.c_int64(4096))
    if k < 0:
        raise ValueError("sample set too large")
    return out[:k].copy()


def gemm_sampled(algo: int, A, B, rows, cols, cutoff: int = 64, policy: int = PEEL):
    m, l = A.exp.shape
    n = B.exp.shape[1]
    rows = np.ascontiguousarray(rows, np.int64)
    cols = np.ascontiguousarray(cols, np.int64)
    Cm = OMat.empty(len(rows), len(cols), A.p)
    ka, aa = _mat_args(A)
    kb, ab = _mat_args(B)
    kc, ac = _mat_args(Cm)
    rc = lib().orc_api_gemm_sampled(C.c_int(algo), C.c_int(cutoff), C.c_int(policy),
                                    C.c_int64(m), C.c_int64(l), C.c_int64(n), C.c_int(A.p),
                                    *aa, *ab, _p(rows), C.c_int64(len(rows)), _p(cols),
                                    C.c_int64(len(cols)), *ac)
    if rc:
        raise ValueError("oracle sampled gemm failed: %d" % rc)
    return OMat(*kc, A.p)


def dot_exact(A, B, rows=None, cols=None, p_out: int | None = None):
    """RN_{p_out}(exact sum_k a_ik b_kj) on rows x cols (all by default)."""
    m, l = A.exp.shape
    n = B.exp.shape[1]
    p_out = A.p if p_out is None else p_out
    rows = np.arange(m) if rows is None else rows
    cols = np.arange(n) if cols is None else cols
    rows = np.ascontiguousarray(rows, np.int64)
    cols = np.ascontiguousarray(cols, np.int64)
    Cm = OMat.empty(len(rows), len(cols), p_out)
    ka, aa = _mat_args(A)
    kb, ab = _mat_args(B)
    kc, ac = _mat_args(Cm)
    rc = lib().orc_api_dot_exact(C.c_int64(m), C.c_int64(l), C.c_int64(n), C.c_int(A.p),
                                 C.c_int(p_out), *aa, *ab, _p(rows), C.c_int64(len(rows)),
                                 _p(cols), C.c_int64(len(cols)), *ac)
    if rc:
        raise ValueError("oracle exact dot failed: %d" % rc)
    return OMat(*kc, p_out)


def lu(A, panel: int = 128, algo: int = SIMPLE, cutoff: int = 64, policy: int = PEEL,
       pivoting: bool = True):
    """Returns (LU factors, piv, status); status 0 ok, k+1 for a zero pivot in
    column k.  pivoting=False is the paper's LU (Sec. 4), piv[k] = k."""
    n = A.exp.shape[0]
    M = OMat(A.limb.copy(), A.exp.copy(), A.sign.copy(), A.p)
    piv = np.zeros(n, np.int64)
    km, am = _mat_args(M)
    rc = lib().orc_api_lu(C.c_int64(n), C.c_int(A.p), C.c_int(panel), C.c_int(algo),
                          C.c_int(cutoff), C.c_int(policy), C.c_int(1 if pivoting else 0), *am, _p(piv))
    return OMat(*km, A.p), piv, rc


def lu_solve(LU, piv, b):
    n = LU.exp.shape[0]
    X = OMat.empty(n, 1, LU.p)
    ka, aa = _mat_args(LU)
    kb, ab = _mat_args(b)
    kx, ax = _mat_args(X)
    piv = np.ascontiguousarray(piv, np.int64)
    rc = lib().orc_api_lu_solve(C.c_int64(n), C.c_int(LU.p), *aa, _p(piv), *ab, *ax)
    if rc:
        raise ValueError("oracle solve failed: %d" % rc)
    return OMat(*kx, LU.p)


# ---------------------------------------------------------------------------
# Section 4 benchmark matrices: a_ij = sqrt(5) (i + j - 1), b_ij = sqrt(3) (n - i + 1)
# ---------------------------------------------------------------------------
def sqrt_product_S(m: int, l: int, n: int) -> list:
    """The exact product of the Section 4 matrices is c_ij = sqrt(15) S_i with
    the integer S_i = sum_{k=1..l} (i + k - 1)(n - k + 1) (1-based; the same
    for every column j).  Returned as Python ints, summed term by term."""
    return [sum((i + k - 1) * (n - k + 1) for k in range(1, l + 1)) for i in range(1, m + 1)]


def _rn_sqrt15(S: int, q: int):
    """(sign, M, s): sqrt(15) S = (-1)^sign M 2^-s rounded to nearest at q bits
    (never a tie: sqrt(15) is irrational).  M = 0 for S = 0."""
    if S == 0:
        return (0, 0, 0)
    X = 15 * S * S
    s = max(0, q + 2 - (X.bit_length() + 1) // 2)
    R = math.isqrt(X << (2 * s))            # floor(sqrt(15) |S| 2^s), >= q + 2 bits
    d = R.bit_length() - q
    keep, low = R >> d, R & ((1 << d) - 1)
    if low >= 1 << (d - 1):                # the dropped part (plus an irrational tail) is >= half
        keep += 1
    if keep >> q:
        keep >>= 1
        d += 1
    return (1 if S < 0 else 0, keep, s - d)


def sqrt_product_rows(m: int, l: int, n: int, q: int) -> OMat:
    """RN_q(c_i) for the m distinct rows of the exact product (an m x 1 matrix)."""
    out = OMat.empty(m, 1, q)
    L = (q + 63) // 64
    for i, S in enumerate(sqrt_product_S(m, l, n)):
        sg, M, s = _rn_sqrt15(S, q)
        if M == 0:
            continue
        bl = M.bit_length()
        mant = M << (64 * L - bl)
        for k in range(L):
            out.limb[k, i, 0] = (mant >> (64 * (L - 1 - k))) & 0xFFFFFFFFFFFFFFFF
        out.exp[i, 0] = bl - s
        out.sign[i, 0] = sg
    return out


def sqrt_rel_errors(Cm, m: int, l: int, n: int) -> np.ndarray:
    """|c~_ij - c_ij| / |c_ij| for a computed product of the Section 4
    matrices, entry by entry, evaluated exactly: with x = c~_ij / S_i,
    |x - sqrt(15)| = |x^2 - 15| / (x + sqrt(15)).  Rows with S_i = 0 give inf
    unless the entry is 0 too.  For small matrices (Python integers)."""
    S = sqrt_product_S(m, l, n)
    L = Cm.limb.shape[0]
    r15 = math.sqrt(15.0)
    out = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            e = int(Cm.exp[i, j])
            if e == EXP_ZERO:
                out[i, j] = 0.0 if S[i] == 0 else 1.0
                continue
            v = 0
            for k in range(L):
                v = (v << 64) | int(Cm.limb[k, i, j])
            x = Fraction(-v if Cm.sign[i, j] else v, 1 << (64 * L)) * Fraction(2) ** e / S[i] \
                if S[i] else None
            if x is None:
                out[i, j] = math.inf
                continue
            if x <= 0:
                out[i, j] = 1.0 + float(-x) / r15
                continue
            out[i, j] = float(abs(x * x - 15)) / ((float(x) + r15) * r15)
    return out


# ---------------------------------------------------------------------------
# Sec. 4's ill-conditioned matrix: cond_1 of the Lotkin matrix, exactly
# ---------------------------------------------------------------------------
def lotkin_norm1_log2(n: int):
    """(log2 ||A||_1, log2 ||A^-1||_1) of the n x n Lotkin matrix (first row
    all ones, a_ij = 1/(i+j-1) below; Sec. 4), from exact integers.

    The Hilbert matrix H (h_ij = 1/(i+j-1)) has the integer inverse
    G_ij = (-1)^(i+j) a_i a_j / (i+j-1), a_i = (n+i-1)! / ((n-i)! ((i-1)!)^2)
    (the binomial closed form of H^-1 regrouped).  The Lotkin matrix is
    A = H + e_1 w^T with w_j = 1 - 1/j, so by Sherman and Morrison
    A^-1 = G - c r^T / d with c = G e_1, r^T = w^T G = s^T - e_1^T (s the
    column sums of G, since the first row of H times G is e_1^T) and
    d = 1 + w^T G e_1 = s_1: every entry is the integer d G_ij - c_i r_j over
    the common denominator d.  ||A||_1 is the first column's sum, the
    harmonic number H_n."""
    fact = [1] * (2 * n + 1)
    for k in range(1, 2 * n + 1):
        fact[k] = fact[k - 1] * k
    a = [0] + [fact[n + i - 1] // (fact[n - i] * fact[i - 1] ** 2) for i in range(1, n + 1)]

    def G(i, j):
        v = a[i] * a[j] // (i + j - 1)
        return -v if (i + j) & 1 else v

    s = [0] * (n + 1)
    for j in range(1, n + 1):
        s[j] = sum(G(i, j) for i in range(1, n + 1))
    d = s[1]
    c = [0] + [G(i, 1) for i in range(1, n + 1)]
    r = [0] + [s[j] - (1 if j == 1 else 0) for j in range(1, n + 1)]
    best = 0
    for j in range(1, n + 1):
        tot = sum(abs(d * G(i, j) - c[i] * r[j]) for i in range(1, n + 1))
        best = max(best, tot)

    def log2_int(v):
        shift = max(v.bit_length() - 60, 0)
        return math.log2(v >> shift) + shift

    def log2_ratio(num, den):
        return log2_int(num) - log2_int(den)

    hn = Fraction(1) + sum(Fraction(1, i) for i in range(2, n + 1))
    return log2_ratio(hn.numerator, hn.denominator), log2_ratio(best, abs(d))
