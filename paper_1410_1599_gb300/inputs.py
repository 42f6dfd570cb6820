"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds only the interchange container and the generators; it does
no multiple-precision arithmetic of the method (no rounded add, multiply or
divide).  Every value it produces is exactly representable in the requested
precision and is built with integer operations.

Interchange format of a rows x cols matrix at precision p, L = ceil(p/64):
    limb[k, r, c]  uint64   limb k of the mantissa, k = 0 most significant;
                            the mantissa is the fraction sum_k limb_k 2^(-64(k+1))
                            in [1/2, 1) with its top bit set
    exp[r, c]      int64    value = (-1)^sign * mantissa * 2^exp;
                            EXP_ZERO (INT64_MIN) marks zero
    sign[r, c]     int8     0 = +, 1 = -

Random draws use SplitMix64 (Steele, Lea, Flood 2014) as a counter-based
generator: word i of stream `seed` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

EXP_ZERO = np.iinfo(np.int64).min
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def limbs_for(p: int) -> int:
    return (p + 63) // 64


@dataclass
class HostMP:
    """A matrix of p-bit numbers in the interchange format (host memory)."""

    limb: np.ndarray  # (L, rows, cols) uint64
    exp: np.ndarray  # (rows, cols) int64
    sign: np.ndarray  # (rows, cols) int8
    p: int

    @property
    def shape(self):
        return self.exp.shape

    @property
    def L(self):
        return self.limb.shape[0]

    @staticmethod
    def zeros(rows: int, cols: int, p: int) -> "HostMP":
        L = limbs_for(p)
        return HostMP(np.zeros((L, rows, cols), np.uint64),
                      np.full((rows, cols), EXP_ZERO, np.int64),
                      np.zeros((rows, cols), np.int8), p)

    def copy(self) -> "HostMP":
        return HostMP(self.limb.copy(), self.exp.copy(), self.sign.copy(), self.p)

    def sub(self, rows, cols) -> "HostMP":
        """Entries at the given row and column index arrays (a new matrix)."""
        r = np.asarray(rows)[:, None]
        c = np.asarray(cols)[None, :]
        return HostMP(self.limb[:, r, c], self.exp[r, c], self.sign[r, c], self.p)

    def equal(self, other: "HostMP") -> bool:
        return (self.p == other.p and self.shape == other.shape
                and np.array_equal(self.limb, other.limb)
                and np.array_equal(self.exp, other.exp)
                and np.array_equal(self.sign, other.sign))

    def mismatches(self, other: "HostMP") -> np.ndarray:
        """Boolean (rows, cols) mask of entries whose bits differ."""
        return ((self.limb != other.limb).any(axis=0) | (self.exp != other.exp)
                | (self.sign != other.sign))

    # exact conversions, for building fixtures and reading results
    def to_fractions(self):
        out = []
        for r in range(self.shape[0]):
            row = []
            for c in range(self.shape[1]):
                row.append(entry_fraction(self, r, c))
            out.append(row)
        return out


def entry_int(M: HostMP, r: int, c: int) -> int:
    """Mantissa of entry (r, c) as an integer of 64*L bits."""
    v = 0
    for k in range(M.limb.shape[0]):
        v = (v << 64) | int(M.limb[k, r, c])
    return v


def entry_fraction(M: HostMP, r: int, c: int) -> Fraction:
    e = int(M.exp[r, c])
    if e == EXP_ZERO:
        return Fraction(0)
    v = Fraction(entry_int(M, r, c), 1 << (64 * M.limb.shape[0])) * (Fraction(2) ** e)
    return -v if M.sign[r, c] else v


def from_exact_ints(values, p: int, shape) -> HostMP:
    """Matrix of exact values given as (sign, integer numerator N, scale s),
    value = (-1)^sign N 2^-s, with N < 2^p (so no rounding is needed)."""
    rows, cols = shape
    M = HostMP.zeros(rows, cols, p)
    L = M.L
    for idx, (sg, N, s) in enumerate(values):
        r, c = divmod(idx, cols)
        if N == 0:
            M.sign[r, c] = sg
            continue
        bl = N.bit_length()
        assert bl <= p, "value needs more than p bits"
        mant = N << (64 * L - bl)
        for k in range(L):
            M.limb[k, r, c] = (mant >> (64 * (L - 1 - k))) & 0xFFFFFFFFFFFFFFFF
        M.exp[r, c] = bl - s
        M.sign[r, c] = sg
    return M


def from_ints(mat, p: int) -> HostMP:
    """Integer matrix (nested lists or 2-D array) to p-bit numbers."""
    a = [[int(x) for x in row] for row in mat]
    rows, cols = len(a), len(a[0]) if a else 0
    vals = [(1 if x < 0 else 0, abs(x), 0) for row in a for x in row]
    return from_exact_ints(vals, p, (rows, cols))


# ---------------------------------------------------------------------------
# SplitMix64
# ---------------------------------------------------------------------------
def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _clz64(v: np.ndarray) -> np.ndarray:
    """Leading zero bits of nonzero uint64 values."""
    v = v.copy()
    n = np.zeros(v.shape, np.int64)
    for s in (32, 16, 8, 4, 2, 1):
        m = (v >> np.uint64(64 - s)) == 0
        n += np.where(m, s, 0)
        v = np.where(m, v << np.uint64(s), v)
    return n


def _normalize(X: np.ndarray, over: np.ndarray):
    """X: (N, L) uint64 fixed-point fractions (limb 0 most significant), value
    X / 2^(64L) + over (over in {0,1}, set only when X == 0).  Returns the
    normalised (N, L) mantissas, exponents and a zero mask."""
    N, L = X.shape
    nz = X != 0
    first = np.where(nz.any(axis=1), nz.argmax(axis=1), L)
    zero = (first == L) & (over == 0)
    lead = X[np.arange(N), np.minimum(first, L - 1)]
    lead = np.where(first < L, lead, np.uint64(1))
    z = first * 64 + _clz64(lead)
    z = np.where(first < L, z, 0)
    out = np.empty_like(X)
    # common case: the leading one is in limb 0, an in-limb shift by zb < 64
    fast = first == 0
    zb = z[fast].astype(np.uint64)[:, None]
    Xf = X[fast]
    nxt = np.concatenate([Xf[:, 1:], np.zeros((Xf.shape[0], 1), np.uint64)], axis=1)
    sh = np.where(zb == 0, Xf, (Xf << zb) | (nxt >> (np.uint64(64) - np.where(zb == 0, 1, zb).astype(np.uint64))))
    out[fast] = sh
    # rare case: whole limbs of leading zeros (or zero), element by element
    for r in np.nonzero(~fast)[0]:
        zw_r, zb_r = int(z[r]) // 64, int(z[r]) % 64
        v = 0
        for t in range(L):
            v = (v << 64) | int(X[r, t])
        v = (v << (64 * zw_r + zb_r)) & ((1 << (64 * L)) - 1)
        for t in range(L):
            out[r, t] = (v >> (64 * (L - 1 - t))) & 0xFFFFFFFFFFFFFFFF
    exp = -z
    # the value exactly 1.0 (X wrapped to 0 with the carry in `over`)
    one = (over == 1)
    out[one, :] = 0
    out[one, 0] = np.uint64(1) << np.uint64(63)
    exp = np.where(one, 1, exp)
    out[zero, :] = 0
    exp = np.where(zero, EXP_ZERO, exp)
    return out, exp.astype(np.int64), zero


def uniform_pm1(rows: int, cols: int, p: int, seed: int, exp_lo: int = 0,
                exp_hi: int = 0) -> HostMP:
    """Entries v * 2^e, v uniform on the grid k / 2^(p-1), k in [-2^(p-1), 2^(p-1)),
    i.e. uniform in [-1, 1) and exact in p bits; e uniform in [exp_lo, exp_hi]."""
    M = HostMP.zeros(rows, cols, p)
    N = rows * cols
    limb, exp, sign = M.limb.reshape(M.L, N), M.exp.reshape(N), M.sign.reshape(N)
    # element t takes draws t(L+1)+1 .. t(L+1)+L+1; chunks keep the
    # temporaries cache-sized and give the same values as one pass
    for s0 in range(0, N, _CHUNK):
        cnt = min(_CHUNK, N - s0)
        mant, ex, neg = _uniform_pm1_flat(cnt, s0, p, seed, exp_lo, exp_hi)
        limb[:, s0:s0 + cnt] = mant.T
        exp[s0:s0 + cnt] = ex
        sign[s0:s0 + cnt] = neg
    return M


_CHUNK = 1 << 12


def _uniform_pm1_flat(N: int, first: int, p: int, seed: int, exp_lo: int, exp_hi: int):
    """Entries first .. first+N-1 of uniform_pm1 in row-major order:
    (N, L) mantissas, exponents (EXP_ZERO for zeros) and signs."""
    L = limbs_for(p)
    w = splitmix64(seed, N * (L + 1), first * (L + 1)).reshape(N, L + 1)
    neg = (w[:, 0] & np.uint64(1)).astype(np.int8)
    span = exp_hi - exp_lo + 1
    e = exp_lo + ((w[:, 0] >> np.uint64(1)) % np.uint64(span)).astype(np.int64)
    X = w[:, 1:].copy()
    # keep the top p-1 bits of the 64L-bit string: j in [0, 2^(p-1))
    drop = 64 * L - (p - 1)
    for t in range(L - 1, -1, -1):
        lo_bit = 64 * (L - 1 - t)  # bit index of this limb's LSB in the string
        k = min(max(drop - lo_bit, 0), 64)
        if k == 64:
            X[:, t] = 0
        elif k > 0:
            X[:, t] &= ~np.uint64((1 << k) - 1)
    # negative half: |k| = j + 1, one unit at bit `drop` of the string
    over = np.zeros(N, np.int64)
    carry = neg.astype(np.uint64)
    unit_limb = L - 1 - drop // 64
    unit = np.uint64(1) << np.uint64(drop % 64)
    for t in range(unit_limb, -1, -1):
        add = np.where(carry == 1, unit if t == unit_limb else np.uint64(1), np.uint64(0))
        with np.errstate(over="ignore"):
            s = X[:, t] + add
        carry = ((s < X[:, t]) & (add > 0)).astype(np.uint64)
        X[:, t] = s
    over = carry.astype(np.int64)
    mant, exp, zero = _normalize(X, over)
    return mant, np.where(zero, EXP_ZERO, exp + e), neg


def rand_bits(seed: int, index: int, bits: int) -> int:
    """An integer of `bits` random bits: draw `index` of stream `seed`."""
    nwords = (bits + 63) // 64
    v = 0
    for x in splitmix64(seed, nwords, offset=index * nwords):
        v = (v << 64) | int(x)
    return v >> (64 * nwords - bits)


def well_conditioned(n: int, p: int, seed: int) -> HostMP:
    """A = U[-1,1) + n I.  Off-diagonal entries as uniform_pm1; the diagonal is
    n + v with v uniform on the grid k / 2^q, k in [-2^q, 2^q),
    q = p - bitlen(n) - 2, so that n + v is exact in p bits."""
    A = uniform_pm1(n, n, p, seed)
    q = p - n.bit_length() - 2
    vals = []
    for i in range(n):
        k = rand_bits(seed ^ 0x5DEECE66D, i, q + 1) - (1 << q)
        num = (n << q) + k
        vals.append((0 if num >= 0 else 1, abs(num), q))
    D = from_exact_ints(vals, p, (1, n))
    for i in range(n):
        A.limb[:, i, i] = D.limb[:, 0, i]
        A.exp[i, i] = D.exp[0, i]
        A.sign[i, i] = D.sign[0, i]
    return A


def rn_reciprocal(d: int, p: int):
    """(sign, N, s) with N 2^-s = 1/d rounded to nearest-even at p bits, d >= 1."""
    t = d.bit_length()
    if d & (d - 1) == 0:
        return (0, 1, t - 1)
    Q, R = divmod(1 << (p + t - 1), d)
    if 2 * R > d or (2 * R == d and Q & 1):
        Q += 1
    return (0, Q, p + t - 1)


def lotkin(n: int, p: int) -> HostMP:
    """First row all ones; a_ij = 1/(i+j-1) (1-based) rounded to p bits.
    Only 2n distinct values occur: they are built once and gathered."""
    table = from_exact_ints([rn_reciprocal(d, p) if d > 0 else (0, 1, 0) for d in range(2 * n + 1)],
                            p, (1, 2 * n + 1))
    one = from_exact_ints([(0, 1, 0)], p, (1, 1))
    d = np.arange(n)[:, None] + np.arange(n)[None, :] + 1          # 0-based i + j + 1
    M = HostMP(np.ascontiguousarray(table.limb[:, 0, :][:, d]), table.exp[0, d].copy(),
               table.sign[0, d].copy(), p)
    M.limb[:, 0, :] = one.limb[:, 0, :1]
    M.exp[0, :] = one.exp[0, 0]
    M.sign[0, :] = 0
    return M


def ones(rows: int, cols: int, p: int) -> HostMP:
    return from_exact_ints([(0, 1, 0)] * (rows * cols), p, (rows, cols))


def identity(n: int, p: int) -> HostMP:
    return from_exact_ints([(0, 1 if i == j else 0, 0) for i in range(n) for j in range(n)],
                           p, (n, n))


def small_ints(rows: int, cols: int, p: int, seed: int, bits: int) -> HostMP:
    """Integers uniform in (-2^bits, 2^bits)."""
    w = splitmix64(seed, rows * cols)
    vals = []
    for x in w:
        x = int(x)
        mag = (x >> 1) & ((1 << bits) - 1)
        vals.append((x & 1 if mag else 0, mag, 0))
    return from_exact_ints(vals, p, (rows, cols))


def rn_sqrt(N: int, p: int):
    """(sign, M, s) with M 2^-s = sqrt(N) rounded to nearest-even at p bits,
    N >= 1 an integer.  sqrt(N) of a non-square N is irrational, so no tie
    occurs; for a square the root is exact."""
    t = (N.bit_length() + 1) // 2                  # sqrt(N) < 2^t
    s = p + 2 - t if p + 2 > t else 0              # root of N 4^s has >= p + 2 bits
    X = N << (2 * s)
    Q = math.isqrt(X)
    sticky = Q * Q != X
    d = Q.bit_length() - p
    if d <= 0:
        return (0, Q, s)
    rem, Q = Q & ((1 << d) - 1), Q >> d
    half = 1 << (d - 1)
    if rem > half or (rem == half and (sticky or Q & 1)):
        Q += 1
    if Q >> p:                                     # rounded up to 2^p
        Q >>= 1
        d += 1
    return (0, Q, s - d)


def sqrt_matrices(m: int, l: int, n: int, p: int, b_cols: int | None = None):
    """The benchmark matrices of the paper's Section 4 ("Benchmark tests of
    square and rectangle matrix multiplications"): a_ij = sqrt(5) (i + j - 1)
    (m x l) and b_ij = sqrt(3) (n - i + 1) (l x n), 1-based, with n the
    literal column count of B.  Each entry is the exact value rounded once
    to p bits, RN_p(sqrt(5 k^2)).  a_ij depends on i + j only and b_ij on i
    only: the distinct values are built once and gathered.  b_cols (default
    n) narrows B to its first columns, which are all alike."""
    def table(c, ks, idx):
        """RN_p(sqrt(c) k) for the integers ks, gathered by idx."""
        ex = [(0, 0, 0) if k == 0 else (1 if k < 0 else 0,) + rn_sqrt(c * k * k, p)[1:] for k in ks]
        T = from_exact_ints(ex, p, (1, len(ex)))
        return HostMP(np.ascontiguousarray(T.limb[:, 0, :][:, idx]), T.exp[0, idx].copy(),
                      T.sign[0, idx].copy(), p)

    A = table(5, range(1, m + l), np.arange(m)[:, None] + np.arange(l)[None, :])     # k = i + j - 1
    B = table(3, [n - i + 1 for i in range(1, l + 1)],
              np.broadcast_to(np.arange(l)[:, None], (l, n if b_cols is None else b_cols)))
    return A, B
