// mp_arith.cuh -- device multiple-precision arithmetic in registers.
//
// A number is held as W little-endian 32-bit words (capacity 32W bits) plus
// an int64 exponent and a sign: value = (-1)^s * m * 2^(e - 32W) with the top
// bit of m[W-1] set (m read as an integer), i.e. a mantissa fraction in
// [1/2, 1).  A precision-p number uses the top p bits; the rest are zero.
// Zero is e == EXP_ZERO with m == 0.
//
// Every operation returns the exact result rounded once to p bits, ties to
// even (arXiv 1410.1599, Sec. 1 and 3: MPFR semantics), so results do not
// depend on W: a p-bit operation gives the same bits in any W >= 2*ceil(p/64).
//
// Classes up to W = 64 (2048 bits) are written for registers: every loop over
// the words is unrolled so that indices are constants.  The wide class above
// 2048 bits (W = BIG_W, the paper's precisions up to 8650 bits) keeps its
// numbers in local memory and takes the same steps in plain loops (the
// big_* routines below), which keeps its code small enough to compile.
#pragma once
#include <cstdint>

#include "mp_internal.h"

#define MP_DEV __device__ __forceinline__

namespace mpg {

constexpr int64_t EXP_ZERO = INT64_MIN;
constexpr int64_t EXP_LIMIT = (int64_t)1 << 62;
template <int W>
constexpr bool is_big() { return W > 64; }

// ---------------------------------------------------------------- carry chains
MP_DEV uint32_t add_cc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
MP_DEV uint32_t addc_cc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
MP_DEV uint32_t addc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("addc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
MP_DEV uint32_t sub_cc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
MP_DEV uint32_t subc_cc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
MP_DEV uint32_t subc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("subc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
MP_DEV uint32_t mad_lo_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("mad.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }
MP_DEV uint32_t madc_lo_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("madc.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }
MP_DEV uint32_t mad_hi_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("mad.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }
MP_DEV uint32_t madc_hi_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("madc.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }
MP_DEV uint32_t madc_hi(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("madc.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }

// Per-launch constants derived from the precision p and the capacity W.
struct RoundSpec {
    int p;        // precision in bits
    int r;        // 32W - p: bits below the kept least significant bit
    int rw, rb;   // r = 32 * rw + rb
    int L;        // storage limbs, ceil(p / 64)
};

template <int W>
MP_DEV RoundSpec make_spec(int p)
{
    RoundSpec s;
    s.p = p;
    s.r = 32 * W - p;
    s.rw = s.r >> 5;
    s.rb = s.r & 31;
    s.L = (p + 63) >> 6;
    return s;
}

template <int W>
struct Mp {
    uint32_t m[W];
    int64_t e;
    uint32_t s;
};

template <int W>
MP_DEV void set_zero(Mp<W> &x, uint32_t sign)
{
    if constexpr (is_big<W>()) {
#pragma unroll 4
        for (int i = 0; i < W; ++i) x.m[i] = 0u;
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) x.m[i] = 0u;
    }
    x.e = EXP_ZERO;
    x.s = sign;
}

// ------------------------------------------------------ wide class (W > 64)
// The steps of round_mant, add_impl, mul_impl, div_impl and cmpabs below,
// written as plain loops over the words (numbers in local memory).

// round m (W words, top bit set) to p bits, nearest-even (see round_mant)
template <int W>
__device__ __noinline__ void big_round(uint32_t *m, int64_t &e, uint32_t below, bool sticky,
                                       const RoundSpec &rs)
{
    uint32_t rbit, st, lsb;
    if (rs.r == 0) {
        rbit = below >> 31;
        st = (below << 1) | (sticky ? 1u : 0u);
        lsb = m[0] & 1u;
    } else {
        const int q = rs.r - 1, qw = q >> 5, qb = q & 31;
        rbit = (m[qw] >> qb) & 1u;
        st = below | (sticky ? 1u : 0u) | (m[qw] & ((1u << qb) - 1u));
        for (int i = 0; i < qw; ++i) st |= m[i];
        for (int i = 0; i < rs.rw; ++i) m[i] = 0u;
        m[rs.rw] &= ~((1u << rs.rb) - 1u);
        lsb = (m[rs.rw] >> rs.rb) & 1u;
    }
    if (rbit && (st | lsb)) {
        uint64_t c = (uint64_t)1 << rs.rb;               // m += 2^r
        for (int i = rs.rw; i < W && c; ++i) {
            c += m[i];
            m[i] = (uint32_t)c;
            c >>= 32;
        }
        if (c) {                                         // carried out of the top
            for (int i = 0; i < W; ++i) m[i] = 0u;
            m[W - 1] = 0x80000000u;
            e += 1;
        }
    }
}

// x (N words) >>= sh bits, 0 <= sh <= 32N; returns the OR of the bits shifted out
MP_DEV uint32_t big_shr_sticky(uint32_t *x, int N, int sh)
{
    const int q = sh >> 5, b = sh & 31;
    uint32_t st = 0u;
    if (q >= N) {
        for (int i = 0; i < N; ++i) {
            st |= x[i];
            x[i] = 0u;
        }
        return st;
    }
    for (int i = 0; i < q; ++i) st |= x[i];
    for (int i = 0; i < N; ++i) x[i] = (i + q < N) ? x[i + q] : 0u;
    st |= x[0] & ((1u << b) - 1u);
    for (int i = 0; i < N - 1; ++i) x[i] = __funnelshift_r(x[i], x[i + 1], b);
    x[N - 1] >>= b;
    return st;
}

// x (N words) <<= sh bits, 0 <= sh < 32N
MP_DEV void big_shl(uint32_t *x, int N, int sh)
{
    const int q = sh >> 5, b = sh & 31;
    for (int i = N - 1; i >= 0; --i) x[i] = (i - q >= 0) ? x[i - q] : 0u;
    for (int i = N - 1; i > 0; --i) x[i] = __funnelshift_l(x[i - 1], x[i], b);
    x[0] <<= b;
}

// leading zero bits of an N-word number (32N when zero)
MP_DEV int big_clz(const uint32_t *x, int N)
{
    for (int i = N - 1; i >= 0; --i)
        if (x[i]) return 32 * (N - 1 - i) + __clz(x[i]);
    return 32 * N;
}

template <int W>
__device__ __noinline__ int big_cmpabs(const Mp<W> &a, const Mp<W> &b)
{
    const bool az = a.e == EXP_ZERO, bz = b.e == EXP_ZERO;
    if (az | bz) return (az && bz) ? 0 : (az ? -1 : 1);
    if (a.e != b.e) return a.e < b.e ? -1 : 1;
    for (int i = W - 1; i >= 0; --i)
        if (a.m[i] != b.m[i]) return a.m[i] < b.m[i] ? -1 : 1;
    return 0;
}

// r = RN_p(x + (-1)^neg_y y), the steps of add_impl; r may alias x or y
template <int W>
__device__ __noinline__ void big_add(Mp<W> &r, const Mp<W> &x, const Mp<W> &y, uint32_t neg_y,
                                     const RoundSpec &rs)
{
    const uint32_t ys = y.s ^ neg_y;
    const bool xz = x.e == EXP_ZERO, yz = y.e == EXP_ZERO;
    if (xz | yz) {
        if (xz & yz) {
            const uint32_t zs = x.s & ys;
            for (int i = 0; i < W; ++i) r.m[i] = 0u;
            r.e = EXP_ZERO;
            r.s = zs;
            return;
        }
        if (xz) {
            for (int i = 0; i < W; ++i) r.m[i] = y.m[i];
            r.e = y.e;
            r.s = ys;
        } else if (&r != &x) {
            for (int i = 0; i < W; ++i) r.m[i] = x.m[i];
            r.e = x.e;
            r.s = x.s;
        }
        return;
    }
    int mc = 0;
    for (int i = W - 1; i >= 0 && mc == 0; --i)
        if (x.m[i] != y.m[i]) mc = x.m[i] < y.m[i] ? -1 : 1;
    const bool sw = (y.e > x.e) || (y.e == x.e && mc < 0);
    uint32_t X[W + 1], Y[W + 1];
    X[0] = 0u;
    Y[0] = 0u;
    for (int i = 0; i < W; ++i) {
        X[i + 1] = sw ? y.m[i] : x.m[i];
        Y[i + 1] = sw ? x.m[i] : y.m[i];
    }
    int64_t e = sw ? y.e : x.e;
    const int64_t d64 = sw ? (y.e - x.e) : (x.e - y.e);
    const uint32_t sx = sw ? ys : x.s;
    const uint32_t eff_sub = (x.s ^ ys) & 1u;
    const int d = d64 > 32 * (W + 1) ? 32 * (W + 1) : (int)d64;
    const uint32_t st = big_shr_sticky(Y, W + 1, d);
    const uint32_t mask = 0u - eff_sub;
    uint64_t c = eff_sub & (st == 0u ? 1u : 0u);
    for (int i = 0; i <= W; ++i) {
        c += (uint64_t)X[i] + (uint64_t)(Y[i] ^ mask);
        X[i] = (uint32_t)c;
        c >>= 32;
    }
    const uint32_t rsh = (eff_sub ^ 1u) & (uint32_t)c & 1u;
    bool sticky = st != 0u;
    if (rsh) {
        sticky |= (X[0] & 1u) != 0u;
        for (int i = 0; i < W; ++i) X[i] = __funnelshift_r(X[i], X[i + 1], 1);
        X[W] = (X[W] >> 1) | 0x80000000u;
        e += 1;
    }
    const int lz = big_clz(X, W + 1);
    if (lz == 32 * (W + 1)) {                     // exact cancellation: +0
        for (int i = 0; i < W; ++i) r.m[i] = 0u;
        r.e = EXP_ZERO;
        r.s = 0u;
        return;
    }
    big_shl(X, W + 1, lz);
    e -= lz;
    for (int i = 0; i < W; ++i) r.m[i] = X[i + 1];
    big_round<W>(r.m, e, X[0], sticky, rs);
    r.e = e;
    r.s = sx;
}

// r = RN_p(a * b) from the full 2W-word product; r may alias a or b
template <int W>
__device__ __noinline__ void big_mul(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    const uint32_t s = a.s ^ b.s;
    if (a.e == EXP_ZERO || b.e == EXP_ZERO) {
        for (int i = 0; i < W; ++i) r.m[i] = 0u;
        r.e = EXP_ZERO;
        r.s = s;
        return;
    }
    int64_t e = a.e + b.e;
    // Schoolbook product, CH words of a at a time held in registers: rows of
    // b run through a register window of CH + 1 words, and each finished
    // window word is added into P (local memory) once, with a running carry,
    // so P is touched once per CH partial products.
    constexpr int CH = 16;
    static_assert(W % CH == 0, "chunked product");
    uint32_t P[2 * W];
    for (int i = 0; i < 2 * W; ++i) P[i] = 0u;
    for (int i0 = 0; i0 < W; i0 += CH) {
        uint32_t ac[CH], w[CH + 1];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            ac[u] = a.m[i0 + u];
            w[u] = 0u;
        }
        w[CH] = 0u;
        uint64_t cp = 0;
        for (int j = 0; j < W; ++j) {
            const uint32_t bj = b.m[j];
            uint64_t c = 0;
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const uint64_t t = (uint64_t)ac[u] * bj + w[u] + c;
                w[u] = (uint32_t)t;
                c = t >> 32;
            }
            w[CH] = (uint32_t)c;
            const uint64_t sm = (uint64_t)P[i0 + j] + w[0] + cp;   // position i0 + j is final
            P[i0 + j] = (uint32_t)sm;
            cp = sm >> 32;
#pragma unroll
            for (int u = 0; u < CH; ++u) w[u] = w[u + 1];
            w[CH] = 0u;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {                // the window's last words
            const uint64_t sm = (uint64_t)P[i0 + W + u] + w[u] + cp;
            P[i0 + W + u] = (uint32_t)sm;
            cp = sm >> 32;
        }
        for (int k = i0 + W + CH; k < 2 * W && cp; ++k) {
            const uint64_t sm = (uint64_t)P[k] + cp;
            P[k] = (uint32_t)sm;
            cp = sm >> 32;
        }
    }
    uint32_t low = 0u;
    for (int i = 0; i < W - 2; ++i) low |= P[i];
    uint32_t below = P[W - 1], below2 = P[W - 2];
    if (!(P[2 * W - 1] >> 31)) {                  // product in [1/4, 1/2): shift left one
        for (int i = 2 * W - 1; i > W; --i) P[i] = __funnelshift_l(P[i - 1], P[i], 1);
        P[W] = __funnelshift_l(below, P[W], 1);
        below = __funnelshift_l(below2, below, 1);
        below2 <<= 1;
        e -= 1;
    }
    for (int i = 0; i < W; ++i) r.m[i] = P[W + i];
    big_round<W>(r.m, e, below, (low | below2) != 0u, rs);
    r.e = e;
    r.s = s;
}

// r = RN_p(a / b), b != 0: the long division of div_impl.  The remainder is
// a window R = buf[base .. base + W] that moves down one word per digit
// (R <- R 2^32 without moving words) and the digits go straight to their
// place in Q.
template <int W>
__device__ __noinline__ void big_div(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    const uint32_t s = a.s ^ b.s;
    if (a.e == EXP_ZERO || b.e == EXP_ZERO) {
        for (int i = 0; i < W; ++i) r.m[i] = 0u;
        r.e = EXP_ZERO;
        r.s = s;
        return;
    }
    uint32_t buf[2 * W + 2], Q[W + 2];
    int base = W + 1;
    uint32_t br = 0u;
    for (int i = 0; i < W; ++i) {                 // R = A - D when A >= D
        const uint64_t df = (uint64_t)a.m[i] - b.m[i] - br;
        buf[base + i] = (uint32_t)df;
        br = (uint32_t)(df >> 63);
    }
    const uint32_t q0 = br ? 0u : 1u;
    if (!q0)
        for (int i = 0; i < W; ++i) buf[base + i] = a.m[i];
    buf[base + W] = 0u;
    Q[W + 1] = q0;
    const uint32_t d1 = b.m[W - 1], d2 = b.m[W - 2];
    const uint32_t v = (uint32_t)(0xffffffffffffffffull / d1 - 0x100000000ull);
    for (int t = 0; t <= W; ++t) {
        buf[--base] = 0u;                         // R <- R 2^32 (its top word was zero)
        uint32_t *R = buf + base;
        const uint32_t u1 = R[W], u0 = R[W - 1];
        uint64_t qh, rh;
        if (u1 >= d1) {
            qh = 0xffffffffull;
            rh = (((uint64_t)u1 << 32) | u0) - qh * d1;
        } else {
            const uint64_t tt = (uint64_t)v * u1 + (((uint64_t)u1 << 32) | u0);
            uint32_t q1 = (uint32_t)(tt >> 32) + 1u;
            const uint32_t ql = (uint32_t)tt;
            uint32_t rr = u0 - q1 * d1;
            if (rr > ql) { q1 -= 1u; rr += d1; }
            if (rr >= d1) { q1 += 1u; rr -= d1; }
            qh = q1;
            rh = rr;
        }
        for (int c = 0; c < 2 && rh <= 0xffffffffull && qh * d2 > ((rh << 32) | R[W - 2]); ++c) {
            --qh;
            rh += d1;
        }
        const uint32_t q = (uint32_t)qh;
        uint64_t cy = 0;
        uint32_t bw = 0u;
        for (int i = 0; i < W; ++i) {
            const uint64_t pr = (uint64_t)b.m[i] * q + cy;
            cy = pr >> 32;
            const uint64_t df = (uint64_t)R[i] - (uint32_t)pr - bw;
            R[i] = (uint32_t)df;
            bw = (uint32_t)(df >> 63);
        }
        const uint64_t dt = (uint64_t)R[W] - cy - bw;
        R[W] = (uint32_t)dt;
        uint32_t qd = q;
        if (dt >> 63) {                           // one too large: add D back
            uint64_t c = 0;
            for (int i = 0; i < W; ++i) {
                c += (uint64_t)R[i] + b.m[i];
                R[i] = (uint32_t)c;
                c >>= 32;
            }
            R[W] += (uint32_t)c;
            qd -= 1u;
        }
        Q[W - t] = qd;
    }
    bool rem = false;
    for (int i = 0; i < W; ++i) rem |= buf[base + i] != 0u;
    const int lz = q0 ? 31 : 32;
    big_shl(Q, W + 2, lz);
    int64_t e = a.e - b.e + 32 - lz;
    for (int i = 0; i < W; ++i) r.m[i] = Q[i + 2];
    big_round<W>(r.m, e, Q[1], rem || Q[0] != 0u, rs);
    r.e = e;
    r.s = s;
}

// ------------------------------------------------------------- load / store
// Limb k (0 = most significant) of a storage number with L limbs occupies
// words W-1-2k (high half) and W-2-2k (low half).
template <int W>
MP_DEV void load(Mp<W> &x, const uint64_t *__restrict__ limb, const int64_t *__restrict__ exp,
                 const int8_t *__restrict__ sign, int64_t off, int64_t plane, int L)
{
#pragma unroll (is_big<W>() ? 4 : W / 2)
    for (int k = 0; k < W / 2; ++k) {
        uint64_t v = (k < L) ? __ldg(limb + (int64_t)k * plane + off) : 0ull;
        x.m[W - 1 - 2 * k] = (uint32_t)(v >> 32);
        x.m[W - 2 - 2 * k] = (uint32_t)v;
    }
    x.e = __ldg(exp + off);
    x.s = (uint32_t)(__ldg(sign + off) & 1);
}

// load that treats out-of-range positions as +0 (zero padding)
template <int W>
MP_DEV void load_or_zero(Mp<W> &x, bool valid, const uint64_t *__restrict__ limb,
                         const int64_t *__restrict__ exp, const int8_t *__restrict__ sign,
                         int64_t off, int64_t plane, int L)
{
    if (valid) load<W>(x, limb, exp, sign, off, plane, L);
    else set_zero<W>(x, 0u);
}

template <int W>
MP_DEV void store(const Mp<W> &x, uint64_t *__restrict__ limb, int64_t *__restrict__ exp,
                  int8_t *__restrict__ sign, int64_t off, int64_t plane, int L)
{
#pragma unroll (is_big<W>() ? 4 : W / 2)
    for (int k = 0; k < W / 2; ++k)
        if (k < L)
            limb[(int64_t)k * plane + off] =
                ((uint64_t)x.m[W - 1 - 2 * k] << 32) | (uint64_t)x.m[W - 2 - 2 * k];
    exp[off] = x.e;
    sign[off] = (int8_t)x.s;
}

// exponent check of a finished result (zero is always in range)
template <int W>
MP_DEV bool out_of_range(const Mp<W> &x)
{
    return x.e != EXP_ZERO && (x.e > EXP_LIMIT || x.e < -EXP_LIMIT);
}

// ------------------------------------------------------------------ rounding
// Round the W-word mantissa m (top bit set) to p bits, nearest-even.  `below`
// is the word directly under m and `sticky` says whether anything lies below
// that.  Bits of m under the kept LSB are cleared.  A carry out of the top
// renormalises to 1/2 and increments e.
template <int W>
MP_DEV void round_mant_reg(uint32_t (&m)[W], int64_t &e, uint32_t below, bool sticky,
                           const RoundSpec &rs)
{
    if (rs.r == 0) {
        // p = 32 W: the kept LSB is bit 0 of m[0]; the round bit tops `below`
        const uint32_t rbit = below >> 31;
        const uint32_t st = (below << 1) | (sticky ? 1u : 0u);
        const uint32_t up = rbit & ((st != 0u) | (m[0] & 1u));
        m[0] = add_cc(m[0], up);
#pragma unroll
        for (int i = 1; i < W; ++i) m[i] = addc_cc(m[i], 0u);
        const uint32_t c = addc(0u, 0u);
        if (c) {   // carried out of the top: m was all ones
            m[W - 1] = 0x80000000u;
            e += 1;
        }
        return;
    }
    uint32_t rbit, st;
    // round bit is bit r-1 of m; sticky is everything under it
    const int q = rs.r - 1;
    const int qw = q >> 5, qb = q & 31;
    rbit = 0u;
    st = below | (sticky ? 1u : 0u);
#pragma unroll
    for (int i = 0; i < W; ++i) {
        uint32_t w = m[i];
        if (i == qw) {
            rbit = (w >> qb) & 1u;
            st |= w & ((1u << qb) - 1u);
        } else if (i < qw) {
            st |= w;
        }
    }
    // clear the bits under the kept LSB (bit r)
#pragma unroll
    for (int i = 0; i < W; ++i) {
        if (i < rs.rw) m[i] = 0u;
        else if (i == rs.rw) m[i] &= ~((1u << rs.rb) - 1u);
    }
    uint32_t lsb = 0u;
#pragma unroll
    for (int i = 0; i < W; ++i)
        if (i == rs.rw) lsb = (m[i] >> rs.rb) & 1u;
    if (rbit && (st | lsb)) {
        // m += 2^r
        uint32_t c = 0u;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            uint32_t add = (i == rs.rw) ? (1u << rs.rb) : 0u;
            uint32_t s1 = m[i] + add;
            uint32_t c1 = s1 < add;
            uint32_t s2 = s1 + c;
            c = c1 | (s2 < c);
            m[i] = s2;
        }
        if (c) {   // carried out of the top: m was all ones above r
#pragma unroll
            for (int i = 0; i < W; ++i) m[i] = 0u;
            m[W - 1] = 0x80000000u;
            e += 1;
        }
    }
}

template <int W>
MP_DEV void round_mant(uint32_t (&m)[W], int64_t &e, uint32_t below, bool sticky,
                       const RoundSpec &rs)
{
    if constexpr (is_big<W>()) big_round<W>(m, e, below, sticky, rs);
    else round_mant_reg<W>(m, e, below, sticky, rs);
}

// ------------------------------------------------------------ multiplication
// Schoolbook products by rows of b.  Each partial product a_i b_j is formed
// with the running row carry as one 64-bit multiply-add
// (a_i b_j + P + c <= 2^64 - 1), which needs fewer instructions than
// separate low/high multiply-add carry chains.
//
// P (2W words) = a * b
template <int W>
MP_DEV void mul_full(uint32_t (&P)[2 * W], const uint32_t (&a)[W], const uint32_t (&b)[W])
{
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) P[i] = 0u;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const uint32_t bj = b[j];
        uint64_t c = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint64_t t = (uint64_t)a[i] * bj + P[i + j] + c;
            P[i + j] = (uint32_t)t;
            c = t >> 32;
        }
        P[j + W] = (uint32_t)c;            // not yet written by any row
    }
}

// Truncated product: the partial products a_i b_j with i + j >= W - 2 only.
// The result T satisfies T <= a b < T + (W - 1) 2^(32(W-1)): the omitted
// columns 0 .. W-3 sum to less than (W - 2) 2^(32(W-1)) and their carries
// into word W-1 are at most W - 2.  Words W-1 .. 2W-1 of T are returned in
// P[W-1 .. 2W-1] (lower words are scratch).
template <int W>
MP_DEV void mul_trunc(uint32_t (&P)[2 * W], const uint32_t (&a)[W], const uint32_t (&b)[W])
{
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) P[i] = 0u;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const uint32_t bj = b[j];
        const int i0 = (W - 2 - j > 0) ? W - 2 - j : 0;
        uint64_t c = 0;
#pragma unroll
        for (int i = i0; i < W; ++i) {
            const uint64_t t = (uint64_t)a[i] * bj + P[i + j] + c;
            P[i + j] = (uint32_t)t;
            c = t >> 32;
        }
        P[j + W] = (uint32_t)c;
    }
}

// Top half of a * b by a sliding window over the product, for large W where
// a fully unrolled 2W-word product is too much code: rows of b are taken four
// at a time (outer loop not unrolled); after each group the four lowest
// window words are final and leave the window.  Returns the top W words in
// hi, the two words just below them (P[W-1], P[W-2]) and whether anything
// below those is nonzero.
// b is anything indexable by word: an array, a pointer or a reader of
// shared-memory limb planes.
template <int W, class BW>
MP_DEV void mul_top(uint32_t (&hi)[W], uint32_t &pw1, uint32_t &pw2, bool &low_nz,
                    const uint32_t (&a)[W], const BW &b)
{
    static_assert(W % 4 == 0, "W must be a multiple of 4");
    uint32_t acc[W + 4];
#pragma unroll
    for (int i = 0; i < W + 4; ++i) acc[i] = 0u;
    uint32_t st = 0u;
    pw1 = pw2 = 0u;
#pragma unroll 1
    for (int j = 0; j < W; j += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t bj = b[j + u];
            uint64_t c = 0;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const uint64_t t = (uint64_t)a[i] * bj + acc[u + i] + c;
                acc[u + i] = (uint32_t)t;
                c = t >> 32;
            }
            acc[u + W] = (uint32_t)c;      // the window's top words start at zero
        }
        if (j == W - 4) {
            st |= acc[0] | acc[1];
            pw2 = acc[2];
            pw1 = acc[3];
        } else {
            st |= acc[0] | acc[1] | acc[2] | acc[3];
        }
#pragma unroll
        for (int i = 0; i < W; ++i) acc[i] = acc[i + 4];
#pragma unroll
        for (int i = W; i < W + 4; ++i) acc[i] = 0u;
    }
#pragma unroll
    for (int i = 0; i < W; ++i) hi[i] = acc[i];
    low_nz = st != 0u;
}

// r = RN_p(a * b)
template <int W>
MP_DEV void mul_impl_reg(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    const uint32_t s = a.s ^ b.s;
    if (a.e == EXP_ZERO || b.e == EXP_ZERO) {
        set_zero<W>(r, s);
        return;
    }
    int64_t e = a.e + b.e;
    if constexpr (W <= 32) {
        uint32_t P[2 * W];
        if (rs.r == 0) {
            // p = 32W: round from the truncated product when its error bound
            // cannot change the decision.  With w = word W-1 of T and the round
            // bit at bit rpos of that word (31, or 30 when the product needs the
            // one-bit normalisation), the exact word lies in [w, w + W - 1]
            // (no carry into word W when w + W - 1 < 2^32).  If that interval
            // stays inside one block of 2^rpos, the round bit is known; when it
            // is 1 the bits under it are certainly nonzero unless w sits exactly
            // on the block start.  Otherwise the full product decides.
            mul_trunc<W>(P, a.m, b.m);
            const uint32_t w = P[W - 1];
            const uint32_t top = P[2 * W - 1] >> 31;
            const int rpos = top ? 31 : 30;
            const uint32_t wend = w + (uint32_t)(W - 1);
            const uint32_t rb = (w >> rpos) & 1u;
            const bool safe = (wend >= w) && ((w >> rpos) == (wend >> rpos)) &&
                              !(rb && (w & ((1u << rpos) - 1u)) == 0u);
            if (safe) {
                if (!top) {
#pragma unroll
                    for (int i = 2 * W - 1; i > W; --i) P[i] = __funnelshift_l(P[i - 1], P[i], 1);
                    P[W] = __funnelshift_l(w, P[W], 1);
                    e -= 1;
                }
                P[W] = add_cc(P[W], rb);
#pragma unroll
                for (int i = W + 1; i < 2 * W; ++i) P[i] = addc_cc(P[i], 0u);
                const uint32_t c = addc(0u, 0u);
#pragma unroll
                for (int i = 0; i < W; ++i) r.m[i] = P[W + i];
                if (c) {
                    r.m[W - 1] = 0x80000000u;
                    e += 1;
                }
                r.e = e;
                r.s = s;
                return;
            }
        }
        mul_full<W>(P, a.m, b.m);
        uint32_t low = 0u;
#pragma unroll
        for (int i = 0; i < W - 2; ++i) low |= P[i];
        uint32_t below = P[W - 1], below2 = P[W - 2];
        if (!(P[2 * W - 1] >> 31)) {          // product in [1/4, 1/2): shift left one
#pragma unroll
            for (int i = 2 * W - 1; i > W; --i) P[i] = __funnelshift_l(P[i - 1], P[i], 1);
            P[W] = __funnelshift_l(below, P[W], 1);
            below = __funnelshift_l(below2, below, 1);
            below2 <<= 1;
            e -= 1;
        }
#pragma unroll
        for (int i = 0; i < W; ++i) r.m[i] = P[W + i];
        round_mant<W>(r.m, e, below, (low | below2) != 0u, rs);
    } else {
        uint32_t pw1, pw2;
        bool low_nz;
        mul_top<W>(r.m, pw1, pw2, low_nz, a.m, b.m);
        if (!(r.m[W - 1] >> 31)) {
#pragma unroll
            for (int i = W - 1; i > 0; --i) r.m[i] = (r.m[i] << 1) | (r.m[i - 1] >> 31);
            r.m[0] = (r.m[0] << 1) | (pw1 >> 31);
            pw1 = (pw1 << 1) | (pw2 >> 31);
            pw2 <<= 1;
            e -= 1;
        }
        round_mant<W>(r.m, e, pw1, low_nz || pw2 != 0u, rs);
    }
    r.e = e;
    r.s = s;
}

template <int W>
MP_DEV void mul_impl(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    if constexpr (is_big<W>()) big_mul<W>(r, a, b, rs);
    else mul_impl_reg<W>(r, a, b, rs);
}

// --------------------------------------------------------------- add / sub
// largest value of v among the converged lanes (a warp-uniform bound)
MP_DEV int warp_max(int v)
{
    return (int)__reduce_max_sync(__activemask(), (unsigned)v);
}

// x (N words) >>= sh bits, 0 <= sh <= 32N; returns the OR of the bits
// shifted out.  A select network over the word shift; stages no lane of the
// warp needs are skipped (warp-uniform branch).
// one stage of the word-shift select network per bit J of the word count;
// the stages are expanded at compile time so every index is a constant
template <int N, int J>
MP_DEV void shr_words_stage(uint32_t (&x)[N], int q, int qmax, uint32_t &st)
{
    if constexpr ((1 << J) <= N) {
        constexpr int d = 1 << J;
        if (qmax >= d) {
            const bool on = (q >> J) & 1;
#pragma unroll
            for (int i = 0; i < d && i < N; ++i) st |= on ? x[i] : 0u;
#pragma unroll
            for (int i = 0; i < N; ++i) x[i] = on ? ((i + d < N) ? x[i + d] : 0u) : x[i];
        }
        shr_words_stage<N, J + 1>(x, q, qmax, st);
    }
}

template <int N>
MP_DEV uint32_t shr_sticky(uint32_t (&x)[N], int sh)
{
    const int q = sh >> 5, b = sh & 31;
    const int qmax = warp_max(q);
    uint32_t st = 0u;
    shr_words_stage<N, 0>(x, q, qmax, st);
    st |= x[0] & ((1u << b) - 1u);
#pragma unroll
    for (int i = 0; i < N - 1; ++i) x[i] = __funnelshift_r(x[i], x[i + 1], b);
    x[N - 1] >>= b;
    return st;
}

template <int N, int J>
MP_DEV void shl_words_stage(uint32_t (&x)[N], int q, int qmax)
{
    if constexpr ((1 << J) < N) {
        constexpr int d = 1 << J;
        if (qmax >= d) {
            const bool on = (q >> J) & 1;
#pragma unroll
            for (int i = N - 1; i >= 0; --i) x[i] = on ? ((i - d >= 0) ? x[i - d] : 0u) : x[i];
        }
        shl_words_stage<N, J + 1>(x, q, qmax);
    }
}

// x (N words) <<= sh bits, 0 <= sh < 32N
template <int N>
MP_DEV void shl(uint32_t (&x)[N], int sh)
{
    const int q = sh >> 5, b = sh & 31;
    const int qmax = warp_max(q);
    shl_words_stage<N, 0>(x, q, qmax);
#pragma unroll
    for (int i = N - 1; i > 0; --i) x[i] = __funnelshift_l(x[i - 1], x[i], b);
    x[0] <<= b;
}

// leading zero bits of an N-word number (32N when zero)
template <int N>
MP_DEV int clz_words(const uint32_t (&x)[N])
{
    if (__all_sync(__activemask(), x[N - 1] != 0u)) return __clz(x[N - 1]);
    int lz = 0;
    bool found = false;
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        if (!found) {
            if (x[i]) { lz += __clz(x[i]); found = true; }
            else lz += 32;
        }
    }
    return lz;
}

// r = RN_p(x + (-1)^neg_y * y).  r may alias x or y.
//
// X is the operand of larger magnitude (exponent, then mantissa), so the
// effective subtraction never goes negative.  Y is aligned to X with a guard
// word and a sticky bit.  One carry chain serves both cases: the effective
// subtraction adds the complement of Y with carry-in 1 - sticky (the sticky
// borrow stands for the nonzero bits of Y below the guard word).  The result
// is renormalised by one bit to the right (carry out of an addition) or by
// the leading-zero count to the left (cancellation), then rounded once.
template <int W>
MP_DEV void add_impl_reg(Mp<W> &r, const Mp<W> &x, const Mp<W> &y, uint32_t neg_y, const RoundSpec &rs)
{
    const uint32_t ys = y.s ^ neg_y;
    const bool xz = x.e == EXP_ZERO, yz = y.e == EXP_ZERO;
    if (xz | yz) {
        if (xz & yz) { set_zero<W>(r, x.s & ys); return; }
        if (xz) {
#pragma unroll
            for (int i = 0; i < W; ++i) r.m[i] = y.m[i];
            r.e = y.e;
            r.s = ys;
        } else if (&r != &x) {
#pragma unroll
            for (int i = 0; i < W; ++i) r.m[i] = x.m[i];
            r.e = x.e;
            r.s = x.s;
        }
        return;
    }
    // |y| > |x| ?  exponents first, mantissas on a tie (borrow of x.m - y.m);
    // the mantissa comparison runs only when some lane of the warp has a tie
    bool sw = y.e > x.e;
    if (__any_sync(__activemask(), y.e == x.e)) {
        uint32_t t = sub_cc(x.m[0], y.m[0]);
#pragma unroll
        for (int i = 1; i < W; ++i) t = subc_cc(x.m[i], y.m[i]);
        const uint32_t mlt = subc(0u, 0u);       // all ones if x.m < y.m
        (void)t;
        sw = sw || (y.e == x.e && mlt != 0u);
    }
    uint32_t X[W + 1], Y[W + 1];
    X[0] = 0u;
    Y[0] = 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        X[i + 1] = sw ? y.m[i] : x.m[i];
        Y[i + 1] = sw ? x.m[i] : y.m[i];
    }
    int64_t e = sw ? y.e : x.e;
    const int64_t d64 = sw ? (y.e - x.e) : (x.e - y.e);
    const uint32_t sx = sw ? ys : x.s;
    const uint32_t eff_sub = (x.s ^ ys) & 1u;
    const int d = d64 > 32 * (W + 1) ? 32 * (W + 1) : (int)d64;
    const uint32_t st = shr_sticky<W + 1>(Y, d);
    // S = X + (Y ^ mask) + cin; the first add only loads cin into the carry flag
    const uint32_t mask = 0u - eff_sub;
    const uint32_t cin = eff_sub & (st == 0u ? 1u : 0u);
    uint32_t (&S)[W + 1] = X;                    // the sum replaces X
    (void)add_cc(cin, 0xffffffffu);
#pragma unroll
    for (int i = 0; i <= W; ++i) S[i] = addc_cc(X[i], Y[i] ^ mask);
    const uint32_t carry = addc(0u, 0u);
    // effective addition with a carry out: shift right by one
    const uint32_t rsh = (eff_sub ^ 1u) & carry & 1u;
    bool sticky = st != 0u;
    sticky |= (rsh & S[0] & 1u) != 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) S[i] = __funnelshift_r(S[i], S[i + 1], rsh);
    S[W] = __funnelshift_r(S[W], rsh, rsh);      // the carry bit enters at the top
    e += rsh;
    // cancellation shifts left (an effective addition has lz = 0 here)
    const int lz = clz_words<W + 1>(S);
    if (lz == 32 * (W + 1)) {                     // exact cancellation: +0
        set_zero<W>(r, 0u);
        return;
    }
    shl<W + 1>(S, lz);
    e -= lz;
#pragma unroll
    for (int i = 0; i < W; ++i) r.m[i] = S[i + 1];
    round_mant<W>(r.m, e, S[0], sticky, rs);
    r.e = e;
    r.s = sx;
}

template <int W>
MP_DEV void add_impl(Mp<W> &r, const Mp<W> &x, const Mp<W> &y, uint32_t neg_y, const RoundSpec &rs)
{
    if constexpr (is_big<W>()) big_add<W>(r, x, y, neg_y, rs);
    else add_impl_reg<W>(r, x, y, neg_y, rs);
}

// |a| vs |b| (-1, 0, 1); zero is the smallest magnitude
template <int W>
MP_DEV int cmpabs_reg(const Mp<W> &a, const Mp<W> &b)
{
    const bool az = a.e == EXP_ZERO, bz = b.e == EXP_ZERO;
    if (az | bz) return (az && bz) ? 0 : (az ? -1 : 1);
    if (a.e != b.e) return a.e < b.e ? -1 : 1;
    int c = 0;
#pragma unroll
    for (int i = W - 1; i >= 0; --i)
        if (c == 0 && a.m[i] != b.m[i]) c = a.m[i] < b.m[i] ? -1 : 1;
    return c;
}

template <int W>
MP_DEV int cmpabs(const Mp<W> &a, const Mp<W> &b)
{
    if constexpr (is_big<W>()) return big_cmpabs<W>(a, b);
    else return cmpabs_reg<W>(a, b);
}

// --------------------------------------------------------------- division
// r = RN_p(a / b), b != 0: exact long division of the mantissas (the
// quotient of two fractions in [1/2, 1) lies in (1/2, 2)), then one rounding
// with the remainder as sticky.
template <int W>
MP_DEV void div_impl_reg(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    const uint32_t s = a.s ^ b.s;
    if (a.e == EXP_ZERO || b.e == EXP_ZERO) { set_zero<W>(r, s); return; }   // callers reject b = 0
    // Schoolbook long division in radix 2^32 (Knuth, TAOCP vol. 2, Sec. 4.3.1,
    // Algorithm D) of the integers A = a.m and D = b.m, both with the top bit
    // set (so D needs no normalisation): Q = floor(A 2^(32(W+1)) / D) with
    // remainder R.  Since A / D lies in (1/2, 2), Q has 32(W+1) or 32(W+1) + 1
    // significant bits -- at least p + 32 -- and R != 0 is the sticky bit.
    uint32_t R[W + 1], Q[W + 2];
    // leading digit (weight 2^(32(W+1))): 1 iff A >= D; R = A - digit * D
    uint32_t T[W];
    T[0] = sub_cc(a.m[0], b.m[0]);
#pragma unroll
    for (int i = 1; i < W; ++i) T[i] = subc_cc(a.m[i], b.m[i]);
    const uint32_t q0 = subc(0u, 0u) ? 0u : 1u;
#pragma unroll
    for (int i = 0; i < W; ++i) R[i] = q0 ? T[i] : a.m[i];
    R[W] = 0u;
#pragma unroll
    for (int i = 0; i < W + 2; ++i) Q[i] = 0u;
    Q[0] = q0;
    const uint32_t d1 = b.m[W - 1], d2 = b.m[W - 2];
    // reciprocal of the top divisor word for the two-by-one digit division
    // (Moller and Granlund, "Improved division by invariant integers", 2011,
    // Alg. 4): v = floor((2^64 - 1) / d1) - 2^32
    const uint32_t v = (uint32_t)(0xffffffffffffffffull / d1 - 0x100000000ull);
#pragma unroll 1
    for (int t = 0; t <= W; ++t) {
        // R < D: bring down a zero digit, R <- R 2^32 (W + 1 words)
#pragma unroll
        for (int i = W; i > 0; --i) R[i] = R[i - 1];
        R[0] = 0u;
        // estimate the digit from the top two words of R and the top word of
        // D, then refine with the second word of D (at most two decrements)
        const uint32_t u1 = R[W], u0 = R[W - 1];
        uint64_t qh, rh;
        if (u1 >= d1) {                         // u1 == d1: the digit estimate saturates
            qh = 0xffffffffull;
            rh = (((uint64_t)u1 << 32) | u0) - qh * d1;
        } else {
            const uint64_t t = (uint64_t)v * u1 + (((uint64_t)u1 << 32) | u0);   // mod 2^64
            uint32_t q1 = (uint32_t)(t >> 32) + 1u;
            const uint32_t q0 = (uint32_t)t;
            uint32_t rr = u0 - q1 * d1;
            if (rr > q0) { q1 -= 1u; rr += d1; }
            if (rr >= d1) { q1 += 1u; rr -= d1; }
            qh = q1;
            rh = rr;
        }
#pragma unroll 1
        for (int c = 0; c < 2 && rh <= 0xffffffffull && qh * d2 > ((rh << 32) | R[W - 2]); ++c) {
            --qh;
            rh += d1;
        }
        const uint32_t q = (uint32_t)qh;
        // R -= q D, one pass: product words and the borrow chain together
        uint64_t cy = 0;
        uint32_t br = 0u;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint64_t pr = (uint64_t)b.m[i] * q + cy;
            cy = pr >> 32;
            const uint64_t df = (uint64_t)R[i] - (uint32_t)pr - br;
            R[i] = (uint32_t)df;
            br = (uint32_t)(df >> 63);
        }
        const uint64_t dt = (uint64_t)R[W] - cy - br;
        R[W] = (uint32_t)dt;
        const uint32_t neg = (uint32_t)(dt >> 63);
        uint32_t qd = q;
        if (neg) {                              // estimate one too large: add D back
            R[0] = add_cc(R[0], b.m[0]);
#pragma unroll
            for (int i = 1; i < W; ++i) R[i] = addc_cc(R[i], b.m[i]);
            R[W] = addc(R[W], 0u);
            qd -= 1u;
        }
#pragma unroll
        for (int i = W + 1; i > 0; --i) Q[i] = Q[i - 1];
        Q[0] = qd;
    }
    bool rem = false;
#pragma unroll
    for (int i = 0; i < W; ++i) rem |= R[i] != 0u;
    // value = Q 2^(-32(W+1)) 2^(ea - eb); the leading one is bit 0 of Q[W+1]
    // (A >= D) or bit 31 of Q[W]
    const int lz = q0 ? 31 : 32;
    shl<W + 2>(Q, lz);
    int64_t e = a.e - b.e + 32 - lz;
#pragma unroll
    for (int i = 0; i < W; ++i) r.m[i] = Q[i + 2];
    round_mant<W>(r.m, e, Q[1], rem || Q[0] != 0u, rs);
    r.e = e;
    r.s = s;
}

template <int W>
MP_DEV void div_impl(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    if constexpr (is_big<W>()) big_div<W>(r, a, b, rs);
    else div_impl_reg<W>(r, a, b, rs);
}

// ------------------------------------------------------------ entry points
// For W >= 32 the operations are out-of-line calls: one copy per kernel
// instead of one per call site keeps the 1024/2048-bit code small.
template <int W>
__device__ __noinline__ void add_call(Mp<W> &r, const Mp<W> &x, const Mp<W> &y, uint32_t neg_y,
                                      const RoundSpec &rs)
{
    add_impl<W>(r, x, y, neg_y, rs);
}
template <int W>
__device__ __noinline__ void mul_call(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    mul_impl<W>(r, a, b, rs);
}
template <int W>
__device__ __noinline__ void div_call(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    div_impl<W>(r, a, b, rs);
}

// INL: inline the operation even for W = 32 (used by the GEMM inner loops,
// where the call overhead through local memory would dominate)
template <int W, bool INL = false>
MP_DEV void add(Mp<W> &r, const Mp<W> &x, const Mp<W> &y, uint32_t neg_y, const RoundSpec &rs)
{
    if constexpr (W >= 64 || (W >= 32 && !INL)) add_call<W>(r, x, y, neg_y, rs);
    else add_impl<W>(r, x, y, neg_y, rs);
}
template <int W, bool INL = false>
MP_DEV void mul(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    if constexpr (W >= 64 || (W >= 32 && !INL)) mul_call<W>(r, a, b, rs);
    else mul_impl<W>(r, a, b, rs);
}
template <int W>
MP_DEV void div(Mp<W> &r, const Mp<W> &a, const Mp<W> &b, const RoundSpec &rs)
{
    div_call<W>(r, a, b, rs);
}

}  // namespace mpg
