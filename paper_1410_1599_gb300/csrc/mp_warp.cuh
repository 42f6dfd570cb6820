// mp_warp.cuh -- one MP division computed by the 32 lanes of a warp together,
// for latency-bound call sites (the LU pivot-column scaling and the
// back substitution, where one division sits on the critical path).
//
// A mantissa of W <= 32 words is spread one word per lane (lane i holds word
// i, least significant first; lanes >= W hold 0).  Carries and borrows cross
// the lanes by carry-lookahead on ballots: with g = lanes that generate and
// p = lanes that propagate, the carries into the lanes are the carries of
// the binary sum (g | p) + g, i.e. ((g|p) + g) ^ (g|p) ^ g.
#pragma once
#include "mp_kernels.cuh"

namespace mpg {

constexpr unsigned FULL_MASK = 0xffffffffu;

// a - b across the lanes; *bout = borrow out of word W-1
template <int W>
MP_DEV uint32_t wsub(uint32_t a, uint32_t b, uint32_t &bout)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t g = __ballot_sync(FULL_MASK, a < b);
    const uint64_t p = __ballot_sync(FULL_MASK, a == b);
    const uint64_t x = g | p;
    const uint64_t c = (x + g) ^ x ^ g;          // bit i: borrow into word i
    bout = (uint32_t)(c >> W) & 1u;
    return a - b - ((uint32_t)(c >> lane) & 1u);
}

// a + b across the lanes; *cout = carry out of word W-1
template <int W>
MP_DEV uint32_t wadd(uint32_t a, uint32_t b, uint32_t &cout)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t s = a + b;
    const uint64_t g = __ballot_sync(FULL_MASK, s < a);
    const uint64_t p = __ballot_sync(FULL_MASK, s == 0xffffffffu);
    const uint64_t x = g | p;
    const uint64_t c = (x + g) ^ x ^ g;
    cout = (uint32_t)(c >> W) & 1u;
    return s + ((uint32_t)(c >> lane) & 1u);
}

// r = RN_p(a / b) for b != 0, by the whole warp.  In: lane i holds word i of
// a's and b's mantissas (am, bm); exponents and signs are the same in every
// lane.  Out: lane i holds word i of the result's mantissa; *re, *rsg are
// uniform.  The steps are those of the scalar div_impl (long division in
// radix 2^32 with a two-by-one digit estimate, then one rounding), so the
// result is the same correctly rounded quotient.
template <int W>
MP_DEV uint32_t warp_div(uint32_t am, int64_t ae, uint32_t as, uint32_t bm, int64_t be, uint32_t bs,
                         int64_t &re, uint32_t &rsg, const RoundSpec &rs)
{
    static_assert(W >= 4 && W <= 32, "one word per lane");
    const int lane = (int)(threadIdx.x & 31u);
    rsg = as ^ bs;
    if (ae == EXP_ZERO || be == EXP_ZERO) {
        re = EXP_ZERO;
        return 0u;
    }
    // leading digit: A >= D
    const uint32_t ne = __ballot_sync(FULL_MASK, am != bm);
    uint32_t q0 = 1u;
    if (ne) q0 = __shfl_sync(FULL_MASK, am > bm ? 1u : 0u, 31 - __clz(ne));
    uint32_t bo;
    const uint32_t t0 = wsub<W>(am, bm, bo);
    uint32_t R = (lane < W) ? (q0 ? t0 : am) : 0u;
    const uint32_t d1 = __shfl_sync(FULL_MASK, bm, W - 1), d2 = __shfl_sync(FULL_MASK, bm, W - 2);
    const uint32_t v = (uint32_t)(0xffffffffffffffffull / d1 - 0x100000000ull);
    uint32_t qd = 0u, qW = 0u;                   // digit `lane` (lanes < W) and digit W
#pragma unroll 1
    for (int t = 0; t <= W; ++t) {
        // R <- R 2^32: the top word leaves the lanes
        const uint32_t u1 = __shfl_sync(FULL_MASK, R, W - 1);
        const uint32_t u0 = __shfl_sync(FULL_MASK, R, W - 2);
        const uint32_t u2 = __shfl_sync(FULL_MASK, R, W - 3);
        uint32_t Rs = __shfl_up_sync(FULL_MASK, R, 1);
        if (lane == 0 || lane >= W) Rs = 0u;
        // digit estimate (Moller-Granlund two-by-one step), refined with d2
        uint64_t qh, rh;
        if (u1 >= d1) {
            qh = 0xffffffffull;
            rh = (((uint64_t)u1 << 32) | u0) - qh * d1;
        } else {
            const uint64_t tt = (uint64_t)v * u1 + (((uint64_t)u1 << 32) | u0);
            uint32_t q1 = (uint32_t)(tt >> 32) + 1u;
            const uint32_t qq0 = (uint32_t)tt;
            uint32_t rr = u0 - q1 * d1;
            if (rr > qq0) { q1 -= 1u; rr += d1; }
            if (rr >= d1) { q1 += 1u; rr -= d1; }
            qh = q1;
            rh = rr;
        }
#pragma unroll 1
        for (int c = 0; c < 2 && rh <= 0xffffffffull && qh * d2 > ((rh << 32) | u2); ++c) {
            --qh;
            rh += d1;
        }
        uint32_t q = (uint32_t)qh;
        // R' - q D over W + 1 words: low words in the lanes, top word u1
        const uint32_t lo = bm * q, hi = __umulhi(bm, q);
        uint32_t hs = __shfl_up_sync(FULL_MASK, hi, 1);
        if (lane == 0 || lane >= W) hs = 0u;
        const uint32_t htop = __shfl_sync(FULL_MASK, hi, W - 1);
        uint32_t b1, b2;
        const uint32_t t1 = wsub<W>(Rs, lo, b1);
        uint32_t R2 = wsub<W>(t1, hs, b2);
        const int64_t top = (int64_t)u1 - (int64_t)htop - (int64_t)b1 - (int64_t)b2;
        if (top < 0) {                           // one too many: add D back
            uint32_t c;
            R2 = wadd<W>(R2, bm, c);
            q -= 1u;
        }
        R = (lane < W) ? R2 : 0u;
        if (t == 0) qW = q;
        else if (lane == W - t) qd = q;
    }
    const bool rem = __ballot_sync(FULL_MASK, R != 0u) != 0u;
    // mantissa: the 32W quotient bits under the leading one (bit 0 of digit
    // W+1 = q0, or bit 31 of digit W)
    uint32_t Q1 = __shfl_down_sync(FULL_MASK, qd, 1), Q2 = __shfl_down_sync(FULL_MASK, qd, 2);
    if (lane + 1 == W) Q1 = qW;
    else if (lane + 1 > W) Q1 = 0u;
    if (lane + 2 == W) Q2 = qW;
    else if (lane + 2 == W + 1) Q2 = q0;
    else if (lane + 2 > W + 1) Q2 = 0u;
    uint32_t M = q0 ? __funnelshift_r(Q1, Q2, 1) : Q1;
    if (lane >= W) M = 0u;
    const uint32_t qlow = __shfl_sync(FULL_MASK, qd, 0), q1w = __shfl_sync(FULL_MASK, Q1, 0);
    const uint32_t below = q0 ? __funnelshift_r(qlow, q1w, 1) : qlow;
    const bool sticky = rem || (q0 && (qlow & 1u));
    int64_t e = ae - be + (q0 ? 1 : 0);
    // round to p bits, nearest-even
    const int r = rs.r;
    uint32_t up;
    if (r == 0) {
        const uint32_t lsb = __shfl_sync(FULL_MASK, M, 0) & 1u;
        const uint32_t st = ((below << 1) != 0u || sticky) ? 1u : 0u;
        up = (below >> 31) & (st | lsb);
    } else {
        const int rw = r >> 5, rb = r & 31, r1 = r - 1;
        const uint32_t lsb = (__shfl_sync(FULL_MASK, M, rw) >> rb) & 1u;
        const uint32_t rbit = (__shfl_sync(FULL_MASK, M, r1 >> 5) >> (r1 & 31)) & 1u;
        // bits of M under the round bit
        uint32_t mask = 0u;
        if (32 * lane + 32 <= r1) mask = 0xffffffffu;
        else if (32 * lane < r1) mask = (1u << (r1 - 32 * lane)) - 1u;
        const bool low = __ballot_sync(FULL_MASK, (M & mask) != 0u) != 0u;
        const uint32_t st = (low || below != 0u || sticky) ? 1u : 0u;
        up = rbit & (st | lsb);
    }
    if (up) {                                    // uniform branch
        uint32_t c;
        M = wadd<W>(M, lane == (r >> 5) ? (1u << (r & 31)) : 0u, c);
        if (c) {
            M = (lane == W - 1) ? 0x80000000u : 0u;
            e += 1;
        }
    }
    // clear the bits under the kept LSB (and the lanes beyond W)
    if (lane >= W || 32 * lane + 32 <= r) M = 0u;
    else if (32 * lane < r) M &= ~((1u << (r - 32 * lane)) - 1u);
    re = e;
    return M;
}

// Lane i < W reads word i of the mantissa of M(b, r, c); exponent and sign
// go to every lane.  Limb k holds words W-1-2k (high half) and W-2-2k.
template <int W>
MP_DEV uint32_t wld(const BMat &M, int64_t b, int64_t r, int64_t c, int L, int64_t &e, uint32_t &s)
{
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t lo = lim_off(M, b, r, c), eo = es_off(M, b, r, c);
    uint32_t w = 0u;
    if (lane < W) {
        const int d = W - 1 - lane, k = d >> 1;
        if (k < L) {
            const uint64_t v = M.limb[lo + (int64_t)k * M.plane];
            w = (d & 1) ? (uint32_t)v : (uint32_t)(v >> 32);
        }
    }
    e = M.exp[eo];
    s = (uint32_t)(M.sign[eo] & 1);
    return w;
}

// Store of a number held one word per lane; returns the exponent range check.
template <int W>
MP_DEV bool wst(uint32_t w, int64_t e, uint32_t s, const BMat &M, int64_t b, int64_t r, int64_t c, int L)
{
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t lo = lim_off(M, b, r, c), eo = es_off(M, b, r, c);
    const uint32_t below = __shfl_up_sync(FULL_MASK, w, 1);   // word lane-1: the low half
    if (lane < W) {
        const int d = W - 1 - lane, k = d >> 1;
        if (!(d & 1) && k < L) M.limb[lo + (int64_t)k * M.plane] = ((uint64_t)w << 32) | below;
    }
    if (lane == 0) {
        M.exp[eo] = e;
        M.sign[eo] = (int8_t)s;
    }
    return e != EXP_ZERO && (e > EXP_LIMIT || e < -EXP_LIMIT);
}

}  // namespace mpg
