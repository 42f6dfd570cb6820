// mp_warp.cuh -- MP division, multiplication and addition computed by the 32
// lanes of a warp together, for latency-bound call sites (the LU
// pivot-column scaling and the triangular solves, where one operation after
// another sits on the critical path).
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

// Round a mantissa held one word per lane (top bit of word W-1 set, lanes
// >= W zero) to p bits, nearest-even: `below` is the word under it and
// `sticky` says whether anything lies lower (both the same in every lane).
// A carry out of the top renormalises and increments e.
template <int W>
MP_DEV uint32_t warp_round(uint32_t M, uint32_t below, bool sticky, int64_t &e, const RoundSpec &rs)
{
    const int lane = (int)(threadIdx.x & 31u);
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
    return M;
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
    M = warp_round<W>(M, below, sticky, e, rs);
    re = e;
    return M;
}

// r = RN_p(a * b) by the whole warp (lane i: word i of each mantissa).
// Lane L forms the column sums of product positions L and L + 32,
// sum_{i+j=k} a_i b_j (a broadcast, b gathered), as 96-bit values; the
// three 32-bit digits of each column are added into their words, and the
// remaining one-bit carries ripple by carry-lookahead on ballots.  The top
// W words (one bit lower when the product is below 1/2) are then rounded
// once with the next word and an OR of the rest.
template <int W>
MP_DEV uint32_t warp_mul(uint32_t am, int64_t ae, uint32_t as, uint32_t bm, int64_t be, uint32_t bs,
                         int64_t &re, uint32_t &rsg, const RoundSpec &rs)
{
    static_assert(W >= 4 && W <= 32, "one word per lane");
    const int lane = (int)(threadIdx.x & 31u);
    rsg = as ^ bs;
    if (ae == EXP_ZERO || be == EXP_ZERO) {
        re = EXP_ZERO;
        return 0u;
    }
    constexpr bool TWO = 2 * W > 32;               // positions beyond 31 exist
    uint64_t s1 = 0, s2 = 0;
    uint32_t h1 = 0u, h2 = 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint32_t ai = __shfl_sync(FULL_MASK, am, i);
        const int j1 = lane - i;
        const uint32_t b1r = __shfl_sync(FULL_MASK, bm, j1 & 31);
        const uint64_t p1 = (uint64_t)ai * ((j1 >= 0 && j1 < W) ? b1r : 0u);
        s1 += p1;
        h1 += (s1 < p1) ? 1u : 0u;
        if constexpr (TWO) {
            const int j2 = lane + 32 - i;
            const uint32_t b2r = __shfl_sync(FULL_MASK, bm, j2 & 31);
            const uint64_t p2 = (uint64_t)ai * ((j2 < W) ? b2r : 0u);
            s2 += p2;
            h2 += (s2 < p2) ? 1u : 0u;
        }
    }
    // word k = c0[k] + c1[k-1] + c2[k-2] (< 3 * 2^32), digits of the columns
    const uint32_t c01 = (uint32_t)s1, c11 = (uint32_t)(s1 >> 32), c21 = h1;
    const uint32_t c02 = (uint32_t)s2, c12 = (uint32_t)(s2 >> 32), c22 = h2;
    const uint32_t up11 = __shfl_up_sync(FULL_MASK, c11, 1), up21 = __shfl_up_sync(FULL_MASK, c21, 2);
    const uint64_t t1 = (uint64_t)c01 + (lane >= 1 ? up11 : 0u) + (lane >= 2 ? up21 : 0u);
    uint64_t t2 = 0;
    if constexpr (TWO) {
        const uint32_t up12 = __shfl_up_sync(FULL_MASK, c12, 1), up22 = __shfl_up_sync(FULL_MASK, c22, 2);
        const uint32_t c11_31 = __shfl_sync(FULL_MASK, c11, 31);
        const uint32_t c21_30 = __shfl_sync(FULL_MASK, c21, 30), c21_31 = __shfl_sync(FULL_MASK, c21, 31);
        t2 = (uint64_t)c02 + (lane >= 1 ? up12 : c11_31) +
             (lane >= 2 ? up22 : (lane == 1 ? c21_31 : c21_30));
    }
    // fold the 0..2 carries one word up, then the one-bit carries
    const uint32_t hi1 = (uint32_t)(t1 >> 32), hi2 = (uint32_t)(t2 >> 32);
    const uint32_t uh1 = __shfl_up_sync(FULL_MASK, hi1, 1);
    const uint64_t u1 = (uint64_t)(uint32_t)t1 + (lane >= 1 ? uh1 : 0u);
    uint64_t u2 = 0;
    if constexpr (TWO) {
        const uint32_t uh2 = __shfl_up_sync(FULL_MASK, hi2, 1);
        const uint32_t hi1_31 = __shfl_sync(FULL_MASK, hi1, 31);
        u2 = (uint64_t)(uint32_t)t2 + (lane >= 1 ? uh2 : hi1_31);
    }
    const uint32_t l1 = (uint32_t)u1, l2 = (uint32_t)u2;
    const uint64_t G = (uint64_t)__ballot_sync(FULL_MASK, (u1 >> 32) != 0u) |
                       ((uint64_t)__ballot_sync(FULL_MASK, (u2 >> 32) != 0u) << 32);
    const uint64_t P = (uint64_t)__ballot_sync(FULL_MASK, l1 == 0xffffffffu) |
                       ((uint64_t)__ballot_sync(FULL_MASK, TWO && l2 == 0xffffffffu) << 32);
    const uint64_t X = G | P;
    const uint64_t C = (X + G) ^ X ^ G;            // bit k: carry into position k
    const uint32_t w1 = l1 + (uint32_t)((C >> lane) & 1u);
    const uint32_t w2 = TWO ? l2 + (uint32_t)((C >> (lane + 32)) & 1u) : 0u;
    // word at product position pos (per lane), 0 outside [0, 2W)
    auto word = [&](int pos) -> uint32_t {
        const uint32_t v1 = __shfl_sync(FULL_MASK, w1, pos & 31);
        const uint32_t v2 = TWO ? __shfl_sync(FULL_MASK, w2, pos & 31) : 0u;
        if (pos < 0 || pos >= 2 * W) return 0u;
        return pos < 32 ? v1 : v2;
    };
    const uint32_t top = word(2 * W - 1);
    const int sh = (top >> 31) ? 0 : 1;            // product in [1/4, 1/2): one bit left
    const uint32_t x = word(W + lane), xl = word(W + lane - 1);
    uint32_t M = sh ? ((x << 1) | (xl >> 31)) : x;
    if (lane >= W) M = 0u;
    const uint32_t bw = word(W - 1), bw2 = word(W - 2);
    const uint32_t below = sh ? ((bw << 1) | (bw2 >> 31)) : bw;
    const int lim = sh ? W - 2 : W - 1;            // whole words under `below`
    bool sticky = __ballot_sync(FULL_MASK, (lane < lim && w1 != 0u) || (TWO && lane + 32 < lim && w2 != 0u)) != 0u;
    if (sh) sticky = sticky || (bw2 & 0x7fffffffu) != 0u;
    int64_t e = ae + be - sh;
    M = warp_round<W>(M, below, sticky, e, rs);
    re = e;
    return M;
}

// r = RN_p(x + (-1)^neg y) by the whole warp, the steps of the scalar
// addition: the larger magnitude X, the other operand aligned to it with a
// guard word and a sticky bit, one carry-lookahead addition (or subtraction
// with the sticky borrow), renormalisation, one rounding.
template <int W>
MP_DEV uint32_t warp_add(uint32_t xm, int64_t xe, uint32_t xs, uint32_t ym, int64_t ye, uint32_t ys,
                         uint32_t neg, int64_t &re, uint32_t &rsg, const RoundSpec &rs)
{
    static_assert(W >= 4 && W <= 32, "one word per lane");
    const int lane = (int)(threadIdx.x & 31u);
    ys ^= neg;
    const bool xz = xe == EXP_ZERO, yz = ye == EXP_ZERO;
    if (xz && yz) {
        re = EXP_ZERO;
        rsg = xs & ys;
        return 0u;
    }
    if (xz) {
        re = ye;
        rsg = ys;
        return ym;
    }
    if (yz) {
        re = xe;
        rsg = xs;
        return xm;
    }
    const uint32_t ne = __ballot_sync(FULL_MASK, xm != ym);
    bool mlt = false;
    if (ne) mlt = __shfl_sync(FULL_MASK, xm < ym ? 1u : 0u, 31 - __clz(ne)) != 0u;
    const bool sw = (ye > xe) || (ye == xe && mlt);
    const uint32_t X = sw ? ym : xm, Y = sw ? xm : ym;
    int64_t e = sw ? ye : xe;
    const int64_t d64 = sw ? (ye - xe) : (xe - ye);
    const uint32_t sx = sw ? ys : xs;
    const uint32_t eff_sub = (xs ^ ys) & 1u;
    // Y aligned: word `lane`, the guard word under it and the sticky rest
    uint32_t Ys, guard;
    bool sticky;
    auto yw = [&](int k) -> uint32_t {            // word k of Y, 0 outside [0, W)
        const uint32_t v = __shfl_sync(FULL_MASK, Y, k & 31);
        return (k >= 0 && k < W) ? v : 0u;
    };
    if (d64 >= 32 * (W + 1)) {
        Ys = 0u;
        guard = 0u;
        sticky = __ballot_sync(FULL_MASK, Y != 0u) != 0u;
    } else {
        const int d = (int)d64, q = d >> 5, b = d & 31;
        Ys = __funnelshift_r(yw(lane + q), yw(lane + q + 1), b);
        if (lane >= W) Ys = 0u;
        guard = __funnelshift_r(yw(q - 1), yw(q), b);
        sticky = __ballot_sync(FULL_MASK, lane < W && ((lane < q - 1 && Y != 0u) ||
                                                       (lane == q - 1 && b != 0 && (Y & ((1u << b) - 1u)) != 0u))) != 0u;
    }
    // S = X + (Y ^ mask) + cin over the guard word and W words
    const uint32_t mask = 0u - eff_sub;
    const uint64_t tg = (uint64_t)(guard ^ mask) + (eff_sub & (sticky ? 0u : 1u));
    uint32_t gsum = (uint32_t)tg;
    const uint64_t sm = (lane < W) ? (uint64_t)X + (Ys ^ mask) : 0ull;
    const uint32_t lo = (uint32_t)sm;
    const uint64_t G = __ballot_sync(FULL_MASK, (sm >> 32) != 0u);
    const uint64_t P = __ballot_sync(FULL_MASK, lane < W && lo == 0xffffffffu);
    const uint64_t XG = G | P;
    const uint64_t C = (XG + G + (tg >> 32)) ^ XG ^ G;   // bit i: carry into word i
    uint32_t S = lo + (uint32_t)((C >> lane) & 1u);
    if (lane >= W) S = 0u;
    const uint32_t carry = (uint32_t)((C >> W) & 1u);
    if ((eff_sub ^ 1u) & carry) {                 // an addition carried out: one bit right
        sticky = sticky || (gsum & 1u) != 0u;
        const uint32_t s0 = __shfl_sync(FULL_MASK, S, 0);
        gsum = (gsum >> 1) | (s0 << 31);
        const uint32_t nx = __shfl_down_sync(FULL_MASK, S, 1);
        S = (S >> 1) | ((lane == W - 1 ? 1u : nx) << 31);
        if (lane >= W) S = 0u;
        e += 1;
    }
    // leading zeros of [S_{W-1} .. S_0, guard]; exact cancellation gives +0
    const uint32_t nz = __ballot_sync(FULL_MASK, S != 0u);
    if (nz == 0u && gsum == 0u) {
        re = EXP_ZERO;
        rsg = 0u;
        return 0u;
    }
    int lz;
    if (nz) {
        const int tw = 31 - __clz(nz);
        lz = 32 * (W - 1 - tw) + __clz(__shfl_sync(FULL_MASK, S, tw));
    } else {
        lz = 32 * W + __clz(gsum);
    }
    // shift left by lz over the virtual words V[0] = guard, V[k] = S_{k-1}
    const int q = lz >> 5, b = lz & 31;
    auto vw = [&](int k) -> uint32_t {
        const uint32_t v = __shfl_sync(FULL_MASK, S, (k - 1) & 31);
        if (k == 0) return gsum;
        return (k >= 1 && k <= W) ? v : 0u;
    };
    uint32_t M = __funnelshift_l(vw(lane - q), vw(lane + 1 - q), b);
    if (lane >= W) M = 0u;
    const uint32_t below = (q == 0) ? (gsum << b) : 0u;
    e -= lz;
    M = warp_round<W>(M, below, sticky, e, rs);
    re = e;
    rsg = sx;
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


// R = X op Y elementwise with one warp per element (op 0 add, 1 subtract,
// 2 multiply, 3 divide): the warp routines above, for call sites that want
// the latency of one operation rather than throughput.  Same bits as the
// one-thread operations.
template <int W>
__global__ void __launch_bounds__(128) elementwise_warp_kernel(int op, BMat X, BMat Y, BMat R, int64_t rows,
                                                               int64_t cols, int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t total = rows * cols;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    bool bad = false, dz = false;
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < total; t += nw) {
        const int64_t r = t / cols, c = t % cols;
        int64_t xe, ye, ze;
        uint32_t xs, ys, zs;
        const uint32_t xm = wld<W>(X, 0, r, c, rs.L, xe, xs);
        const uint32_t ym = wld<W>(Y, 0, r, c, rs.L, ye, ys);
        uint32_t zm;
        if (op == 0 || op == 1) {
            zm = warp_add<W>(xm, xe, xs, ym, ye, ys, (uint32_t)op, ze, zs, rs);
        } else if (op == 2) {
            zm = warp_mul<W>(xm, xe, xs, ym, ye, ys, ze, zs, rs);
        } else {
            if (ye == EXP_ZERO) {
                dz = true;
                continue;
            }
            zm = warp_div<W>(xm, xe, xs, ym, ye, ys, ze, zs, rs);
        }
        bad |= wst<W>(zm, ze, zs, R, 0, r, c, rs.L);
    }
    if (lane == 0 && bad) flag(status, ST_RANGE);
    if (lane == 0 && dz) flag(status, ST_DIVZERO);
}

template <int W>
void launch_elementwise_warp(int op, BMat X, BMat Y, BMat R, int64_t rows, int64_t cols, int p,
                             DevStatus *st, cudaStream_t s)
{
    const int64_t total = rows * cols;
    if (total <= 0) return;
    elementwise_warp_kernel<W><<<grid_for(total * 32, 128), 128, 0, s>>>(op, X, Y, R, rows, cols, p, st);
}

#define MPG_INSTANTIATE_WARP(W)                                                                 \
    template void launch_elementwise_warp<W>(int, BMat, BMat, BMat, int64_t, int64_t, int,      \
                                             DevStatus *, cudaStream_t);

}  // namespace mpg
