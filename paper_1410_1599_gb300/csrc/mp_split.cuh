// mp_split.cuh -- the split form of C = RN_p(exact A B) on tensor cores.
//
// 1. Alignment (split_prep_*): each row i of A (column j of B) gets the
//    largest exponent emax of its nonzero entries; every entry becomes the
//    integer x = a * 2^(F - emax), F = p + SB, exact when the entry's
//    exponent is at least emax - SB (SB = 64, the spread budget).  Rows or
//    columns with a wider spread are marked and recomputed by the exact limb
//    kernel.  x (|x| < 2^F) is cut into S = ceil(F/8) + 1 signed base-256
//    digits in [-128, 128] (balanced, so that all digits fit the tensor
//    core's inputs exactly), stored as fp16 planes A_u[i][k], B_v[j][k].
// 2. Slice products (split_slice_kernel): for every weight diagonal
//    s = u + v, D_s(i, j) = sum_{u+v=s} sum_k A_u(i,k) B_v(k,j), exactly.
//    Digit products are integers of at most 2^14 in magnitude; the fp32
//    tensor-core accumulators hold sums of at most CHUNK of them (< 2^24, so
//    every partial sum is an exact fp32 integer) before they are folded into
//    int64 registers.
// 3. Recombination (split_finish_kernel): the exact sum
//    sum_s D_s 256^s * 2^(emaxA(i) + emaxB(j) - 2F) is carried into a
//    two's complement fixed-point integer and rounded once to p bits.
// Truncation: the diagonals s < s0 lie far below the rounding position of a
// typical output and are skipped.  Their sum is below
// l S 2^14 256^s0 <= 2^eb (|digit product| <= 2^14, at most S pairs per
// diagonal, sum_{s<s0} 256^s < 256^s0).  The rounding of the kept sum V is
// then the rounding of the exact sum unless V +- 2^eb reaches a midpoint
// between p-bit neighbours; such outputs (and those too close to zero) are
// recomputed exactly (a Ziv-style test: the result is identical either way).
// No floating-point rounding enters anywhere: every fp16 and fp32 value is
// an exactly represented integer.
#pragma once
#include <cuda_fp16.h>

#include "mp_exact.cuh"

namespace mpg {

constexpr int SPLIT_SB = 64;        // exponent spread budget, bits
constexpr int SPLIT_CHUNK = 512;    // k-terms per exact fp32 accumulation
constexpr int SPLIT_TM = 64, SPLIT_TN = 64, SPLIT_TK = 32;

inline int split_digits(int p) { return (p + SPLIT_SB + 7) / 8 + 1; }
inline int64_t split_lpad(int64_t l) { return (l + SPLIT_TK - 1) / SPLIT_TK * SPLIT_TK; }

// largest of an int64 across the warp
MP_DEV int64_t warp_max64(int64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Digits of one entry x (held as Mp<W>) aligned to emax: the balanced base-256
// digits of x * 2^(F - emax), written to out[u * ustride] for u < S.
template <int W>
MP_DEV void write_digits(const Mp<W> &x, int64_t emax, int p, int S, __half *out, int64_t ustride)
{
    if (x.e == EXP_ZERO) {
        for (int u = 0; u < S; ++u) out[u * ustride] = __float2half(0.f);
        return;
    }
    // bit b of the aligned integer is bit (b - sh) of the 32W-bit mantissa
    const int64_t sh = x.e - emax + SPLIT_SB + p - 32 * W;
    uint32_t mw[W];
#pragma unroll
    for (int t = 0; t < W; ++t) mw[t] = x.m[t];
    int carry = 0;
    for (int u = 0; u < S; ++u) {
        const int64_t lo = 8 * (int64_t)u - sh;        // mantissa bit of digit bit 0
        uint32_t byte = 0;
        if (lo > -8 && lo < 32 * W) {
            const int64_t w0 = lo >> 5;                  // may be -1
            const int s0 = (int)(lo & 31);
            const uint32_t a0 = (w0 >= 0 && w0 < W) ? mw[w0] : 0u;
            const uint32_t a1 = (w0 + 1 >= 0 && w0 + 1 < W) ? mw[w0 + 1] : 0u;
            const uint64_t pair = ((uint64_t)a1 << 32) | a0;
            byte = (uint32_t)(pair >> s0) & 0xffu;
        }
        int t = (int)byte + carry;
        int d;
        if (t >= 128) { d = t - 256; carry = 1; } else { d = t; carry = 0; }
        if (x.s) d = -d;
        out[u * ustride] = __int2half_rn(d);
    }
}

// one warp per row of A: emax, spread flag, digit planes [S][m][lp]
template <int W>
__global__ void split_prep_rows(BMat A, int64_t m, int64_t l, int64_t lp, int p, int S,
                                __half *planes, int64_t *emax_out, uint8_t *wide_out)
{
    const RoundSpec rs = make_spec<W>(p);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nwarps) {
        int64_t emax = INT64_MIN;
        for (int64_t k = lane; k < l; k += 32) {
            const int64_t e = A.exp[i * A.ld + k];
            if (e != EXP_ZERO && e > emax) emax = e;
        }
        emax = warp_max64(emax);
        bool wide = false;
        for (int64_t k = lane; k < l; k += 32) {
            const int64_t e = A.exp[i * A.ld + k];
            if (e != EXP_ZERO && e < emax - SPLIT_SB) wide = true;
        }
        wide = __any_sync(0xffffffffu, wide);
        if (lane == 0) {
            emax_out[i] = emax;
            wide_out[i] = wide ? 1 : 0;
        }
        const int64_t ustride = m * lp;
        Mp<W> x;
        for (int64_t k = lane; k < lp; k += 32) {
            if (k < l && !wide) ld<W>(x, A, 0, i, k, rs.L);
            else set_zero<W>(x, 0u);
            write_digits<W>(x, emax, p, S, planes + i * lp + k, ustride);
        }
    }
}

// one warp per column of B: emax, spread flag, digit planes [S][n][lp]
template <int W>
__global__ void split_prep_cols(BMat B, int64_t l, int64_t n, int64_t lp, int p, int S,
                                __half *planes, int64_t *emax_out, uint8_t *wide_out)
{
    const RoundSpec rs = make_spec<W>(p);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < n; j += nwarps) {
        int64_t emax = INT64_MIN;
        for (int64_t k = lane; k < l; k += 32) {
            const int64_t e = B.exp[k * B.ld + j];
            if (e != EXP_ZERO && e > emax) emax = e;
        }
        emax = warp_max64(emax);
        bool wide = false;
        for (int64_t k = lane; k < l; k += 32) {
            const int64_t e = B.exp[k * B.ld + j];
            if (e != EXP_ZERO && e < emax - SPLIT_SB) wide = true;
        }
        wide = __any_sync(0xffffffffu, wide);
        if (lane == 0) {
            emax_out[j] = emax;
            wide_out[j] = wide ? 1 : 0;
        }
        const int64_t ustride = n * lp;
        Mp<W> x;
        for (int64_t k = lane; k < lp; k += 32) {
            if (k < l && !wide) ld<W>(x, B, 0, k, j, rs.L);
            else set_zero<W>(x, 0u);
            write_digits<W>(x, emax, p, S, planes + j * lp + k, ustride);
        }
    }
}

// bits [lo, hi) of acc (na words, lo >= 0) all equal to v (0 or 1)
MP_DEV bool bits_all(const uint32_t *acc, int na, int64_t lo, int64_t hi, uint32_t v)
{
    const uint32_t want = v ? 0xffffffffu : 0u;
    for (int64_t b = lo; b < hi;) {
        const int w = (int)(b >> 5), o = (int)(b & 31);
        const int64_t take = (hi - b) < (32 - o) ? (hi - b) : (32 - o);
        const uint32_t mask = (take == 32 ? 0xffffffffu : ((1u << take) - 1u)) << o;
        const uint32_t x = w < na ? acc[w] : 0u;
        if ((x & mask) != (want & mask)) return false;
        b += take;
    }
    return true;
}

// value = acc (two's complement, na words) * 2^e0, rounded once to p bits.
// With ebits >= 0 the exact value is acc + d for an unknown |d| < 2^ebits;
// returns false (c untouched) when that leaves the rounding open.
template <int W>
MP_DEV bool round_fixed(uint32_t *acc, int na, int64_t e0, const RoundSpec &rs, Mp<W> &c,
                        int64_t ebits = -1)
{
    set_zero<W>(c, 0u);
    const bool negative = (acc[na - 1] >> 31) != 0u;
    if (negative) {
        uint64_t cc = 1;
        for (int t = 0; t < na; ++t) {
            cc += (uint64_t)(~acc[t]);
            acc[t] = (uint32_t)cc;
            cc >>= 32;
        }
    }
    int top = na - 1;
    while (top >= 0 && acc[top] == 0u) --top;
    if (top < 0) return ebits < 0;                        // exact zero: +0
    const int lz = __clz(acc[top]);
    const int64_t lb = 32 * (int64_t)top + (31 - lz);
    if (ebits >= 0) {
        // round bit at lb - p; the midpoints have it set and zeros below
        const int64_t rb = lb - rs.p;
        if (rb < ebits + 2) return false;
        const uint32_t rbit = (acc[rb >> 5] >> (rb & 31)) & 1u;
        if (bits_all(acc, na, ebits, rb, rbit ? 0u : 1u)) return false;
    }
    auto bits_at = [&](int64_t lo) -> uint32_t {
        if (lo <= -32) return 0u;
        if (lo < 0) return acc[0] << (-lo);
        const int w = (int)(lo >> 5), s = (int)(lo & 31);
        const uint32_t x0 = (w < na) ? acc[w] : 0u;
        const uint32_t x1 = (w + 1 < na) ? acc[w + 1] : 0u;
        return s ? ((x0 >> s) | (x1 << (32 - s))) : x0;
    };
    const int64_t base = lb - 32 * W + 1;
#pragma unroll
    for (int t = 0; t < W; ++t) c.m[t] = bits_at(base + 32 * t);
    const uint32_t below = bits_at(base - 32);
    bool sticky = false;
    if (base - 32 > 0) {
        const int64_t nb = base - 32;
        const int w = (int)(nb >> 5), s = (int)(nb & 31);
        for (int t = 0; t < w && t < na; ++t) sticky |= acc[t] != 0u;
        if (s && w < na) sticky |= (acc[w] & ((1u << s) - 1u)) != 0u;
    }
    c.e = e0 + lb + 1;
    c.s = negative ? 1u : 0u;
    round_mant<W>(c.m, c.e, below, sticky, rs);
    return true;
}

template <int W> struct SplitCfg {
    static constexpr int NWD = (2 * ((32 * W + SPLIT_SB + 7) / 8 + 1) + 8) / 4 + 4;
};

// c_ij from the diagonal sums D (planes s0 .. 2S-2; rows/columns beyond the
// spread budget skipped).  ebits >= 0: the skipped diagonals sum to less
// than 2^ebits; outputs whose rounding that leaves open go to list.
template <int W>
__global__ void __launch_bounds__(64)
split_finish_kernel(const long long *__restrict__ D, int64_t m, int64_t n, int S, int p, int s0,
                    int64_t ebits, const int64_t *emaxA, const int64_t *emaxB, const uint8_t *wideA,
                    const uint8_t *wideB, BMat C, int64_t *list, unsigned long long *count,
                    DevStatus *status)
{
    constexpr int NWD = SplitCfg<W>::NWD;
    const RoundSpec rs = make_spec<W>(p);
    const int64_t total = m * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / n, j = t % n;
        if (wideA[i] || wideB[j]) continue;
        Mp<W> c;
        if (emaxA[i] == INT64_MIN || emaxB[j] == INT64_MIN) {    // a zero row or column
            set_zero<W>(c, 0u);
            if (st<W>(c, C, 0, i, j, rs.L)) flag(status, ST_RANGE);
            continue;
        }
        uint32_t acc[NWD];
        for (int w = 0; w < NWD; ++w) acc[w] = 0u;
        long long carry = 0;
        const int nd = 2 * S - 1;
        for (int s = s0; s < nd; ++s) {
            const long long v = carry + D[(int64_t)(s - s0) * total + t];
            acc[s >> 2] |= ((uint32_t)v & 0xffu) << (8 * (s & 3));
            carry = v >> 8;                                   // arithmetic: floor division
        }
        // the carry (signed) continues above digit nd - 1, sign-extended
        for (int s = nd; s < 4 * NWD; ++s) {
            acc[s >> 2] |= ((uint32_t)carry & 0xffu) << (8 * (s & 3));
            carry >>= 8;
        }
        const int64_t F = p + SPLIT_SB;
        if (!round_fixed<W>(acc, NWD, emaxA[i] + emaxB[j] - 2 * F, rs, c, ebits)) {
            list[atomicAdd(count, 1ull)] = t;                 // decided by the exact kernel
            continue;
        }
        if (st<W>(c, C, 0, i, j, rs.L)) flag(status, ST_RANGE);
    }
}

// ================================================================ launchers
template <int W>
void launch_split_prep(BMat A, BMat B, int64_t m, int64_t l, int64_t n, int p, __half *pa,
                       __half *pb, int64_t *ea, int64_t *eb, uint8_t *wa, uint8_t *wb, cudaStream_t s)
{
    const int S = split_digits(p);
    const int64_t lp = split_lpad(l);
    split_prep_rows<W><<<grid_for(m * 32, 128), 128, 0, s>>>(A, m, l, lp, p, S, pa, ea, wa);
    split_prep_cols<W><<<grid_for(n * 32, 128), 128, 0, s>>>(B, l, n, lp, p, S, pb, eb, wb);
}

template <int W>
void launch_split_finish(const long long *D, int64_t m, int64_t n, int p, int s0, int64_t ebits,
                         const int64_t *ea, const int64_t *eb, const uint8_t *wa, const uint8_t *wb,
                         BMat C, int64_t *list, unsigned long long *count, DevStatus *st, cudaStream_t s)
{
    split_finish_kernel<W><<<grid_for(m * n, 64), 64, 0, s>>>(D, m, n, split_digits(p), p, s0, ebits, ea,
                                                               eb, wa, wb, C, list, count, st);
}

#define MPG_INSTANTIATE_SPLIT(W)                                                                \
    template void launch_split_prep<W>(BMat, BMat, int64_t, int64_t, int64_t, int, __half *,    \
                                       __half *, int64_t *, int64_t *, uint8_t *, uint8_t *,    \
                                       cudaStream_t);                                           \
    template void launch_split_finish<W>(const long long *, int64_t, int64_t, int, int, int64_t, \
                                         const int64_t *, const int64_t *, const uint8_t *,     \
                                         const uint8_t *, BMat, int64_t *, unsigned long long *, \
                                         DevStatus *, cudaStream_t);

}  // namespace mpg
