// mp_exact.cuh -- C = RN_p(A B) with every dot product formed exactly and
// rounded once (the result the split form must reproduce bit for bit).
//
// One thread per c_ij.  Pass 1 reads the exponents of row i of A and column
// j of B to find the range [Emin, Emax] of the products' exponents.  Pass 2
// adds every exact 2W-word product a_ik b_kj into a two's complement
// fixed-point accumulator (per-thread local memory) whose bit 0 has weight
// 2^(Emin - 64W); the width covers the products' spread, 64W product bits,
// log2(l) bits of headroom and a sign bit.  The accumulator is then rounded
// once to p bits.  A spread too wide for the accumulator cap is reported
// (ST_WIDE) and that c_ij is left +0.
#pragma once
#include "mp_kernels.cuh"

namespace mpg {

template <int W> struct ExactCfg {
    static constexpr int NA = 4 * W + 48;          // accumulator words (cap)
    static constexpr int THREADS = (W <= 16) ? 128 : 64;
};

// acc[q .. q + N] += x (N words) << r   (0 <= r < 32), carry rippled up to NA
template <int W, int N>
MP_DEV void acc_add_shifted(uint32_t *acc, int na, int q, int r, const uint32_t (&x)[N], bool neg)
{
    // shifted value in N + 1 words; two's complement when subtracting
    uint32_t s[N + 1];
    s[0] = x[0] << r;
#pragma unroll
    for (int i = 1; i < N; ++i) s[i] = __funnelshift_l(x[i - 1], x[i], r);
    s[N] = r ? (x[N - 1] >> (32 - r)) : 0u;
    const uint32_t mask = neg ? 0xffffffffu : 0u;
    // add (s ^ mask) + neg at word q, then extend with mask words (sign) upward
    uint64_t c = neg ? 1u : 0u;
#pragma unroll
    for (int i = 0; i <= N; ++i) {
        c += (uint64_t)acc[q + i] + (uint64_t)(s[i] ^ mask);
        acc[q + i] = (uint32_t)c;
        c >>= 32;
    }
    for (int i = q + N + 1; i < na; ++i) {
        c += (uint64_t)acc[i] + (uint64_t)mask;
        acc[i] = (uint32_t)c;
        c >>= 32;
    }
}

template <int W>
__device__ __noinline__ void exact_one(const BMat &A, const BMat &B, const BMat &C, int64_t i,
                                       int64_t j, int64_t l, const RoundSpec &rs, DevStatus *status);

// rowsel / colsel (optional): compute only c_ij with rowsel[i] | colsel[j]
template <int W>
__global__ void __launch_bounds__(ExactCfg<W>::THREADS)
gemm_exact_kernel(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p, DevStatus *status,
                  const uint8_t *rowsel, const uint8_t *colsel)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const bool cj = colsel ? colsel[j] != 0 : true;
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
        if (rowsel && !(rowsel[i] || cj)) continue;
        exact_one<W>(A, B, C, i, j, l, rs, status);
    }
}

template <int W>
__device__ __noinline__ void exact_one(const BMat &A, const BMat &B, const BMat &C, int64_t i,
                                       int64_t j, int64_t l, const RoundSpec &rs, DevStatus *status)
{
    constexpr int NA = ExactCfg<W>::NA;
    // pass 1: exponent range of the nonzero products
    int64_t emin = 0, emax = 0;
    bool any = false;
    for (int64_t k = 0; k < l; ++k) {
        const int64_t ea = __ldg(A.exp + i * A.ld + k), eb = __ldg(B.exp + k * B.ld + j);
        if (ea == EXP_ZERO || eb == EXP_ZERO) continue;
        const int64_t e = ea + eb;
        if (!any) { emin = emax = e; any = true; }
        emin = e < emin ? e : emin;
        emax = e > emax ? e : emax;
    }
    Mp<W> c;
    set_zero<W>(c, 0u);
    if (!any) {                                   // every product is zero: +0
        if (st<W>(c, C, 0, i, j, rs.L)) flag(status, ST_RANGE);
        return;
    }
    int hb = 1;                                   // headroom bits for l terms
    while (((int64_t)1 << hb) <= l) ++hb;
    const int64_t width = (emax - emin) + 64 * W + hb + 2;
    const int na = (int)((width + 31) / 32) + 1;
    if (na > NA) {
        flag(status, ST_WIDE);
        st<W>(c, C, 0, i, j, rs.L);
        return;
    }
    uint32_t acc[NA];
    for (int t = 0; t < na; ++t) acc[t] = 0u;
    // pass 2: exact accumulation
    Mp<W> a, b;
    for (int64_t k = 0; k < l; ++k) {
        ld<W>(a, A, 0, i, k, rs.L);
        ld<W>(b, B, 0, k, j, rs.L);
        if (a.e == EXP_ZERO || b.e == EXP_ZERO) continue;
        const int64_t off = a.e + b.e - emin;
        const int q = (int)(off >> 5), r = (int)(off & 31);
        uint32_t P[2 * W];
        if constexpr (W <= 32) {
            mul_full<W>(P, a.m, b.m);
        } else {
            // 2048-bit: the product row by row through local memory
#pragma unroll 1
            for (int t = 0; t < 2 * W; ++t) P[t] = 0u;
#pragma unroll 1
            for (int jj = 0; jj < W; ++jj) {
                uint64_t cc = 0;
#pragma unroll 1
                for (int ii = 0; ii < W; ++ii) {
                    cc += (uint64_t)a.m[ii] * b.m[jj] + P[ii + jj];
                    P[ii + jj] = (uint32_t)cc;
                    cc >>= 32;
                }
                P[jj + W] = (uint32_t)cc;
            }
        }
        acc_add_shifted<W, 2 * W>(acc, na, q, r, P, (a.s ^ b.s) != 0u);
    }
    // sign and magnitude of the exact sum
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
    if (top < 0) {                                // exact zero sum: +0
        if (st<W>(c, C, 0, i, j, rs.L)) flag(status, ST_RANGE);
        return;
    }
    // leading one at bit lb; the top W words below it form the mantissa
    const int lz = __clz(acc[top]);
    const int64_t lb = 32 * (int64_t)top + (31 - lz);
    // gather bits [lb - 32W + 1, lb] into m (word i covers bits lb-32W+1+32i ..)
    auto bits_at = [&](int64_t lo) -> uint32_t {   // 32 bits starting at bit lo (lo may be < 0)
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
        const int64_t nb = base - 32;              // bits [0, nb) remain
        const int w = (int)(nb >> 5), s = (int)(nb & 31);
        for (int t = 0; t < w && t < na; ++t) sticky |= acc[t] != 0u;
        if (s && w < na) sticky |= (acc[w] & ((1u << s) - 1u)) != 0u;
    }
    // value = acc * 2^(emin - 64W); the mantissa fraction starts at bit lb
    c.e = emin - 64 * (int64_t)W + lb + 1;
    c.s = negative ? 1u : 0u;
    round_mant<W>(c.m, c.e, below, sticky, rs);
    if (st<W>(c, C, 0, i, j, rs.L)) flag(status, ST_RANGE);
}

// the outputs t = i n + j listed in list[0 .. *count), one thread each
template <int W>
__global__ void __launch_bounds__(ExactCfg<W>::THREADS)
gemm_exact_list_kernel(BMat A, BMat B, BMat C, int64_t n, int64_t l, int p, DevStatus *status,
                       const int64_t *list, const unsigned long long *count)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t cnt = (int64_t)*count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && cnt) atomicAdd(&status->split_fallbacks, (unsigned long long)cnt);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < cnt;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = list[q];
        exact_one<W>(A, B, C, t / n, t % n, l, rs, status);
    }
}

template <int W>
void launch_gemm_exact_list(BMat A, BMat B, BMat C, int64_t n, int64_t l, int p, DevStatus *st,
                            cudaStream_t s, const int64_t *list, const unsigned long long *count)
{
    constexpr int T = ExactCfg<W>::THREADS;
    gemm_exact_list_kernel<W><<<152 * 4, T, 0, s>>>(A, B, C, n, l, p, st, list, count);
}

template <int W>
void launch_gemm_exact(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p,
                       DevStatus *st, cudaStream_t s, const uint8_t *rowsel, const uint8_t *colsel)
{
    if (m <= 0 || n <= 0) return;
    constexpr int T = ExactCfg<W>::THREADS;
    dim3 grid((unsigned)((n + T - 1) / T), (unsigned)(m < 65535 ? m : 65535));
    gemm_exact_kernel<W><<<grid, T, 0, s>>>(A, B, C, m, l, n, p, st, rowsel, colsel);
}

#define MPG_INSTANTIATE_EXACT(W)                                                                \
    template void launch_gemm_exact<W>(BMat, BMat, BMat, int64_t, int64_t, int64_t, int,        \
                                       DevStatus *, cudaStream_t, const uint8_t *,              \
                                       const uint8_t *);                                        \
    template void launch_gemm_exact_list<W>(BMat, BMat, BMat, int64_t, int64_t, int, DevStatus *, \
                                            cudaStream_t, const int64_t *,                      \
                                            const unsigned long long *);

}  // namespace mpg
