// mp_kernels.cuh -- kernel templates of the MP GEMM path (arXiv 1410.1599
// Sec. 2), instantiated once per word-capacity class W by gemm_w*.cu and
// rec_w*.cu.
#pragma once
#include <cstring>
#include <mutex>

#include "mp_arith.cuh"
#include "mp_internal.h"
#include "mp_tc.cuh"

namespace mpg {

// ----------------------------------------------------------------- helpers
MP_DEV int64_t lim_off(const BMat &M, int64_t b, int64_t r, int64_t c)
{
    return b * M.bs_limb + r * M.ld + c;
}
MP_DEV int64_t es_off(const BMat &M, int64_t b, int64_t r, int64_t c)
{
    return b * M.bs_es + r * M.ld + c;
}

template <int W>
MP_DEV void ld(Mp<W> &x, const BMat &M, int64_t b, int64_t r, int64_t c, int L)
{
    const int64_t lo = lim_off(M, b, r, c), eo = es_off(M, b, r, c);
#pragma unroll (is_big<W>() ? 4 : W / 2)
    for (int k = 0; k < W / 2; ++k) {
        uint64_t v = (k < L) ? __ldg(M.limb + lo + (int64_t)k * M.plane) : 0ull;
        x.m[W - 1 - 2 * k] = (uint32_t)(v >> 32);
        x.m[W - 2 - 2 * k] = (uint32_t)v;
    }
    x.e = __ldg(M.exp + eo);
    x.s = (uint32_t)(__ldg(M.sign + eo) & 1);
}

// load through the coherent path (for data written earlier in the same kernel)
template <int W>
MP_DEV void ld_rw(Mp<W> &x, const BMat &M, int64_t b, int64_t r, int64_t c, int L)
{
    const int64_t lo = lim_off(M, b, r, c), eo = es_off(M, b, r, c);
#pragma unroll (is_big<W>() ? 4 : W / 2)
    for (int k = 0; k < W / 2; ++k) {
        uint64_t v = (k < L) ? M.limb[lo + (int64_t)k * M.plane] : 0ull;
        x.m[W - 1 - 2 * k] = (uint32_t)(v >> 32);
        x.m[W - 2 - 2 * k] = (uint32_t)v;
    }
    x.e = M.exp[eo];
    x.s = (uint32_t)(M.sign[eo] & 1);
}

template <int W>
MP_DEV void ld_or_zero(Mp<W> &x, bool valid, const BMat &M, int64_t b, int64_t r, int64_t c,
                       int L)
{
    if (valid) ld<W>(x, M, b, r, c, L);
    else set_zero<W>(x, 0u);
}

template <int W>
MP_DEV bool st(const Mp<W> &x, const BMat &M, int64_t b, int64_t r, int64_t c, int L)
{
    const int64_t lo = lim_off(M, b, r, c), eo = es_off(M, b, r, c);
#pragma unroll (is_big<W>() ? 4 : W / 2)
    for (int k = 0; k < W / 2; ++k)
        if (k < L)
            M.limb[lo + (int64_t)k * M.plane] =
                ((uint64_t)x.m[W - 1 - 2 * k] << 32) | (uint64_t)x.m[W - 2 - 2 * k];
    M.exp[eo] = x.e;
    M.sign[eo] = (int8_t)x.s;
    return out_of_range<W>(x);
}

MP_DEV void flag(DevStatus *st, unsigned f)
{
    if (st) atomicOr(&st->flags, f);
}

// ----------------------------------------------------------- elementwise
template <int W>
__global__ void elementwise_kernel(int op, BMat X, BMat Y, BMat R, int64_t rows, int64_t cols,
                                   int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t total = rows * cols;
    bool bad = false, dz = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols, c = t % cols;
        Mp<W> x, y, z;
        ld<W>(x, X, 0, r, c, rs.L);
        ld<W>(y, Y, 0, r, c, rs.L);
        if (op == 0) add<W>(z, x, y, 0u, rs);
        else if (op == 1) add<W>(z, x, y, 1u, rs);
        else if (op == 2) mul<W>(z, x, y, rs);
        else {
            if (y.e == EXP_ZERO) { dz = true; continue; }
            div<W>(z, x, y, rs);
        }
        bad |= st<W>(z, R, 0, r, c, rs.L);
    }
    if (bad) flag(status, ST_RANGE);
    if (dz) flag(status, ST_DIVZERO);
}

template <int W>
__global__ void convert_kernel(BMat X, int px, BMat R, int pr, int64_t rows, int64_t cols,
                               DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(pr);
    const int Lx = (px + 63) >> 6;
    const int64_t total = rows * cols;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols, c = t % cols;
        Mp<W> x;
        ld<W>(x, X, 0, r, c, Lx);
        if (x.e != EXP_ZERO) round_mant<W>(x.m, x.e, 0u, false, rs);
        bad |= st<W>(x, R, 0, r, c, rs.L);
    }
    if (bad) flag(status, ST_RANGE);
}

// ---------------------------------------------------------- Simple (Eq. 1)
// One thread per c_ij of product blockIdx.z of a batch; operands read
// straight from global memory (through the read-only cache), k ascending:
// c = RN(c + RN(a_ik b_kj)).  The wide class also takes its Block leaves
// here (same bits): its numbers live in local memory either way, and this
// kernel keeps four CTAs per SM where the shared-memory leaf fits one.
template <int W> struct SimpleCfg {
    static constexpr int TY = (W <= 16) ? 8 : (W == 32 ? 4 : (W == 64 ? 2 : 4));
    static constexpr int MIN_CTAS = (W <= 16) ? 3 : (is_big<W>() ? 4 : 1);
};

// SUB: c starts from C's own entry and each product is subtracted,
// c = RN(c - RN(a_ik b_kj)) for k ascending (the LU's elimination sequence).
template <int W, bool BATCHED = false, bool SUB = false>
__global__ void __launch_bounds__(32 * SimpleCfg<W>::TY, SimpleCfg<W>::MIN_CTAS)
gemm_simple_kernel(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p,
                   DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
    const int64_t bt = BATCHED ? (int64_t)blockIdx.z : 0;
    if (i >= m || j >= n) return;
    Mp<W> c, a, b, t;
    if (SUB) ld_rw<W>(c, C, bt, i, j, rs.L);
    else set_zero<W>(c, 0u);
    for (int64_t k = 0; k < l; ++k) {
        ld<W>(a, A, bt, i, k, rs.L);
        ld<W>(b, B, bt, k, j, rs.L);
        mul<W, true>(t, a, b, rs);
        add<W, true>(c, c, t, SUB ? 1u : 0u, rs);
    }
    if (st<W>(c, C, bt, i, j, rs.L)) flag(status, ST_RANGE);
}

// ---------------------------------------------------- Block (Eq. 2), batched
// C_b = A_b B_b for a batch of equally shaped products (the leaves of the
// Strassen/Winograd recursion, or one plain product).  Each CTA owns a
// BM x 32 tile of C (one element per thread) and walks k in slabs of BK; every
// c_ij accumulates in k-ascending order, so the bits equal Simple's.
// Each thread keeps c and a_ik in registers and reads b_kj word by word from
// shared memory (four words per 16-byte load) while it forms the product:
// three register operands would cost resident CTAs at every precision and do
// not fit at all at 2048 bits.  The slabs are stored one element per record
// (mantissa words little-endian; B records padded so that a warp's 16-byte
// loads hit every bank once).

// rows of b words streamed from shared memory (four at a time, through the
// reader br: RecWords or PlaneWords); each partial product with the row
// carry as one 64-bit multiply-add
template <int W, class BR>
MP_DEV void mul_trunc_rows_sm(uint32_t (&acc)[W + 2], const uint32_t (&a)[W], const BR &br)
{
#pragma unroll
    for (int q = 0; q < W + 2; ++q) acc[q] = 0u;
#pragma unroll
    for (int j0 = 0; j0 < W; j0 += 4) {
        uint32_t bv[4];
        br.load4(j0, bv);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u;
            const uint32_t bj = bv[u];
            const int i0 = (W - 2 - j > 0) ? W - 2 - j : 0;
            // position i + j lives in acc[i + j - (W - 2)]
            uint64_t c = 0;
#pragma unroll
            for (int i = i0; i < W; ++i) {
                const uint64_t t = (uint64_t)a[i] * bj + acc[j + i - (W - 2)] + c;
                acc[j + i - (W - 2)] = (uint32_t)t;
                c = t >> 32;
            }
            acc[j + 2] = (uint32_t)c;                   // not yet written by any row
        }
    }
}

// top words of the truncated product a * b (b loaded into registers from
// shared memory): acc[q] = word W-2+q of sum_{i+j >= W-2} a_i b_j 2^(32(i+j))
//
// Up to 1024 bits the product is formed column by column (product
// scanning): the partial products of word s = i + j are summed into a
// three-word accumulator by one multiply-add chain with carry flags
// (mad.lo.cc, madc.hi.cc, addc), the low word leaves as word s and the
// other two move down.  Each partial product costs one wide multiply-add
// and one carry add -- about 30 % fewer instructions than rows of 64-bit
// multiply-adds, whose row carries need separate adds (the 512-bit leaf
// measured 682 against 871 instructions per multiply-add, same bits).  At
// 2048 bits b does not fit in registers beside a, c and the product, and
// rows of b words streamed from shared memory are used instead.
template <int W>
MP_DEV void mul_trunc_cols(uint32_t (&acc)[W + 2], const uint32_t (&a)[W], const uint32_t (&b)[W])
{
    static_assert(W <= 32, "b in registers");
    uint32_t c0 = 0u, c1 = 0u, c2 = 0u;
#pragma unroll
    for (int s = W - 2; s <= 2 * W - 2; ++s) {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int j = s - i;
            if (j < 0 || j >= W) continue;
            asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
                "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
                "addc.u32 %2, %2, 0;"
                : "+r"(c0), "+r"(c1), "+r"(c2) : "r"(a[i]), "r"(b[j]));
        }
        acc[s - (W - 2)] = c0;
        c0 = c1;
        c1 = c2;
        c2 = 0u;
    }
    acc[W + 1] = c0;
}

// b's mantissa in shared memory, as one record of W words (little-endian,
// 16-byte aligned: four words per load) ...
template <int W>
struct RecWords {
    const uint32_t *p;
    MP_DEV void load(uint32_t (&b)[W]) const
    {
#pragma unroll
        for (int j0 = 0; j0 < W; j0 += 4) {
            const uint4 v = *reinterpret_cast<const uint4 *>(p + j0);
            b[j0] = v.x;
            b[j0 + 1] = v.y;
            b[j0 + 2] = v.z;
            b[j0 + 3] = v.w;
        }
    }
    MP_DEV uint32_t operator[](int j) const { return p[j]; }
    // words j0 .. j0+3 (j0 a multiple of 4)
    MP_DEV void load4(int j0, uint32_t (&v)[4]) const
    {
        const uint4 x = *reinterpret_cast<const uint4 *>(p + j0);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    }
};

// ... or as limb planes (limb q, most significant first, at p[q * stride]:
// words W-1-2q and W-2-2q), the layout the bulk tensor copies produce
template <int W>
struct PlaneWords {
    const uint64_t *p;
    int stride;
    MP_DEV void load(uint32_t (&b)[W]) const
    {
#pragma unroll
        for (int q = 0; q < W / 2; ++q) {
            const uint64_t v = p[q * stride];
            b[W - 2 - 2 * q] = (uint32_t)v;
            b[W - 1 - 2 * q] = (uint32_t)(v >> 32);
        }
    }
    MP_DEV uint32_t operator[](int j) const
    {
        const uint64_t v = p[((W - 1 - j) >> 1) * stride];
        return (j & 1) ? (uint32_t)(v >> 32) : (uint32_t)v;
    }
    // words j0 .. j0+3 (j0 a multiple of 4): the low and high halves of
    // limbs (W-2-j0)/2 and (W-4-j0)/2
    MP_DEV void load4(int j0, uint32_t (&v)[4]) const
    {
        const uint64_t x = p[((W - 2 - j0) >> 1) * stride], y = p[((W - 4 - j0) >> 1) * stride];
        v[0] = (uint32_t)x;
        v[1] = (uint32_t)(x >> 32);
        v[2] = (uint32_t)y;
        v[3] = (uint32_t)(y >> 32);
    }
};

// t = RN_p(a * b) with b's mantissa in shared memory (p = 32W or below),
// read through bm (RecWords or PlaneWords; PlaneWords for W <= 32 only)
template <int W, class BR>
MP_DEV void mul_sm(Mp<W> &t, const uint32_t (&am)[W], int64_t ae, uint32_t as, const BR &bm,
                   int64_t be, uint32_t bs, const RoundSpec &rs)
{
    t.s = as ^ bs;
    if (ae == EXP_ZERO || be == EXP_ZERO) {
        set_zero<W>(t, t.s);
        return;
    }
    int64_t e = ae + be;
    if (rs.r == 0) {
        // the truncation test of mul_impl: decide from the truncated product
        // unless its error bound reaches the rounding boundary
        uint32_t acc[W + 2];
        if constexpr (W <= 32) {
            uint32_t b[W];
            bm.load(b);
            mul_trunc_cols<W>(acc, am, b);
        } else {
            mul_trunc_rows_sm<W>(acc, am, bm);
        }
        const uint32_t w = acc[1];
        const uint32_t top = acc[W + 1] >> 31;
        const int rpos = top ? 31 : 30;
        const uint32_t wend = w + (uint32_t)(W - 1);
        const uint32_t rb = (w >> rpos) & 1u;
        const bool safe = (wend >= w) && ((w >> rpos) == (wend >> rpos)) &&
                          !(rb && (w & ((1u << rpos) - 1u)) == 0u);
        if (safe) {
            if (!top) {
#pragma unroll
                for (int i = W + 1; i > 2; --i) acc[i] = __funnelshift_l(acc[i - 1], acc[i], 1);
                acc[2] = __funnelshift_l(w, acc[2], 1);
                e -= 1;
            }
            acc[2] = add_cc(acc[2], rb);
#pragma unroll
            for (int i = 3; i < W + 2; ++i) acc[i] = addc_cc(acc[i], 0u);
            const uint32_t c = addc(0u, 0u);
#pragma unroll
            for (int i = 0; i < W; ++i) t.m[i] = acc[i + 2];
            if (c) {
                t.m[W - 1] = 0x80000000u;
                e += 1;
            }
            t.e = e;
            return;
        }
    }
    // exact top half with sticky (rare for p = 32W)
    uint32_t pw1, pw2;
    bool low_nz;
    mul_top<W>(t.m, pw1, pw2, low_nz, am, bm);
    if (!(t.m[W - 1] >> 31)) {
#pragma unroll
        for (int i = W - 1; i > 0; --i) t.m[i] = (t.m[i] << 1) | (t.m[i - 1] >> 31);
        t.m[0] = (t.m[0] << 1) | (pw1 >> 31);
        pw1 = (pw1 << 1) | (pw2 >> 31);
        pw2 <<= 1;
        e -= 1;
    }
    round_mant<W>(t.m, e, pw1, low_nz || pw2 != 0u, rs);
    t.e = e;
}

#ifndef MPG_SM16_BM
#define MPG_SM16_BM 8
#endif
#ifndef MPG_SM16_BK
#define MPG_SM16_BK 16
#endif
#ifndef MPG_SM16_MINCTAS
#define MPG_SM16_MINCTAS 3
#endif
#ifndef MPG_SM8_MINCTAS
#define MPG_SM8_MINCTAS 4
#endif
#ifndef MPG_SM4_MINCTAS
#define MPG_SM4_MINCTAS 6
#endif
template <int W> struct BlockSmCfg {
    static constexpr int BN = 32, BM = (W <= 16) ? MPG_SM16_BM : 4;
    static constexpr int BK = (W == 64) ? 4 : (W <= 16 ? MPG_SM16_BK : 8), THREADS = BM * BN;
    static constexpr int RB = (W == 4) ? 12 : W + 4;  // words per B record (bank-conflict-free 16-byte loads)
    static constexpr int MIN_CTAS = (W == 4) ? MPG_SM4_MINCTAS : (W == 8) ? MPG_SM8_MINCTAS
                                  : (W == 16) ? MPG_SM16_MINCTAS : ((W <= 32) ? 3 : 1);   // resident CTAs per SM to plan registers for
    static constexpr size_t smem()
    {
        return (size_t)BK * BN * RB * 4 + (size_t)BM * BK * W * 4 + (size_t)(BM * BK + BK * BN) * 9;
    }
};

// product b's operand: M shifted to batch element b (a view with no batch
// stride of its own)
MP_DEV BMat batch_view(const BMat &M, int64_t b)
{
    return BMat{M.limb + b * M.bs_limb, M.exp + b * M.bs_es, M.sign + b * M.bs_es, M.ld, M.plane, 0, 0};
}

// quadrant q (1..4: 11, 12, 21, 22) of parent node `node` of P, quadrants of
// hq x wq numbers
MP_DEV BMat quadrant_view(const BMat &P, int64_t node, int q, int64_t hq, int64_t wq)
{
    const int64_t off = ((q - 1) >> 1) * hq * P.ld + ((q - 1) & 1) * wq;
    return BMat{P.limb + node * P.bs_limb + off, P.exp + node * P.bs_es + off, P.sign + node * P.bs_es + off,
                P.ld, P.plane, 0, 0};
}

// The tile with product b's operands given as views (Ab, Bb); C is indexed
// by batch element b.
template <int W, bool SUB>
MP_DEV void block_sm_tile_views(const BMat &A, const BMat &B, const BMat &C, int64_t b, int64_t m, int64_t l,
                                int64_t n, int p, int64_t tiles_m, int64_t tiles_n, int64_t tile,
                                DevStatus *status)
{
    using Cfg = BlockSmCfg<W>;
    static_assert(W == 4 || W == 8 || W == 16 || W == 32 || W == 64, "leaf class (the wide class takes the Simple kernel)");
    constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, RB = Cfg::RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RoundSpec rs = make_spec<W>(p);
    const int L = rs.L;
    // [BK][BN] records of RB words, [BM][BK] records of W words, exps, signs
    uint32_t *sB = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *sA = sB + BK * BN * RB;
    int64_t *sAe = reinterpret_cast<int64_t *>(sA + BM * BK * W);
    int64_t *sBe = sAe + BM * BK;
    int8_t *sAs = reinterpret_cast<int8_t *>(sBe + BK * BN);
    int8_t *sBs = sAs + BM * BK;

    const int64_t tm = (tile / tiles_n) % tiles_m, tn = tile % tiles_n;
    const int tx = threadIdx.x % BN, ty = threadIdx.x / BN;
    const int64_t i = tm * BM + ty, j = tn * BN + tx;
    const bool valid = (i < m) && (j < n);

    Mp<W> c, t;
    if (SUB && valid) ld_rw<W>(c, C, b, i, j, L);
    else set_zero<W>(c, 0u);
    for (int64_t k0 = 0; k0 < l; k0 += BK) {
        const int kc = (int)((l - k0) < BK ? (l - k0) : BK);
        // limb q of a record goes to words W-2-2q (low half) and W-1-2q
        for (int e = threadIdx.x; e < W / 2 * BK * BN; e += blockDim.x) {
            const int cc = e % BN, kk = (e / BN) % BK, q = e / (BN * BK);
            const int64_t gj = tn * BN + cc, gk = k0 + kk;
            const uint64_t v = (q < L && gj < n && kk < kc)
                                   ? __ldg(B.limb + (int64_t)q * B.plane + gk * B.ld + gj)
                                   : 0ull;
            *reinterpret_cast<uint64_t *>(sB + (kk * BN + cc) * RB + (W - 2 - 2 * q)) = v;
        }
        for (int e = threadIdx.x; e < W / 2 * BM * BK; e += blockDim.x) {
            const int kk = e % BK, rr = (e / BK) % BM, q = e / (BK * BM);
            const int64_t gi = tm * BM + rr, gk = k0 + kk;
            const uint64_t v = (q < L && gi < m && kk < kc)
                                   ? __ldg(A.limb + (int64_t)q * A.plane + gi * A.ld + gk)
                                   : 0ull;
            *reinterpret_cast<uint64_t *>(sA + (rr * BK + kk) * W + (W - 2 - 2 * q)) = v;
        }
        for (int e = threadIdx.x; e < BM * BK; e += blockDim.x) {
            const int kk = e % BK, rr = e / BK;
            const int64_t gi = tm * BM + rr, gk = k0 + kk;
            const bool ok = gi < m && kk < kc;
            sAe[e] = ok ? __ldg(A.exp + gi * A.ld + gk) : EXP_ZERO;
            sAs[e] = ok ? __ldg(A.sign + gi * A.ld + gk) : (int8_t)0;
        }
        for (int e = threadIdx.x; e < BK * BN; e += blockDim.x) {
            const int cc = e % BN, kk = e / BN;
            const int64_t gj = tn * BN + cc, gk = k0 + kk;
            const bool ok = gj < n && kk < kc;
            sBe[e] = ok ? __ldg(B.exp + gk * B.ld + gj) : EXP_ZERO;
            sBs[e] = ok ? __ldg(B.sign + gk * B.ld + gj) : (int8_t)0;
        }
        __syncthreads();
        if (valid) {
            for (int kk = 0; kk < kc; ++kk) {
                uint32_t am[W];
                const uint32_t *ap = sA + (ty * BK + kk) * W;
#pragma unroll
                for (int q = 0; q < W; q += 4) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(ap + q);
                    am[q] = v.x;
                    am[q + 1] = v.y;
                    am[q + 2] = v.z;
                    am[q + 3] = v.w;
                }
                mul_sm<W>(t, am, sAe[ty * BK + kk], (uint32_t)(sAs[ty * BK + kk] & 1),
                          RecWords<W>{sB + (kk * BN + tx) * RB}, sBe[kk * BN + tx],
                          (uint32_t)(sBs[kk * BN + tx] & 1), rs);
                add_impl<W>(c, c, t, SUB ? 1u : 0u, rs);
            }
        }
        __syncthreads();
    }
    if (valid && st<W>(c, C, b, i, j, L)) flag(status, ST_RANGE);
}

// One BM x 32 tile of C_b = A_b B_b: tile = (b, tm, tn) in row-major order
// over batch x tiles_m x tiles_n.  SUB: c starts from C's own entry and the
// products are subtracted (see gemm_simple_kernel).
template <int W, bool SUB>
MP_DEV void block_sm_tile(const BMat &A, const BMat &B, const BMat &C, int64_t m, int64_t l, int64_t n,
                          int p, int64_t tiles_m, int64_t tiles_n, int64_t tile, DevStatus *status)
{
    const int64_t b = tile / (tiles_m * tiles_n);
    block_sm_tile_views<W, SUB>(batch_view(A, b), batch_view(B, b), C, b, m, l, n, p, tiles_m, tiles_n, tile,
                                status);
}

template <int W, bool SUB = false>
__global__ void __launch_bounds__(BlockSmCfg<W>::THREADS, BlockSmCfg<W>::MIN_CTAS)
gemm_block_sm_kernel(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p,
                     int64_t tiles_m, int64_t tiles_n, DevStatus *status)
{
    block_sm_tile<W, SUB>(A, B, C, m, l, n, p, tiles_m, tiles_n, (int64_t)blockIdx.x, status);
}

// The leaves of a Strassen / Winograd recursion, where the children that
// are plain quadrants of their parent node (Winograd's M2, M3, M7 on the A
// side, M2, M3, M6 on the B side; Strassen's P3, P4 / P2, P5) were not
// copied: leaf b = 7 node + t reads such an operand straight from the
// parent's quadrant (LeafViews), the others from the children buffers.
template <int W>
__global__ void __launch_bounds__(BlockSmCfg<W>::THREADS, BlockSmCfg<W>::MIN_CTAS)
gemm_block_leaf_views_kernel(BMat A, BMat B, BMat C, const __grid_constant__ LeafViews v, int64_t m, int64_t l,
                             int64_t n, int p, int64_t tiles_m, int64_t tiles_n, DevStatus *status)
{
    const int64_t tile = blockIdx.x;
    const int64_t b = tile / (tiles_m * tiles_n);
    const int64_t node = b / 7;
    const int t = (int)(b % 7);
    const BMat Ab = v.qa[t] ? quadrant_view(v.Ap, node, v.qa[t], m, l) : batch_view(A, b);
    const BMat Bb = v.qb[t] ? quadrant_view(v.Bp, node, v.qb[t], l, n) : batch_view(B, b);
    block_sm_tile_views<W, false>(Ab, Bb, C, b, m, l, n, p, tiles_m, tiles_n, tile, status);
}

// Several batches of products of one precision in one launch (the serving
// loop's groups: the leaves of several requests' recursions).  Batch g owns
// the CTAs [first[g], first[g + 1]); each runs one tile of its batch.
template <int W>
__global__ void __launch_bounds__(BlockSmCfg<W>::THREADS, BlockSmCfg<W>::MIN_CTAS)
gemm_block_group_kernel(const __grid_constant__ LeafGroup grp, int p, DevStatus *status)
{
    const int64_t t = blockIdx.x;
    int g = 0;
    while (g + 1 < grp.count && t >= grp.first[g + 1]) ++g;
    const LeafBatch &lb = grp.batch[g];
    block_sm_tile<W, false>(lb.A, lb.B, lb.C, lb.m, lb.l, lb.n, p, lb.tiles_m, lb.tiles_n, t - grp.first[g],
                            status);
}

// ------------------------------------------- Block leaf with TMA staging
// The same tile as block_sm_tile_views -- one output per thread, c and a_ik
// in registers, k ascending, so the same bits -- with the A and B limb tiles
// of each k-chunk brought into shared memory by bulk tensor copies (TMA)
// instead of the threads' loads.  Two stages: while the CTA works on chunk
// c, the copy engine fetches chunk c + 1 into the other stage, and one
// barrier per chunk separates the stages' reuse.  The copies land as limb
// planes ([L][BK][BN] for B, [L][BM][BK] for A), which the product reads
// through PlaneWords; planes L .. W/2-1 are zeroed once and never written.
// Exponents and signs (9 bytes an element against 8L of limbs) are loaded by
// the threads, with zero exponents outside the product, so the copies may
// read past a ragged tile's edge without effect.  Slab depths BK per class
// were chosen by measurement.
#ifndef MPG_TMA8_BK
#define MPG_TMA8_BK 16
#endif
#ifndef MPG_TMA16_BK
#define MPG_TMA16_BK 8
#endif
#ifndef MPG_TMA32_BK
#define MPG_TMA32_BK 6
#endif
template <int W> struct BlockTmaCfg {
    using S = BlockSmCfg<W>;
    static constexpr int BN = S::BN, BM = S::BM, THREADS = S::THREADS, MIN_CTAS = S::MIN_CTAS;
    static constexpr int LM = W / 2;                                  // limb planes a stage holds
    static constexpr int BK = (W == 4) ? 16 : (W == 8) ? MPG_TMA8_BK : (W == 16) ? MPG_TMA16_BK
                            : (W == 32) ? MPG_TMA32_BK : 4;
    static constexpr int NB = BK * BN, NA = BM * BK;                 // elements of a B / A chunk
    static constexpr size_t B_ST = (size_t)NB * LM * 8, A_ST = (size_t)NA * LM * 8;
    static_assert(B_ST % 128 == 0 && A_ST % 128 == 0, "stages keep 128-byte alignment");
    static_assert((BK * 8) % 16 == 0, "A box rows of whole 16-byte units");
    static constexpr size_t smem()
    {
        return 128 + 2 * (B_ST + A_ST) + 2 * (size_t)(NB + NA) * 9 + 16;
    }
};

// the tensor maps of one launch: the operands' batches and, for the leaves
// with in-place quadrants, the parents (LeafViews)
struct TmaOps {
    CUtensorMap a, b, ap, bp;
};

constexpr long long TMA_WAIT_LIMIT = 1ll << 31;   // clock cycles, about a second

template <int W, bool VIEWS>
__global__ void __launch_bounds__(BlockTmaCfg<W>::THREADS, BlockTmaCfg<W>::MIN_CTAS)
gemm_block_tma_kernel(const __grid_constant__ TmaOps ops, BMat A, BMat B, BMat C, const __grid_constant__ LeafViews v,
                      int64_t m, int64_t l, int64_t n, int p, int64_t tiles_m, int64_t tiles_n, DevStatus *status)
{
    using Cfg = BlockTmaCfg<W>;
    static_assert(W <= 64, "register classes");
    constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, LM = Cfg::LM, NB = Cfg::NB, NA = Cfg::NA;
    constexpr int NT = Cfg::THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((128u - (tc::saddr(smem_raw) & 127u)) & 127u);
    uint64_t *sB = reinterpret_cast<uint64_t *>(sm);                 // [2][LM][BK][BN]
    uint64_t *sA = sB + 2 * LM * NB;                                 // [2][LM][BM][BK]
    int64_t *sBe = reinterpret_cast<int64_t *>(sA + 2 * LM * NA);   // [2][BK * BN]
    int64_t *sAe = sBe + 2 * NB;                                     // [2][BM * BK]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sAe + 2 * NA);      // [2]
    int8_t *sBs = reinterpret_cast<int8_t *>(bar + 2);               // [2][BK * BN]
    int8_t *sAs = sBs + 2 * NB;                                      // [2][BM * BK]

    const RoundSpec rs = make_spec<W>(p);
    const int L = rs.L;
    const int64_t tile = blockIdx.x;
    const int64_t b = tile / (tiles_m * tiles_n);
    const int64_t tm = (tile / tiles_n) % tiles_m, tn = tile % tiles_n;
    // product b's operands: views for the exponents and signs, tensor map
    // and box origin (x = column, y = row, w = batch element) for the limbs
    const CUtensorMap *ma = &ops.a, *mb = &ops.b;
    int32_t ax = 0, ay = 0, aw = (int32_t)b, bx = 0, by = 0, bw = (int32_t)b;
    BMat Ab = batch_view(A, b), Bb = batch_view(B, b);
    if constexpr (VIEWS) {
        const int64_t node = b / 7;
        const int t = (int)(b % 7);
        if (v.qa[t]) {
            Ab = quadrant_view(v.Ap, node, v.qa[t], m, l);
            ma = &ops.ap;
            ax = (int32_t)(((v.qa[t] - 1) & 1) * l);
            ay = (int32_t)(((v.qa[t] - 1) >> 1) * m);
            aw = (int32_t)node;
        }
        if (v.qb[t]) {
            Bb = quadrant_view(v.Bp, node, v.qb[t], l, n);
            mb = &ops.bp;
            bx = (int32_t)(((v.qb[t] - 1) & 1) * n);
            by = (int32_t)(((v.qb[t] - 1) >> 1) * l);
            bw = (int32_t)node;
        }
    }
    const int tx = threadIdx.x % BN, ty = threadIdx.x / BN;
    const int64_t i = tm * BM + ty, j = tn * BN + tx;
    const bool valid = (i < m) && (j < n);
    const int nch = (int)((l + BK - 1) / BK);
    const uint32_t bytes = (uint32_t)((NB + NA) * L * 8);

    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::mbar_fence_init();
    }
    // limb planes the copies do not write stay zero
    const int zb = (LM - L) * NB, za = (LM - L) * NA;
    for (int e = threadIdx.x; e < 2 * zb; e += NT) sB[(e / zb) * LM * NB + L * NB + e % zb] = 0ull;
    for (int e = threadIdx.x; e < 2 * za; e += NT) sA[(e / za) * LM * NA + L * NA + e % za] = 0ull;
    // exponents and signs of chunk ch into stage sg (zero exponent outside)
    auto stage_es = [&](int ch, int sg) {
        const int64_t k0 = (int64_t)ch * BK;
        for (int e = threadIdx.x; e < NB + NA; e += NT) {
            if (e < NB) {
                const int kk = e / BN, cc = e % BN;
                const int64_t gk = k0 + kk, gj = tn * BN + cc;
                const bool ok = gk < l && gj < n;
                sBe[sg * NB + e] = ok ? __ldg(Bb.exp + gk * Bb.ld + gj) : EXP_ZERO;
                sBs[sg * NB + e] = ok ? __ldg(Bb.sign + gk * Bb.ld + gj) : (int8_t)0;
            } else {
                const int f = e - NB, rr = f / BK, kk = f % BK;
                const int64_t gi = tm * BM + rr, gk = k0 + kk;
                const bool ok = gi < m && gk < l;
                sAe[sg * NA + f] = ok ? __ldg(Ab.exp + gi * Ab.ld + gk) : EXP_ZERO;
                sAs[sg * NA + f] = ok ? __ldg(Ab.sign + gi * Ab.ld + gk) : (int8_t)0;
            }
        }
    };
    // limb tiles of chunk ch into stage sg (one thread)
    auto issue = [&](int ch, int sg) {
        const int32_t k0 = ch * BK;
        tc::mbar_expect_tx(&bar[sg], bytes);
        tc::tma_load_4d(sB + sg * LM * NB, mb, bx + (int32_t)(tn * BN), by + k0, 0, bw, &bar[sg]);
        tc::tma_load_4d(sA + sg * LM * NA, ma, ax + k0, ay + (int32_t)(tm * BM), 0, aw, &bar[sg]);
    };
    stage_es(0, 0);
    __syncthreads();
    if (nch > 0 && threadIdx.x == 0) issue(0, 0);

    Mp<W> c, t;
    set_zero<W>(c, 0u);
    for (int ch = 0; ch < nch; ++ch) {
        const int sg = ch & 1;
        const bool more = ch + 1 < nch;
        if (more) {
            if (threadIdx.x == 0) issue(ch + 1, sg ^ 1);   // that stage was released by the last barrier
            stage_es(ch + 1, sg ^ 1);
        }
        const bool got = tc::mbar_wait(&bar[sg], (uint32_t)(ch >> 1) & 1u, nullptr, TMA_WAIT_LIMIT);
        if (got && valid) {
            const int kc = (int)((l - (int64_t)ch * BK) < BK ? (l - (int64_t)ch * BK) : BK);
            const uint64_t *pa = sA + sg * LM * NA + ty * BK;
            const uint64_t *pb = sB + sg * LM * NB + tx;
            const int64_t *ae = sAe + sg * NA + ty * BK, *be = sBe + sg * NB + tx;
            const int8_t *as = sAs + sg * NA + ty * BK, *bs = sBs + sg * NB + tx;
            for (int kk = 0; kk < kc; ++kk) {
                uint32_t am[W];
                PlaneWords<W>{pa + kk, NA}.load(am);
                mul_sm<W>(t, am, ae[kk], (uint32_t)(as[kk] & 1), PlaneWords<W>{pb + kk * BN, NB}, be[kk * BN],
                          (uint32_t)(bs[kk * BN] & 1), rs);
                add_impl<W>(c, c, t, 0u, rs);
            }
        }
        if (__syncthreads_or(!got)) {
            // a copy that did not complete in time: report it, give the
            // copies still in flight their chance to land, and stop
            if (threadIdx.x == 0) {
                flag(status, ST_TIMEOUT);
                tc::mbar_wait(&bar[sg], (uint32_t)(ch >> 1) & 1u, nullptr, TMA_WAIT_LIMIT);
                if (more) tc::mbar_wait(&bar[sg ^ 1], (uint32_t)((ch + 1) >> 1) & 1u, nullptr, TMA_WAIT_LIMIT);
            }
            __syncthreads();
            return;
        }
    }
    if (valid && st<W>(c, C, b, i, j, L)) flag(status, ST_RANGE);
}

// ------------------------------------------- recursion: operand sums (Sec. 2)
// Thread per (node, r < h, c < k).  Quadrant reads outside the parent's real
// m x l are zero (padding); the even part never reaches a peeled last row
// or column.  Children of node b are written at 7b + t, t = product index.
template <int W>
__global__ void operands_a_kernel(int algo, BMat P, BMat Ch, int64_t nodes, int64_t m,
                                  int64_t l, int64_t h, int64_t k, int p, int skip_plain)
{
    const bool cp = !skip_plain;           // write the plain-quadrant children
    const RoundSpec rs = make_spec<W>(p);
    const int64_t total = nodes * h * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t % k, r = (t / k) % h, b = t / (h * k);
        Mp<W> a11, a12, a21, a22, x, y;
        ld_or_zero<W>(a11, r < m && c < l, P, b, r, c, rs.L);
        ld_or_zero<W>(a12, r < m && c + k < l, P, b, r, c + k, rs.L);
        ld_or_zero<W>(a21, r + h < m && c < l, P, b, r + h, c, rs.L);
        ld_or_zero<W>(a22, r + h < m && c + k < l, P, b, r + h, c + k, rs.L);
        const int64_t cb = 7 * b;
        if (algo == 2) {   // Strassen: left operands of P1..P7
            add<W>(x, a11, a22, 0u, rs); st<W>(x, Ch, cb + 0, r, c, rs.L);   // A11 + A22
            add<W>(x, a21, a22, 0u, rs); st<W>(x, Ch, cb + 1, r, c, rs.L);   // A21 + A22
            if (cp) st<W>(a11, Ch, cb + 2, r, c, rs.L);                      // A11
            if (cp) st<W>(a22, Ch, cb + 3, r, c, rs.L);                      // A22
            add<W>(x, a11, a12, 0u, rs); st<W>(x, Ch, cb + 4, r, c, rs.L);   // A11 + A12
            add<W>(x, a21, a11, 1u, rs); st<W>(x, Ch, cb + 5, r, c, rs.L);   // A21 - A11
            add<W>(x, a12, a22, 1u, rs); st<W>(x, Ch, cb + 6, r, c, rs.L);   // A12 - A22
        } else {           // Winograd: left operands of M1..M7
            add<W>(x, a21, a22, 0u, rs);                                     // S1 = A21 + A22
            add<W>(y, x, a11, 1u, rs);                                       // S2 = S1 - A11
            st<W>(y, Ch, cb + 0, r, c, rs.L);                                // M1: S2
            if (cp) st<W>(a11, Ch, cb + 1, r, c, rs.L);                      // M2: A11
            if (cp) st<W>(a12, Ch, cb + 2, r, c, rs.L);                      // M3: A12
            st<W>(x, Ch, cb + 4, r, c, rs.L);                                // M5: S1
            add<W>(x, a12, y, 1u, rs);                                       // S4 = A12 - S2
            st<W>(x, Ch, cb + 5, r, c, rs.L);                                // M6: S4
            add<W>(x, a11, a21, 1u, rs);                                     // S3 = A11 - A21
            st<W>(x, Ch, cb + 3, r, c, rs.L);                                // M4: S3
            if (cp) st<W>(a22, Ch, cb + 6, r, c, rs.L);                      // M7: A22
        }
    }
}

template <int W>
__global__ void operands_b_kernel(int algo, BMat P, BMat Ch, int64_t nodes, int64_t l,
                                  int64_t n, int64_t k, int64_t w, int p, int skip_plain)
{
    const bool cp = !skip_plain;           // write the plain-quadrant children
    const RoundSpec rs = make_spec<W>(p);
    const int64_t total = nodes * k * w;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t % w, r = (t / w) % k, b = t / (k * w);
        Mp<W> b11, b12, b21, b22, x, y;
        ld_or_zero<W>(b11, r < l && c < n, P, b, r, c, rs.L);
        ld_or_zero<W>(b12, r < l && c + w < n, P, b, r, c + w, rs.L);
        ld_or_zero<W>(b21, r + k < l && c < n, P, b, r + k, c, rs.L);
        ld_or_zero<W>(b22, r + k < l && c + w < n, P, b, r + k, c + w, rs.L);
        const int64_t cb = 7 * b;
        if (algo == 2) {   // Strassen: right operands of P1..P7
            add<W>(x, b11, b22, 0u, rs); st<W>(x, Ch, cb + 0, r, c, rs.L);   // B11 + B22
            if (cp) st<W>(b11, Ch, cb + 1, r, c, rs.L);                      // B11
            add<W>(x, b12, b22, 1u, rs); st<W>(x, Ch, cb + 2, r, c, rs.L);   // B12 - B22
            add<W>(x, b21, b11, 1u, rs); st<W>(x, Ch, cb + 3, r, c, rs.L);   // B21 - B11
            if (cp) st<W>(b22, Ch, cb + 4, r, c, rs.L);                      // B22
            add<W>(x, b11, b12, 0u, rs); st<W>(x, Ch, cb + 5, r, c, rs.L);   // B11 + B12
            add<W>(x, b21, b22, 0u, rs); st<W>(x, Ch, cb + 6, r, c, rs.L);   // B21 + B22
        } else {           // Winograd: right operands of M1..M7
            add<W>(x, b12, b11, 1u, rs);                                     // S5 = B12 - B11
            st<W>(x, Ch, cb + 4, r, c, rs.L);                                // M5: S5
            add<W>(y, b22, x, 1u, rs);                                       // S6 = B22 - S5
            st<W>(y, Ch, cb + 0, r, c, rs.L);                                // M1: S6
            add<W>(x, y, b21, 1u, rs);                                       // S8 = S6 - B21
            st<W>(x, Ch, cb + 6, r, c, rs.L);                                // M7: S8
            add<W>(x, b22, b12, 1u, rs);                                     // S7 = B22 - B12
            st<W>(x, Ch, cb + 3, r, c, rs.L);                                // M4: S7
            if (cp) st<W>(b11, Ch, cb + 1, r, c, rs.L);                      // M2: B11
            if (cp) st<W>(b21, Ch, cb + 2, r, c, rs.L);                      // M3: B21
            if (cp) st<W>(b22, Ch, cb + 5, r, c, rs.L);                      // M6: B22
        }
    }
}

// ------------------------------------------- recursion: C combination (Sec. 2)
template <int W>
__global__ void combine_kernel(int algo, BMat Ch, BMat C, int64_t nodes, int64_t h, int64_t w,
                               int64_t mr, int64_t nr, int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t total = nodes * h * w;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t % w, r = (t / w) % h, b = t / (h * w);
        const int64_t cb = 7 * b;
        const bool lo_r = r < mr, hi_r = r + h < mr, lo_c = c < nr, hi_c = c + w < nr;
        Mp<W> x, y, z, u;
        if (algo == 2) {
            // C11 = P1 + P4 - P5 + P7 ; C12 = P3 + P5 ; C21 = P2 + P4 ; C22 = P1 + P3 - P2 + P6
            Mp<W> p1, p4;
            ld<W>(p1, Ch, cb + 0, r, c, rs.L);
            ld<W>(p4, Ch, cb + 3, r, c, rs.L);
            if (lo_r && lo_c) {
                ld<W>(y, Ch, cb + 4, r, c, rs.L);
                add<W>(x, p1, p4, 0u, rs);
                add<W>(x, x, y, 1u, rs);
                ld<W>(y, Ch, cb + 6, r, c, rs.L);
                add<W>(x, x, y, 0u, rs);
                bad |= st<W>(x, C, b, r, c, rs.L);
            }
            if (lo_r && hi_c) {
                ld<W>(x, Ch, cb + 2, r, c, rs.L);
                ld<W>(y, Ch, cb + 4, r, c, rs.L);
                add<W>(x, x, y, 0u, rs);
                bad |= st<W>(x, C, b, r, c + w, rs.L);
            }
            if (hi_r && lo_c) {
                ld<W>(x, Ch, cb + 1, r, c, rs.L);
                add<W>(x, x, p4, 0u, rs);
                bad |= st<W>(x, C, b, r + h, c, rs.L);
            }
            if (hi_r && hi_c) {
                ld<W>(y, Ch, cb + 2, r, c, rs.L);
                add<W>(x, p1, y, 0u, rs);
                ld<W>(y, Ch, cb + 1, r, c, rs.L);
                add<W>(x, x, y, 1u, rs);
                ld<W>(y, Ch, cb + 5, r, c, rs.L);
                add<W>(x, x, y, 0u, rs);
                bad |= st<W>(x, C, b + 0, r + h, c + w, rs.L);
            }
        } else {
            // T1 = M1 + M2 ; T2 = T1 + M4 ; C11 = M2 + M3 ; C12 = T1 + M5 + M6 ;
            // C21 = T2 - M7 ; C22 = T2 + M5
            Mp<W> m2, t1, t2, m5;
            ld<W>(x, Ch, cb + 0, r, c, rs.L);
            ld<W>(m2, Ch, cb + 1, r, c, rs.L);
            add<W>(t1, x, m2, 0u, rs);
            ld<W>(x, Ch, cb + 3, r, c, rs.L);
            add<W>(t2, t1, x, 0u, rs);
            ld<W>(m5, Ch, cb + 4, r, c, rs.L);
            if (lo_r && lo_c) {
                ld<W>(x, Ch, cb + 2, r, c, rs.L);
                add<W>(z, m2, x, 0u, rs);
                bad |= st<W>(z, C, b, r, c, rs.L);
            }
            if (lo_r && hi_c) {
                add<W>(z, t1, m5, 0u, rs);
                ld<W>(x, Ch, cb + 5, r, c, rs.L);
                add<W>(z, z, x, 0u, rs);
                bad |= st<W>(z, C, b, r, c + w, rs.L);
            }
            if (hi_r && lo_c) {
                ld<W>(x, Ch, cb + 6, r, c, rs.L);
                add<W>(u, t2, x, 1u, rs);
                bad |= st<W>(u, C, b, r + h, c, rs.L);
            }
            if (hi_r && hi_c) {
                add<W>(u, t2, m5, 0u, rs);
                bad |= st<W>(u, C, b, r + h, c + w, rs.L);
            }
        }
    }
    if (bad) flag(status, ST_RANGE);
}

// ------------------------------------------------- recursion: peel fix-ups
// l peeled: c_ij = RN(c_ij + RN(a_{i,l-1} b_{l-1,j})) on the recursive part
template <int W>
__global__ void rank1_kernel(BMat A, BMat B, BMat C, int64_t nodes, int64_t mr, int64_t nr,
                             int64_t l, int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t total = nodes * mr * nr;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t % nr, r = (t / nr) % mr, b = t / (mr * nr);
        Mp<W> x, a, bb, y;
        ld_rw<W>(x, C, b, r, c, rs.L);
        ld<W>(a, A, b, r, l - 1, rs.L);
        ld<W>(bb, B, b, l - 1, c, rs.L);
        mul<W>(y, a, bb, rs);
        add<W>(x, x, y, 0u, rs);
        bad |= st<W>(x, C, b, r, c, rs.L);
    }
    if (bad) flag(status, ST_RANGE);
}

// m peeled: last row by Simple over the whole l; n peeled: last column
// (rows < mr) likewise.  Thread per output element.
template <int W>
__global__ void border_kernel(BMat A, BMat B, BMat C, int64_t nodes, int64_t m, int64_t l,
                              int64_t n, int64_t mr, int last_row, int last_col, int p,
                              DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t per = (last_row ? n : 0) + (last_col ? mr : 0);
    const int64_t total = nodes * per;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / per, q = t % per;
        int64_t i, j;
        if (last_row && q < n) { i = m - 1; j = q; }
        else { i = q - (last_row ? n : 0); j = n - 1; }
        Mp<W> c, a, bb, y;
        set_zero<W>(c, 0u);
        for (int64_t k = 0; k < l; ++k) {
            ld<W>(a, A, b, i, k, rs.L);
            ld<W>(bb, B, b, k, j, rs.L);
            mul<W>(y, a, bb, rs);
            add<W>(c, c, y, 0u, rs);
        }
        bad |= st<W>(c, C, b, i, j, rs.L);
    }
    if (bad) flag(status, ST_RANGE);
}

// ================================================================ launchers
inline int grid_for(int64_t total, int threads)
{
    int64_t g = (total + threads - 1) / threads;
    const int64_t cap = 152 * 64;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <int W>
void launch_elementwise(int op, BMat X, BMat Y, BMat R, int64_t rows, int64_t cols, int p,
                        DevStatus *st, cudaStream_t s)
{
    const int64_t total = rows * cols;
    if (total <= 0) return;
    elementwise_kernel<W><<<grid_for(total, 128), 128, 0, s>>>(op, X, Y, R, rows, cols, p, st);
}

template <int W>
void launch_convert(BMat X, int px, BMat R, int pr, int64_t rows, int64_t cols, DevStatus *st,
                    cudaStream_t s)
{
    const int64_t total = rows * cols;
    if (total <= 0) return;
    convert_kernel<W><<<grid_for(total, 128), 128, 0, s>>>(X, px, R, pr, rows, cols, st);
}

template <int W>
void launch_gemm_simple(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p,
                        DevStatus *st, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return;
    constexpr int ty = SimpleCfg<W>::TY;
    dim3 block(32, ty);
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + ty - 1) / ty));
    gemm_simple_kernel<W><<<grid, block, 0, s>>>(A, B, C, m, l, n, p, st);
}

// the TMA-staged leaf over a batch (VIEWS: with in-place quadrants)
template <int W, bool VIEWS>
bool launch_block_tma(const TmaOps &ops, BMat A, BMat B, BMat C, const LeafViews &v, int64_t batch, int64_t m,
                      int64_t l, int64_t n, int p, DevStatus *st, cudaStream_t s)
{
    using Cfg = BlockTmaCfg<W>;
    static std::once_flag once;                      // one GPU per process
    static bool ready = false;
    std::call_once(once, [] {
        ready = cudaFuncSetAttribute(gemm_block_tma_kernel<W, VIEWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Cfg::smem()) == cudaSuccess;
        if (!ready) cudaGetLastError();
    });
    if (!ready) return false;
    const int64_t tm = (m + Cfg::BM - 1) / Cfg::BM, tn = (n + Cfg::BN - 1) / Cfg::BN;
    gemm_block_tma_kernel<W, VIEWS><<<(unsigned)(batch * tm * tn), Cfg::THREADS, Cfg::smem(), s>>>(
        ops, A, B, C, v, m, l, n, p, tm, tn, st);
    return true;
}

template <int W>
bool launch_gemm_block(BMat A, BMat B, BMat C, int64_t batch, int64_t m, int64_t l, int64_t n,
                       int p, DevStatus *st, cudaStream_t s, bool tma)
{
    if (batch <= 0 || m <= 0 || n <= 0) return false;
    if constexpr (W <= TMA_MAX_W) {
        if (tma) {
            using Cfg = BlockTmaCfg<W>;
            const int L = (p + 63) / 64;
            TmaOps ops;
            memset(&ops, 0, sizeof(ops));
            LeafViews none;
            memset(&none, 0, sizeof(none));
            if (limb_map(&ops.a, A, batch, m, l, L, Cfg::BK, Cfg::BM) &&
                limb_map(&ops.b, B, batch, l, n, L, Cfg::BN, Cfg::BK) &&
                launch_block_tma<W, false>(ops, A, B, C, none, batch, m, l, n, p, st, s))
                return true;
        }
    }
    if constexpr (is_big<W>()) {
        // wide class: the batched Simple kernel, up to 65535 products a launch
        constexpr int ty = SimpleCfg<W>::TY;
        for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
            const int64_t nb = batch - b0 < 65535 ? batch - b0 : 65535;
            BMat Ab = A, Bb = B, Cb = C;
            Ab.limb += b0 * A.bs_limb; Ab.exp += b0 * A.bs_es; Ab.sign += b0 * A.bs_es;
            Bb.limb += b0 * B.bs_limb; Bb.exp += b0 * B.bs_es; Bb.sign += b0 * B.bs_es;
            Cb.limb += b0 * C.bs_limb; Cb.exp += b0 * C.bs_es; Cb.sign += b0 * C.bs_es;
            dim3 block(32, ty);
            dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + ty - 1) / ty), (unsigned)nb);
            gemm_simple_kernel<W, true><<<grid, block, 0, s>>>(Ab, Bb, Cb, m, l, n, p, st);
        }
    } else {
        using Cfg = BlockSmCfg<W>;
        const int64_t tm = (m + Cfg::BM - 1) / Cfg::BM, tn = (n + Cfg::BN - 1) / Cfg::BN;
        static std::once_flag once;                  // one GPU per process
        std::call_once(once, [] {
            cudaFuncSetAttribute(gemm_block_sm_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg::smem());
        });
        gemm_block_sm_kernel<W><<<(unsigned)(batch * tm * tn), Cfg::THREADS, Cfg::smem(), s>>>(
            A, B, C, m, l, n, p, tm, tn, st);
    }
    return false;
}

// The batches of grp (one precision, at most LEAF_GROUP_MAX) in one launch;
// the tile counts and first[] are filled in here.  Narrow classes only.
template <int W>
void launch_gemm_block_group(LeafGroup grp, int p, DevStatus *st, cudaStream_t s)
{
    if constexpr (is_big<W>()) {
        for (int g = 0; g < grp.count; ++g) {
            const LeafBatch &lb = grp.batch[g];
            launch_gemm_block<W>(lb.A, lb.B, lb.C, lb.batch, lb.m, lb.l, lb.n, p, st, s);
        }
    } else {
        using Cfg = BlockSmCfg<W>;
        int64_t total = 0;
        for (int g = 0; g < grp.count; ++g) {
            LeafBatch &lb = grp.batch[g];
            lb.tiles_m = (lb.m + Cfg::BM - 1) / Cfg::BM;
            lb.tiles_n = (lb.n + Cfg::BN - 1) / Cfg::BN;
            grp.first[g] = total;
            if (lb.m > 0 && lb.n > 0) total += lb.batch * lb.tiles_m * lb.tiles_n;
        }
        grp.first[grp.count] = total;
        if (total <= 0) return;
        static std::once_flag once;                  // one GPU per process
        std::call_once(once, [] {
            cudaFuncSetAttribute(gemm_block_group_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg::smem());
        });
        gemm_block_group_kernel<W><<<(unsigned)total, Cfg::THREADS, Cfg::smem(), s>>>(grp, p, st);
    }
}

// C := C - A B with every element's products subtracted one by one,
// k ascending (one product, not batched)
template <int W>
void launch_gemm_sub(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p,
                     DevStatus *st, cudaStream_t s)
{
    if (m <= 0 || n <= 0 || l <= 0) return;
    if constexpr (is_big<W>()) {
        constexpr int ty = SimpleCfg<W>::TY;
        dim3 block(32, ty);
        dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + ty - 1) / ty));
        gemm_simple_kernel<W, false, true><<<grid, block, 0, s>>>(A, B, C, m, l, n, p, st);
    } else {
        using Cfg = BlockSmCfg<W>;
        const int64_t tm = (m + Cfg::BM - 1) / Cfg::BM, tn = (n + Cfg::BN - 1) / Cfg::BN;
        static std::once_flag once;                  // one GPU per process
        std::call_once(once, [] {
            cudaFuncSetAttribute(gemm_block_sm_kernel<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg::smem());
        });
        gemm_block_sm_kernel<W, true><<<(unsigned)(tm * tn), Cfg::THREADS, Cfg::smem(), s>>>(
            A, B, C, m, l, n, p, tm, tn, st);
    }
}

template <int W>
void launch_operands_a(int algo, BMat P, BMat Ch, int64_t nodes, int64_t m, int64_t l,
                       int64_t h, int64_t k, int p, cudaStream_t s, bool skip_plain)
{
    const int64_t total = nodes * h * k;
    if (total <= 0) return;
    operands_a_kernel<W><<<grid_for(total, 128), 128, 0, s>>>(algo, P, Ch, nodes, m, l, h, k, p, skip_plain ? 1 : 0);
}

template <int W>
void launch_operands_b(int algo, BMat P, BMat Ch, int64_t nodes, int64_t l, int64_t n,
                       int64_t k, int64_t w, int p, cudaStream_t s, bool skip_plain)
{
    const int64_t total = nodes * k * w;
    if (total <= 0) return;
    operands_b_kernel<W><<<grid_for(total, 128), 128, 0, s>>>(algo, P, Ch, nodes, l, n, k, w, p, skip_plain ? 1 : 0);
}

template <int W>
bool launch_gemm_leaf_views(BMat A, BMat B, BMat C, const LeafViews &v, int64_t batch, int64_t m, int64_t l,
                            int64_t n, int p, DevStatus *st, cudaStream_t s, bool tma)
{
    if (batch <= 0 || m <= 0 || n <= 0) return false;
    if constexpr (W <= TMA_MAX_W) {
        if (tma) {
            // a quadrant in the right half starts l (A) or n (B) columns in:
            // the copies need that offset a whole number of 16-byte units
            bool odd_x = false;
            for (int t = 0; t < 7; ++t) {
                if ((v.qa[t] == 2 || v.qa[t] == 4) && (l & 1)) odd_x = true;
                if ((v.qb[t] == 2 || v.qb[t] == 4) && (n & 1)) odd_x = true;
            }
            using Cfg = BlockTmaCfg<W>;
            const int L = (p + 63) / 64;
            TmaOps ops;
            memset(&ops, 0, sizeof(ops));
            if (!odd_x && limb_map(&ops.a, A, batch, m, l, L, Cfg::BK, Cfg::BM) &&
                limb_map(&ops.b, B, batch, l, n, L, Cfg::BN, Cfg::BK) &&
                limb_map(&ops.ap, v.Ap, v.nodes, v.a_rows, v.a_cols, L, Cfg::BK, Cfg::BM) &&
                limb_map(&ops.bp, v.Bp, v.nodes, v.b_rows, v.b_cols, L, Cfg::BN, Cfg::BK) &&
                launch_block_tma<W, true>(ops, A, B, C, v, batch, m, l, n, p, st, s))
                return true;
        }
    }
    if constexpr (is_big<W>()) {
        return false;                                // not used: the wide class materialises its children
    } else {
        using Cfg = BlockSmCfg<W>;
        const int64_t tm = (m + Cfg::BM - 1) / Cfg::BM, tn = (n + Cfg::BN - 1) / Cfg::BN;
        static std::once_flag once;                  // one GPU per process
        std::call_once(once, [] {
            cudaFuncSetAttribute(gemm_block_leaf_views_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg::smem());
        });
        gemm_block_leaf_views_kernel<W><<<(unsigned)(batch * tm * tn), Cfg::THREADS, Cfg::smem(), s>>>(
            A, B, C, v, m, l, n, p, tm, tn, st);
    }
    return false;
}

template <int W>
void launch_combine(int algo, BMat Ch, BMat C, int64_t nodes, int64_t h, int64_t w, int64_t mr,
                    int64_t nr, int p, DevStatus *st, cudaStream_t s)
{
    const int64_t total = nodes * h * w;
    if (total <= 0) return;
    combine_kernel<W><<<grid_for(total, 128), 128, 0, s>>>(algo, Ch, C, nodes, h, w, mr, nr, p, st);
}

template <int W>
void launch_rank1(BMat A, BMat B, BMat C, int64_t nodes, int64_t mr, int64_t nr, int64_t l,
                  int p, DevStatus *st, cudaStream_t s)
{
    const int64_t total = nodes * mr * nr;
    if (total <= 0) return;
    rank1_kernel<W><<<grid_for(total, 128), 128, 0, s>>>(A, B, C, nodes, mr, nr, l, p, st);
}

template <int W>
void launch_border(BMat A, BMat B, BMat C, int64_t nodes, int64_t m, int64_t l, int64_t n,
                   int64_t mr, bool last_row, bool last_col, int p, DevStatus *st,
                   cudaStream_t s)
{
    const int64_t per = (last_row ? n : 0) + (last_col ? mr : 0);
    const int64_t total = nodes * per;
    if (total <= 0) return;
    border_kernel<W><<<grid_for(total, 64), 64, 0, s>>>(A, B, C, nodes, m, l, n, mr,
                                                         last_row ? 1 : 0, last_col ? 1 : 0, p, st);
}

#define MPG_INSTANTIATE_GEMM(W)                                                                 \
    template void launch_elementwise<W>(int, BMat, BMat, BMat, int64_t, int64_t, int,           \
                                        DevStatus *, cudaStream_t);                             \
    template void launch_convert<W>(BMat, int, BMat, int, int64_t, int64_t, DevStatus *,        \
                                    cudaStream_t);                                              \
    template void launch_gemm_simple<W>(BMat, BMat, BMat, int64_t, int64_t, int64_t, int,       \
                                        DevStatus *, cudaStream_t);                             \
    template bool launch_gemm_block<W>(BMat, BMat, BMat, int64_t, int64_t, int64_t, int64_t,    \
                                       int, DevStatus *, cudaStream_t, bool);                   \
    template void launch_gemm_sub<W>(BMat, BMat, BMat, int64_t, int64_t, int64_t, int,          \
                                     DevStatus *, cudaStream_t);                                \
    template void launch_gemm_block_group<W>(LeafGroup, int, DevStatus *, cudaStream_t);        \
    template void launch_rank1<W>(BMat, BMat, BMat, int64_t, int64_t, int64_t, int64_t, int,    \
                                  DevStatus *, cudaStream_t);                                   \
    template void launch_border<W>(BMat, BMat, BMat, int64_t, int64_t, int64_t, int64_t,        \
                                   int64_t, bool, bool, int, DevStatus *, cudaStream_t);

#define MPG_INSTANTIATE_REC(W)                                                                  \
    template void launch_operands_a<W>(int, BMat, BMat, int64_t, int64_t, int64_t, int64_t,     \
                                       int64_t, int, cudaStream_t, bool);                       \
    template void launch_operands_b<W>(int, BMat, BMat, int64_t, int64_t, int64_t, int64_t,     \
                                       int64_t, int, cudaStream_t, bool);                       \
    template bool launch_gemm_leaf_views<W>(BMat, BMat, BMat, const LeafViews &, int64_t, int64_t, \
                                            int64_t, int64_t, int, DevStatus *, cudaStream_t,   \
                                            bool);                                              \
    template void launch_combine<W>(int, BMat, BMat, int64_t, int64_t, int64_t, int64_t,        \
                                    int64_t, int, DevStatus *, cudaStream_t);

}  // namespace mpg
