// mp_lu.cuh -- kernels of the blocked right-looking LU with partial pivoting
// and the triangular solves (arXiv 1410.1599 Sec. 4), one instantiation per
// word-capacity class W (lu_w*.cu).
#pragma once
#include "mp_warp.cuh"

namespace mpg {

// threads of the single-CTA pivot kernel: fewer for wide numbers,
// so each thread keeps its operands in registers
template <int W> struct LuCfg {
    static constexpr int PIVOT = (W <= 8) ? 512 : 256;
};

// |x| > |y| on loaded numbers (zero is the smallest magnitude)
template <int W>
MP_DEV bool absgreater(const Mp<W> &x, const Mp<W> &y)
{
    return cmpabs<W>(x, y) > 0;
}

// One CTA: pivot = first row i in [k, iend) of largest |a_ik| (iend = n
// with partial pivoting, k + 1 for the paper's unpivoted LU); record it, then
// exchange rows k and pivot over the columns [c0, c1) (all n, or the panel
// when the other columns are exchanged later by lu_laswp_kernel).  A zero
// pivot column is recorded (smallest such column wins) and nothing is
// exchanged.
//
// Each thread finds the first largest of its rows by full comparison.  The
// block then reduces the key (exponent, top 64 mantissa bits), which orders
// magnitudes except between numbers that agree in the key; the threads whose
// candidate carries the largest key list it, and one thread settles the list
// (usually one entry) by full comparison, lower row first among equals.
template <int W>
__global__ void __launch_bounds__(LuCfg<W>::PIVOT) lu_pivot_kernel(BMat A, int64_t iend, int64_t k, int64_t *piv,
                                                        int p, DevStatus *status, int64_t c0, int64_t c1)
{
    constexpr int NT = LuCfg<W>::PIVOT, NW = NT / 32;
    const RoundSpec rs = make_spec<W>(p);
    __shared__ int64_t s_row[NT];
    __shared__ int64_t s_we[NW];
    __shared__ uint64_t s_wm[NW];
    __shared__ int s_nc;
    __shared__ int64_t s_best;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int64_t best = -1;
    Mp<W> bx, x;
    set_zero<W>(bx, 0u);
    for (int64_t i = k + tid; i < iend; i += NT) {
        ld_rw<W>(x, A, 0, i, k, rs.L);
        if (best < 0 || absgreater<W>(x, bx)) {
            best = i;
            bx = x;
        }
    }
    if (tid == 0) s_nc = 0;
    // key of this thread's candidate (no candidate or zero: smallest key)
    const int64_t ke = (best < 0) ? EXP_ZERO : bx.e;
    const uint64_t km = (best < 0 || bx.e == EXP_ZERO)
                            ? 0ull : (((uint64_t)bx.m[W - 1] << 32) | bx.m[W - 2]);
    int64_t me = ke;
    uint64_t mm = km;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t oe = __shfl_xor_sync(0xffffffffu, me, o);
        const uint64_t om = __shfl_xor_sync(0xffffffffu, mm, o);
        if (oe > me || (oe == me && om > mm)) { me = oe; mm = om; }
    }
    if (lane == 0) { s_we[wid] = me; s_wm[wid] = mm; }
    __syncthreads();
    me = s_we[0];
    mm = s_wm[0];
    for (int w = 1; w < NW; ++w)
        if (s_we[w] > me || (s_we[w] == me && s_wm[w] > mm)) { me = s_we[w]; mm = s_wm[w]; }
    if (best >= 0 && ke == me && km == mm) s_row[atomicAdd(&s_nc, 1)] = best;
    __syncthreads();
    if (tid == 0) {
        int64_t pr = k;
        if (s_nc > 0) {
            pr = s_row[0];
            Mp<W> xa, xb;
            ld_rw<W>(xa, A, 0, pr, k, rs.L);
            for (int c = 1; c < s_nc; ++c) {
                const int64_t rb = s_row[c];
                ld_rw<W>(xb, A, 0, rb, k, rs.L);
                const int cmp = cmpabs<W>(xb, xa);
                if (cmp > 0 || (cmp == 0 && rb < pr)) { pr = rb; xa = xb; }
            }
        }
        Mp<W> v;
        ld_rw<W>(v, A, 0, pr, k, rs.L);
        piv[k] = pr;
        if (v.e == EXP_ZERO) {
            atomicOr(&status->flags, ST_SINGULAR);
            atomicMin(&status->singular_col, (long long)k);
            s_best = k;   // no exchange
        } else {
            s_best = pr;
        }
    }
    __syncthreads();
    const int64_t pr = s_best;
    if (pr == k) return;
    const int L = rs.L;
    for (int64_t c = c0 + tid; c < c1; c += NT) {
        for (int q = 0; q < L; ++q) {
            uint64_t *a = A.limb + (int64_t)q * A.plane + k * A.ld + c;
            uint64_t *b = A.limb + (int64_t)q * A.plane + pr * A.ld + c;
            const uint64_t t = *a;
            *a = *b;
            *b = t;
        }
        int64_t *ea = A.exp + k * A.ld + c, *eb = A.exp + pr * A.ld + c;
        const int64_t te = *ea;
        *ea = *eb;
        *eb = te;
        int8_t *sa = A.sign + k * A.ld + c, *sb = A.sign + pr * A.ld + c;
        const int8_t ts = *sa;
        *sa = *sb;
        *sb = ts;
    }
}

// l_ik = RN(a_ik / a_kk) for i in (k, n); a zero a_kk (already reported by
// the pivot step) leaves the column untouched.  Up to 1024 bits one warp
// forms each quotient (the division's latency is on the critical path of
// the factorisation); wider numbers take one thread per row.
template <int W>
__global__ void lu_divide_kernel(BMat A, int64_t n, int64_t k, int p)
{
    const RoundSpec rs = make_spec<W>(p);
    if constexpr (W <= 32) {
        const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
        int64_t de;
        uint32_t ds;
        const uint32_t dm = wld<W>(A, 0, k, k, rs.L, de, ds);
        if (de == EXP_ZERO) return;
        for (int64_t i = k + 1 + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; i < n;
             i += nwarps) {
            int64_t xe, qe;
            uint32_t xs, qs;
            const uint32_t xm = wld<W>(A, 0, i, k, rs.L, xe, xs);
            const uint32_t qm = warp_div<W>(xm, xe, xs, dm, de, ds, qe, qs, rs);
            wst<W>(qm, qe, qs, A, 0, i, k, rs.L);
        }
    } else {
        Mp<W> d, x, q;
        ld_rw<W>(d, A, 0, k, k, rs.L);
        if (d.e == EXP_ZERO) return;
        for (int64_t i = k + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            ld_rw<W>(x, A, 0, i, k, rs.L);
            div<W>(q, x, d, rs);
            st<W>(q, A, 0, i, k, rs.L);
        }
    }
}

// a_ij = RN(a_ij - RN(a_ik a_kj)) for i in [r0, r1), j in [c0, c1): one
// elimination step of the panel (column k) or of the U12 solve (row s = k)
template <int W>
__global__ void lu_rank1_kernel(BMat A, int64_t k, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                                int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t w = c1 - c0, total = (r1 - r0) * w;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r0 + t / w, j = c0 + t % w;
        Mp<W> l, u, y, z;
        ld_rw<W>(l, A, 0, i, k, rs.L);
        ld_rw<W>(u, A, 0, k, j, rs.L);
        ld_rw<W>(y, A, 0, i, j, rs.L);
        mul<W, true>(z, l, u, rs);
        add<W, true>(y, y, z, 1u, rs);
        bad |= st<W>(y, A, 0, i, j, rs.L);
    }
    if (bad) flag(status, ST_RANGE);
}

// ---------------------------------------------- fused column step (W <= 32)
// One launch per panel column k does what the pivot / divide / rank-1 kernels
// do in three: a warp per row i > k forms l_ik = RN(a_ik / a_kk) together,
// then its lanes update the row's panel columns k+1 .. je-1
// (a_ij = RN(a_ij - RN(l_ik a_kj))), lane 0 tracking the first largest
// |a_i,k+1| of the warp's rows.  Each CTA posts its candidate; the last CTA to
// finish (ticket counter, no waiting) picks the pivot of column k+1 among
// the posted rows and exchanges the two rows over the panel's columns, so
// the next launch starts on a pivoted column; the other columns take the
// panel's exchanges afterwards, in the same order (lu_laswp_kernel).  The
// operations and their order per element are the same as in the separate
// kernels.
constexpr int LU_COL_WARPS = 4;

// First row of largest |a_{r,col}| among the rows rows[0 .. cnt), ties to the
// lower row, by the NT threads of a CTA (key reduction as in lu_pivot_kernel,
// full comparison only among key ties).  Returns -1 when cnt == 0 or every
// listed row is negative.
// load through L2 only: the rows were written by other CTAs of this launch
template <int W>
MP_DEV void ld_cg(Mp<W> &x, const BMat &M, int64_t r, int64_t c, int L)
{
    const int64_t lo = lim_off(M, 0, r, c), eo = es_off(M, 0, r, c);
#pragma unroll
    for (int k = 0; k < W / 2; ++k) {
        const uint64_t v = (k < L) ? __ldcg(M.limb + lo + (int64_t)k * M.plane) : 0ull;
        x.m[W - 1 - 2 * k] = (uint32_t)(v >> 32);
        x.m[W - 2 - 2 * k] = (uint32_t)v;
    }
    x.e = __ldcg(M.exp + eo);
    x.s = (uint32_t)(__ldcg(M.sign + eo) & 1);
}

template <int W, int NT, class RowOf>
__device__ int64_t cta_pick_row(const BMat &A, int64_t col, int cnt, RowOf row_of, const RoundSpec &rs,
                                int64_t *s_list, int *s_nc, int64_t *s_we, uint64_t *s_wm)
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int64_t best = -1;
    Mp<W> bx, x;
    set_zero<W>(bx, 0u);
    for (int c = tid; c < cnt; c += NT) {
        const int64_t r = row_of(c);
        if (r < 0) continue;
        ld_cg<W>(x, A, r, col, rs.L);
        const int cmp = best < 0 ? 1 : cmpabs<W>(x, bx);
        if (cmp > 0 || (cmp == 0 && r < best)) {
            best = r;
            bx = x;
        }
    }
    if (tid == 0) *s_nc = 0;
    const int64_t ke = (best < 0) ? EXP_ZERO : bx.e;
    const uint64_t km = (best < 0 || bx.e == EXP_ZERO) ? 0ull : (((uint64_t)bx.m[W - 1] << 32) | bx.m[W - 2]);
    int64_t me = ke;
    uint64_t mm = km;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t oe = __shfl_xor_sync(0xffffffffu, me, o);
        const uint64_t om = __shfl_xor_sync(0xffffffffu, mm, o);
        if (oe > me || (oe == me && om > mm)) { me = oe; mm = om; }
    }
    if (lane == 0) { s_we[wid] = me; s_wm[wid] = mm; }
    __syncthreads();
    me = s_we[0];
    mm = s_wm[0];
    for (int w = 1; w < NW; ++w)
        if (s_we[w] > me || (s_we[w] == me && s_wm[w] > mm)) { me = s_we[w]; mm = s_wm[w]; }
    if (best >= 0 && ke == me && km == mm) s_list[atomicAdd(s_nc, 1)] = best;
    __syncthreads();
    int64_t pr = -1;
    if (tid == 0 && *s_nc > 0) {
        pr = s_list[0];
        Mp<W> xa, xb;
        ld_cg<W>(xa, A, pr, col, rs.L);
        for (int c = 1; c < *s_nc; ++c) {
            const int64_t rb = s_list[c];
            ld_cg<W>(xb, A, rb, col, rs.L);
            const int cmp = cmpabs<W>(xb, xa);
            if (cmp > 0 || (cmp == 0 && rb < pr)) { pr = rb; xa = xb; }
        }
    }
    return pr;    // meaningful in thread 0
}

// exchange rows r1 and r2 of A over the columns [c0, c1) (one CTA)
template <int W>
__device__ void cta_swap_rows(const BMat &A, int64_t c0, int64_t c1, int64_t r1, int64_t r2, int L)
{
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        for (int q = 0; q < L; ++q) {
            uint64_t *a = A.limb + (int64_t)q * A.plane + r1 * A.ld + c;
            uint64_t *b = A.limb + (int64_t)q * A.plane + r2 * A.ld + c;
            const uint64_t t = *a;
            *a = *b;
            *b = t;
        }
        int64_t *ea = A.exp + r1 * A.ld + c, *eb = A.exp + r2 * A.ld + c;
        const int64_t te = *ea;
        *ea = *eb;
        *eb = te;
        int8_t *sa = A.sign + r1 * A.ld + c, *sb = A.sign + r2 * A.ld + c;
        const int8_t ts = *sa;
        *sa = *sb;
        *sb = ts;
    }
}

// The row updates cover the columns k+1 .. ce-1 only (ce <= je, the end of
// the current sub-panel): every row below k is in the same state, so row
// exchanges keep the later columns' pending updates consistent.  Those
// columns take this step's update later, in the same order (the subtracting
// Block product for rows below the sub-panel, lu_u12_kernel for the
// sub-panel's own rows).  The next pivot is picked when k+1 < ce.
template <int W>
__global__ void __launch_bounds__(LU_COL_WARPS * 32)
lu_column_kernel(BMat A, int64_t n, int64_t j0, int64_t k, int64_t je, int64_t ce, int64_t *piv, int p,
                 DevStatus *status, int64_t *cand, unsigned *ticket, int pivoting)
{
    static_assert(W <= 32, "warp-per-row column step");
    constexpr int NT = LU_COL_WARPS * 32;
    const RoundSpec rs = make_spec<W>(p);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * LU_COL_WARPS;
    const bool next = k + 1 < ce;
    __shared__ int64_t s_list[NT];
    __shared__ int64_t s_we[LU_COL_WARPS];
    __shared__ uint64_t s_wm[LU_COL_WARPS];
    __shared__ int s_nc;
    __shared__ int s_last;
    __shared__ int64_t s_wrow[LU_COL_WARPS];
    int64_t de;
    uint32_t ds;
    const uint32_t dm = wld<W>(A, 0, k, k, rs.L, de, ds);
    int64_t best = -1;                      // lane 0: the warp's first largest |a_i,k+1|
    Mp<W> bx;
    set_zero<W>(bx, 0u);
    bool bad = false;
    for (int64_t i = k + 1 + (int64_t)blockIdx.x * LU_COL_WARPS + wid; i < n; i += nw) {
        int64_t qe;
        uint32_t qs;
        uint32_t qm = wld<W>(A, 0, i, k, rs.L, qe, qs);
        if (de != EXP_ZERO) {               // a zero pivot leaves the column as it is
            int64_t xe = qe;
            uint32_t xs = qs;
            qm = warp_div<W>(qm, xe, xs, dm, de, ds, qe, qs, rs);
            wst<W>(qm, qe, qs, A, 0, i, k, rs.L);
        }
        Mp<W> l;
#pragma unroll
        for (int w = 0; w < W; ++w) l.m[w] = __shfl_sync(0xffffffffu, qm, w);
        l.e = qe;
        l.s = qs;
        for (int64_t j = k + 1 + lane; j < ce; j += 32) {
            Mp<W> u, y, z;
            ld_rw<W>(u, A, 0, k, j, rs.L);
            ld_rw<W>(y, A, 0, i, j, rs.L);
            mul<W, true>(z, l, u, rs);
            add<W, true>(y, y, z, 1u, rs);
            bad |= st<W>(y, A, 0, i, j, rs.L);
            if (j == k + 1 && (pivoting || i == k + 1) && (best < 0 || absgreater<W>(y, bx))) {
                best = i;
                bx = y;
            }
        }
        __syncwarp();
    }
    if (bad) flag(status, ST_RANGE);
    if (!next) return;
    // this CTA's candidate for the pivot of column k+1
    if (lane == 0) s_wrow[wid] = best;
    __syncthreads();
    const int64_t cb = cta_pick_row<W, NT>(A, k + 1, LU_COL_WARPS, [&](int c) { return s_wrow[c]; }, rs,
                                           s_list, &s_nc, s_we, s_wm);
    if (threadIdx.x == 0) cand[blockIdx.x] = cb;
    // publish, then the last CTA to arrive picks among all candidates
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int cnt = (int)gridDim.x;
    const int64_t pr0 = cta_pick_row<W, NT>(A, k + 1, cnt, [&](int c) { return ((volatile int64_t *)cand)[c]; },
                                            rs, s_list, &s_nc, s_we, s_wm);
    __shared__ int64_t s_pr;
    if (threadIdx.x == 0) {
        const int64_t pr = pr0 < 0 ? k + 1 : pr0;
        Mp<W> v;
        ld_cg<W>(v, A, pr, k + 1, rs.L);
        piv[k + 1] = pr;
        if (v.e == EXP_ZERO) {
            atomicOr(&status->flags, ST_SINGULAR);
            atomicMin(&status->singular_col, (long long)(k + 1));
            s_pr = k + 1;
        } else {
            s_pr = pr;
        }
        *ticket = 0u;                       // ready for the next launch
    }
    __syncthreads();
    if (s_pr != k + 1) cta_swap_rows<W>(A, j0, je, k + 1, s_pr, rs.L);   // panel columns only
}

// ------------------------------------------- U12 = L11^-1 A12, one launch
// One CTA per column j in [je, cend) (grid-stride), thread t <-> panel row
// j0 + t (panels of at most 128 columns).  Row r is final after the steps
// s < r; it is then shared, and every row below takes
// a_ij = RN(a_ij - RN(l_ir a_rj)) -- per element the steps s = j0 .. i-1 in
// ascending order, as the row-step launches do.
// three CTAs (columns) per SM: at 1024 bits that caps the kernel at 168
// registers (a few spilled); the first panels' 640-896 columns then take two
// rounds instead of three.  With the row value read from shared memory as
// the product forms, the 1024-bit U12 time fell by 21 % (n = 1024) and 23 %
// (n = 2048) against registers and two CTAs per SM.
#ifndef MPG_U12_MINCTAS
#define MPG_U12_MINCTAS 3
#endif
template <int W>
__global__ void __launch_bounds__(128, MPG_U12_MINCTAS) lu_u12_kernel(BMat A, int64_t cend, int64_t j0, int64_t je, int p,
                                                     DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    __shared__ __align__(16) Mp<W> s_x;
    const int64_t i = j0 + threadIdx.x;
    const bool mine = i < je;
    bool bad = false;
    for (int64_t j = je + blockIdx.x; j < cend; j += gridDim.x) {
        Mp<W> y, l, ln, z;
        if (mine) ld_rw<W>(y, A, 0, i, j, rs.L);
        if (threadIdx.x == 0) s_x = y;
        if (mine && i > j0) ld_rw<W>(ln, A, 0, i, j0, rs.L);
        for (int64_t r = j0; r + 1 < je; ++r) {
            __syncthreads();                 // s_x = a_rj, final
            if (mine && i > r) {
                l = ln;
                // the next step's multiplier loads while this one multiplies
                if (i > r + 1) ld_rw<W>(ln, A, 0, i, r + 1, rs.L);
                // a_rj's words are read from shared memory as the product
                // forms, as the Block leaf reads b_kj (same bits as mul)
                mul_sm<W>(z, l.m, l.e, l.s, RecWords<W>{s_x.m}, s_x.e, s_x.s, rs);
                add<W, true>(y, y, z, 1u, rs);
            }
            __syncthreads();
            if (i == r + 1) s_x = y;
        }
        if (mine && i > j0) bad |= st<W>(y, A, 0, i, j, rs.L);
        __syncthreads();
    }
    if (bad) flag(status, ST_RANGE);
}

// ------------------------------------------------------- triangular solves
// x = U^-1 L^-1 P b, both substitutions column-oriented: row i of the
// forward pass takes y_i <- RN(y_i - RN(l_ij y_j)) for j = 0, 1, .., i-1 in
// that order; the backward pass sets x_j = RN(y_j / u_jj) for j = n-1 down to
// 0 and then y_i <- RN(y_i - RN(u_ij x_j)) for every i < j.  The rows are cut
// into blocks of SB: a one-CTA kernel finishes the diagonal block (its
// columns in order), then a grid kernel applies those columns to every row
// beyond the block, each row taking them in the same order as above.  Every
// y_i therefore sees exactly the update sequence of the plain column loop.
constexpr int SB = 64;

// perm = the row exchanges applied in order; y = P b
template <int W>
__global__ void __launch_bounds__(1024) lu_permute_kernel(int64_t n, const int64_t *piv, BMat b,
                                                          BMat y, int64_t *perm, int p)
{
    const RoundSpec rs = make_spec<W>(p);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t i = tid; i < n; i += nt) perm[i] = i;
    __syncthreads();
    if (tid == 0) {
        for (int64_t k = 0; k < n; ++k) {
            const int64_t q = piv[k];
            const int64_t t = perm[k];
            perm[k] = perm[q];
            perm[q] = t;
        }
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += nt) {
        const int64_t src = perm[i];
        for (int q = 0; q < rs.L; ++q) y.limb[(int64_t)q * y.plane + i * y.ld] = b.limb[(int64_t)q * b.plane + src * b.ld];
        y.exp[i * y.ld] = b.exp[src * b.ld];
        y.sign[i * y.ld] = b.sign[src * b.ld];
    }
}

// forward, diagonal block [c0, c1): one thread per row
template <int W>
__global__ void __launch_bounds__(SB) lu_fwd_diag_kernel(BMat LU, BMat y, int64_t c0, int64_t c1, int p,
                                                         DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t i = c0 + threadIdx.x;
    Mp<W> yi, yj, l, z;
    bool bad = false;
    if (i < c1) ld_rw<W>(yi, y, 0, i, 0, rs.L);
    for (int64_t j = c0; j + 1 < c1; ++j) {
        __syncthreads();                     // y_j is final
        if (i > j && i < c1) {
            ld_rw<W>(yj, y, 0, j, 0, rs.L);
            ld_rw<W>(l, LU, 0, i, j, rs.L);
            mul<W, true>(z, l, yj, rs);
            add<W, true>(yi, yi, z, 1u, rs);
            if (i == j + 1) bad |= st<W>(yi, y, 0, i, 0, rs.L);    // y_i final next step
        }
    }
    if (bad) flag(status, ST_RANGE);
}

// forward, rows [c1, n) take columns [c0, c1)
template <int W>
__global__ void lu_fwd_update_kernel(BMat LU, BMat y, int64_t n, int64_t c0, int64_t c1, int p,
                                     DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t i = c1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Mp<W> yi, yj, l, z;
    ld_rw<W>(yi, y, 0, i, 0, rs.L);
    for (int64_t j = c0; j < c1; ++j) {
        ld_rw<W>(yj, y, 0, j, 0, rs.L);
        ld_rw<W>(l, LU, 0, i, j, rs.L);
        mul<W, true>(z, l, yj, rs);
        add<W, true>(yi, yi, z, 1u, rs);
    }
    if (st<W>(yi, y, 0, i, 0, rs.L)) flag(status, ST_RANGE);
}

// backward, diagonal block [c0, c1): x_j for j = c1-1 down to c0; a zero
// u_jj gives x_j = +0 and reports the matrix singular.  Up to 1024 bits the
// first warp forms each x_j together.
template <int W>
__global__ void __launch_bounds__(SB) lu_bwd_diag_kernel(BMat LU, BMat y, BMat x, int64_t c0, int64_t c1,
                                                         int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t i = c0 + threadIdx.x;
    Mp<W> yi, xj, u, z;
    bool bad = false, zero = false;
    if (i < c1) ld_rw<W>(yi, y, 0, i, 0, rs.L);
    for (int64_t j = c1 - 1; j >= c0; --j) {
        if constexpr (W <= 32) {
            if (i == j) st<W>(yi, y, 0, j, 0, rs.L);          // y_j is final
            __syncthreads();
            if (threadIdx.x < 32) {
                int64_t ye, ue, qe;
                uint32_t ys, us, qs;
                const uint32_t um = wld<W>(LU, 0, j, j, rs.L, ue, us);
                const uint32_t ym = wld<W>(y, 0, j, 0, rs.L, ye, ys);
                uint32_t qm = 0u;
                if (ue == EXP_ZERO) {
                    zero = true;
                    qe = EXP_ZERO;
                    qs = 0u;
                } else {
                    qm = warp_div<W>(ym, ye, ys, um, ue, us, qe, qs, rs);
                }
                bad |= wst<W>(qm, qe, qs, x, 0, j, 0, rs.L);
            }
        } else {
            if (i == j) {                        // y_j is final: x_j = y_j / u_jj
                ld_rw<W>(u, LU, 0, j, j, rs.L);
                if (u.e == EXP_ZERO) {
                    zero = true;
                    set_zero<W>(z, 0u);
                } else {
                    div<W>(z, yi, u, rs);
                }
                bad |= st<W>(z, x, 0, j, 0, rs.L);
            }
        }
        __syncthreads();
        if (i >= c0 && i < j) {
            ld_rw<W>(xj, x, 0, j, 0, rs.L);
            ld_rw<W>(u, LU, 0, i, j, rs.L);
            mul<W, true>(z, u, xj, rs);
            add<W, true>(yi, yi, z, 1u, rs);
        }
    }
    if (zero) atomicOr(&status->flags, ST_SINGULAR);
    if (bad) flag(status, ST_RANGE);
}

// backward, rows [0, c0) take columns c1-1 down to c0
template <int W>
__global__ void lu_bwd_update_kernel(BMat LU, BMat y, BMat x, int64_t c0, int64_t c1, int p,
                                     DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= c0) return;
    Mp<W> yi, xj, u, z;
    ld_rw<W>(yi, y, 0, i, 0, rs.L);
    for (int64_t j = c1 - 1; j >= c0; --j) {
        ld_rw<W>(xj, x, 0, j, 0, rs.L);
        ld_rw<W>(u, LU, 0, i, j, rs.L);
        mul<W, true>(z, u, xj, rs);
        add<W, true>(yi, yi, z, 1u, rs);
    }
    if (st<W>(yi, y, 0, i, 0, rs.L)) flag(status, ST_RANGE);
}

// --------------------------------- solves by warps (512 to 1024 bits)
// The same blocked order as above, but each row belongs to a warp (lane =
// word) and every multiply-add and division is formed by warp_mul,
// warp_add and warp_div: the solves are chains of dependent operations,
// so the latency of one operation is what counts.  Diagonal blocks of SBW
// rows; the row that becomes final publishes its value through shared
// memory.
constexpr int SBW = 16;

template <int W>
__global__ void __launch_bounds__(SBW * 32) lu_fwd_diag_warp(BMat LU, BMat y, int64_t c0, int64_t c1, int p,
                                                            DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int lane = (int)(threadIdx.x & 31u), wid = (int)(threadIdx.x >> 5);
    const int64_t i = c0 + wid;
    const bool mine = i < c1;
    __shared__ uint32_t s_m[32];
    __shared__ int64_t s_e;
    __shared__ uint32_t s_s;
    int64_t ye = EXP_ZERO;
    uint32_t ys = 0u, ym = 0u;
    if (mine) ym = wld<W>(y, 0, i, 0, rs.L, ye, ys);
    for (int64_t j = c0; j + 1 < c1; ++j) {
        if (i == j) {                            // y_j is final
            s_m[lane] = ym;
            if (lane == 0) {
                s_e = ye;
                s_s = ys;
            }
        }
        __syncthreads();
        if (mine && i > j) {
            int64_t le, te;
            uint32_t ls, ts;
            const uint32_t lm = wld<W>(LU, 0, i, j, rs.L, le, ls);
            const uint32_t tm = warp_mul<W>(lm, le, ls, s_m[lane], s_e, s_s, te, ts, rs);
            ym = warp_add<W>(ym, ye, ys, tm, te, ts, 1u, ye, ys, rs);
        }
        __syncthreads();
    }
    if (mine && i > c0 && wst<W>(ym, ye, ys, y, 0, i, 0, rs.L) && lane == 0) flag(status, ST_RANGE);
}

// forward, rows [c1, n) take columns [c0, c1): one warp per row
template <int W>
__global__ void __launch_bounds__(128) lu_fwd_update_warp(BMat LU, BMat y, int64_t n, int64_t c0, int64_t c1,
                                                          int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t i = c1 + (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (i >= n) return;
    int64_t ye;
    uint32_t ys;
    uint32_t ym = wld<W>(y, 0, i, 0, rs.L, ye, ys);
    for (int64_t j = c0; j < c1; ++j) {
        int64_t ve, le, te;
        uint32_t vs, ls, ts;
        const uint32_t vm = wld<W>(y, 0, j, 0, rs.L, ve, vs);
        const uint32_t lm = wld<W>(LU, 0, i, j, rs.L, le, ls);
        const uint32_t tm = warp_mul<W>(lm, le, ls, vm, ve, vs, te, ts, rs);
        ym = warp_add<W>(ym, ye, ys, tm, te, ts, 1u, ye, ys, rs);
    }
    if (wst<W>(ym, ye, ys, y, 0, i, 0, rs.L) && lane == 0) flag(status, ST_RANGE);
}

// backward, diagonal block [c0, c1): x_j = y_j / u_jj for j = c1-1 down to
// c0 (a zero u_jj gives x_j = +0 and reports the matrix singular)
template <int W>
__global__ void __launch_bounds__(SBW * 32) lu_bwd_diag_warp(BMat LU, BMat y, BMat x, int64_t c0, int64_t c1,
                                                            int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int lane = (int)(threadIdx.x & 31u), wid = (int)(threadIdx.x >> 5);
    const int64_t i = c0 + wid;
    const bool mine = i < c1;
    __shared__ uint32_t s_m[32];
    __shared__ int64_t s_e;
    __shared__ uint32_t s_s;
    int64_t ye = EXP_ZERO;
    uint32_t ys = 0u, ym = 0u;
    bool bad = false, zero = false;
    if (mine) ym = wld<W>(y, 0, i, 0, rs.L, ye, ys);
    for (int64_t j = c1 - 1; j >= c0; --j) {
        if (i == j) {                            // y_j is final: x_j = y_j / u_jj
            int64_t ue, qe;
            uint32_t us, qs;
            const uint32_t um = wld<W>(LU, 0, j, j, rs.L, ue, us);
            uint32_t qm = 0u;
            if (ue == EXP_ZERO) {
                zero = true;
                qe = EXP_ZERO;
                qs = 0u;
            } else {
                qm = warp_div<W>(ym, ye, ys, um, ue, us, qe, qs, rs);
            }
            bad |= wst<W>(qm, qe, qs, x, 0, j, 0, rs.L);
            s_m[lane] = qm;
            if (lane == 0) {
                s_e = qe;
                s_s = qs;
            }
        }
        __syncthreads();
        if (mine && i < j) {
            int64_t ue, te;
            uint32_t us, ts;
            const uint32_t um = wld<W>(LU, 0, i, j, rs.L, ue, us);
            const uint32_t tm = warp_mul<W>(um, ue, us, s_m[lane], s_e, s_s, te, ts, rs);
            ym = warp_add<W>(ym, ye, ys, tm, te, ts, 1u, ye, ys, rs);
        }
        __syncthreads();
    }
    if (lane == 0 && zero) atomicOr(&status->flags, ST_SINGULAR);
    if (lane == 0 && bad) flag(status, ST_RANGE);
}

// backward, rows [0, c0) take columns c1-1 down to c0: one warp per row
template <int W>
__global__ void __launch_bounds__(128) lu_bwd_update_warp(BMat LU, BMat y, BMat x, int64_t c0, int64_t c1,
                                                          int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int lane = (int)(threadIdx.x & 31u);
    const int64_t i = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (i >= c0) return;
    int64_t ye;
    uint32_t ys;
    uint32_t ym = wld<W>(y, 0, i, 0, rs.L, ye, ys);
    for (int64_t j = c1 - 1; j >= c0; --j) {
        int64_t ve, ue, te;
        uint32_t vs, us, ts;
        const uint32_t vm = wld<W>(x, 0, j, 0, rs.L, ve, vs);
        const uint32_t um = wld<W>(LU, 0, i, j, rs.L, ue, us);
        const uint32_t tm = warp_mul<W>(um, ue, us, vm, ve, vs, te, ts, rs);
        ym = warp_add<W>(ym, ye, ys, tm, te, ts, 1u, ye, ys, rs);
    }
    if (wst<W>(ym, ye, ys, y, 0, i, 0, rs.L) && lane == 0) flag(status, ST_RANGE);
}

// Row exchanges k = j0 .. je-1 (rows k and piv[k], in order) on the columns
// outside the panel, [0, j0) and [je, n): one thread per column.  Exchanges
// of whole rows commute with the panel's work, which touches only the
// panel's columns, so the factors equal those of exchanging full rows at once.
template <int W>
__global__ void lu_laswp_kernel(BMat A, int64_t n, int64_t j0, int64_t je, const int64_t *piv, int L)
{
    const int64_t outside = n - (je - j0);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < outside;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t < j0 ? t : t + (je - j0);
        for (int64_t k = j0; k < je; ++k) {
            const int64_t r = piv[k];
            if (r == k) continue;
            for (int q = 0; q < L; ++q) {
                uint64_t *a = A.limb + (int64_t)q * A.plane + k * A.ld + c;
                uint64_t *b = A.limb + (int64_t)q * A.plane + r * A.ld + c;
                const uint64_t x = *a;
                *a = *b;
                *b = x;
            }
            int64_t *ea = A.exp + k * A.ld + c, *eb = A.exp + r * A.ld + c;
            const int64_t te = *ea;
            *ea = *eb;
            *eb = te;
            int8_t *sa = A.sign + k * A.ld + c, *sb = A.sign + r * A.ld + c;
            const int8_t ts = *sa;
            *sa = *sb;
            *sb = ts;
        }
    }
}

// ================================================================ launchers
template <int W>
void launch_lu_pivot(BMat A, int64_t n, int64_t k, int64_t *piv, int p, DevStatus *st,
                     cudaStream_t s, int64_t c0, int64_t c1, bool pivoting)
{
    lu_pivot_kernel<W><<<1, LuCfg<W>::PIVOT, 0, s>>>(A, pivoting ? n : k + 1, k, piv, p, st, c0, c1);
}

template <int W>
void launch_lu_divide(BMat A, int64_t n, int64_t k, int p, cudaStream_t s)
{
    const int64_t rows = n - k - 1;
    if (rows <= 0) return;
    if constexpr (W <= 32)
        lu_divide_kernel<W><<<grid_for(rows * 32, 128), 128, 0, s>>>(A, n, k, p);
    else
        lu_divide_kernel<W><<<grid_for(rows, 64), 64, 0, s>>>(A, n, k, p);
}

template <int W>
void launch_lu_rank1(BMat A, int64_t k, int64_t r0, int64_t r1, int64_t c0, int64_t c1, int p,
                     DevStatus *st, cudaStream_t s)
{
    const int64_t total = (r1 - r0) * (c1 - c0);
    if (r1 <= r0 || c1 <= c0) return;
    lu_rank1_kernel<W><<<grid_for(total, 128), 128, 0, s>>>(A, k, r0, r1, c0, c1, p, st);
}

template <int W>
void launch_lu_solve(BMat LU, int64_t n, const int64_t *piv, BMat b, BMat y, BMat x,
                     int64_t *perm, int p, DevStatus *st, cudaStream_t s)
{
    constexpr int T = 64;
    lu_permute_kernel<W><<<1, 1024, 0, s>>>(n, piv, b, y, perm, p);
    if constexpr (W >= 16 && W <= 32) {          // one thread per row is as fast below 512 bits
        for (int64_t c0 = 0; c0 < n; c0 += SBW) {
            const int64_t c1 = c0 + SBW < n ? c0 + SBW : n;
            lu_fwd_diag_warp<W><<<1, SBW * 32, 0, s>>>(LU, y, c0, c1, p, st);
            if (c1 < n)
                lu_fwd_update_warp<W><<<(unsigned)((n - c1 + 3) / 4), 128, 0, s>>>(LU, y, n, c0, c1, p, st);
        }
        for (int64_t c0 = ((n - 1) / SBW) * SBW; c0 >= 0; c0 -= SBW) {
            const int64_t c1 = c0 + SBW < n ? c0 + SBW : n;
            lu_bwd_diag_warp<W><<<1, SBW * 32, 0, s>>>(LU, y, x, c0, c1, p, st);
            if (c0 > 0) lu_bwd_update_warp<W><<<(unsigned)((c0 + 3) / 4), 128, 0, s>>>(LU, y, x, c0, c1, p, st);
        }
        return;
    }
    for (int64_t c0 = 0; c0 < n; c0 += SB) {
        const int64_t c1 = c0 + SB < n ? c0 + SB : n;
        lu_fwd_diag_kernel<W><<<1, SB, 0, s>>>(LU, y, c0, c1, p, st);
        if (c1 < n) lu_fwd_update_kernel<W><<<grid_for(n - c1, T), T, 0, s>>>(LU, y, n, c0, c1, p, st);
    }
    for (int64_t c0 = ((n - 1) / SB) * SB; c0 >= 0; c0 -= SB) {
        const int64_t c1 = c0 + SB < n ? c0 + SB : n;
        lu_bwd_diag_kernel<W><<<1, SB, 0, s>>>(LU, y, x, c0, c1, p, st);
        if (c0 > 0) lu_bwd_update_kernel<W><<<grid_for(c0, T), T, 0, s>>>(LU, y, x, c0, c1, p, st);
    }
}

// ------------------------------------ solves with several right-hand sides
// X = U^-1 L^-1 P B column by column of B, every column with exactly the
// update sequence of the one-column solve above: forward, y_i takes
// RN(y_i - RN(l_ij y_j)) for j = 0, 1, .., i-1; backward, x_j = RN(y_j / u_jj)
// for j = n-1 down to 0, then y_i takes RN(y_i - RN(u_ij x_j)) for i < j.
// One launch per column step j, all rows and right-hand sides at once.

// perm = the row exchanges of piv applied in order (one thread)
template <int W>
__global__ void lu_perm_kernel(int64_t n, const int64_t *piv, int64_t *perm)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t q = piv[k];
        const int64_t t = perm[k];
        perm[k] = perm[q];
        perm[q] = t;
    }
}

// Y(i, c) = B(perm[i], c)
template <int W>
__global__ void lu_gather_rows_kernel(BMat B, BMat Y, const int64_t *perm, int64_t n, int64_t nrhs, int L)
{
    const int64_t total = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nrhs, c = t % nrhs, src = perm[i];
        for (int q = 0; q < L; ++q)
            Y.limb[(int64_t)q * Y.plane + i * Y.ld + c] = B.limb[(int64_t)q * B.plane + src * B.ld + c];
        Y.exp[i * Y.ld + c] = B.exp[src * B.ld + c];
        Y.sign[i * Y.ld + c] = B.sign[src * B.ld + c];
    }
}

// Y(i, c) = RN(Y(i, c) - RN(M(i, j) S(j, c))) for i in [r0, r1), c < nrhs
template <int W>
__global__ void lu_multi_update_kernel(BMat M, BMat S, BMat Y, int64_t j, int64_t r0, int64_t r1, int64_t nrhs,
                                       int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t total = (r1 - r0) * nrhs;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r0 + t / nrhs, c = t % nrhs;
        Mp<W> m, x, y, z;
        ld<W>(m, M, 0, i, j, rs.L);
        ld_rw<W>(x, S, 0, j, c, rs.L);
        ld_rw<W>(y, Y, 0, i, c, rs.L);
        mul<W>(z, m, x, rs);
        add<W>(y, y, z, 1u, rs);
        bad |= st<W>(y, Y, 0, i, c, rs.L);
    }
    if (bad) flag(status, ST_RANGE);
}

// X(j, c) = RN(Y(j, c) / u_jj) for c < nrhs; a zero u_jj gives +0 and
// reports the matrix singular
template <int W>
__global__ void lu_multi_divide_kernel(BMat LU, BMat Y, BMat X, int64_t j, int64_t nrhs, int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    bool bad = false, sing = false;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nrhs;
         c += (int64_t)gridDim.x * blockDim.x) {
        Mp<W> u, y, x;
        ld<W>(u, LU, 0, j, j, rs.L);
        ld_rw<W>(y, Y, 0, j, c, rs.L);
        if (u.e == EXP_ZERO) {
            set_zero<W>(x, 0u);
            sing = true;
        } else {
            div<W>(x, y, u, rs);
        }
        bad |= st<W>(x, X, 0, j, c, rs.L);
    }
    if (bad) flag(status, ST_RANGE);
    if (sing && status) {
        atomicOr(&status->flags, ST_SINGULAR);
        atomicMin(&status->singular_col, (long long)j);
    }
}

template <int W>
void launch_lu_solve_multi(BMat LU, int64_t n, const int64_t *piv, BMat B, BMat Y, BMat X, int64_t nrhs,
                           int64_t *perm, int p, DevStatus *st, cudaStream_t s)
{
    if (n <= 0 || nrhs <= 0) return;
    constexpr int T = 128;
    lu_perm_kernel<W><<<1, 32, 0, s>>>(n, piv, perm);
    lu_gather_rows_kernel<W><<<grid_for(n * nrhs, T), T, 0, s>>>(B, Y, perm, n, nrhs, (p + 63) >> 6);
    for (int64_t j = 0; j + 1 < n; ++j)
        lu_multi_update_kernel<W><<<grid_for((n - j - 1) * nrhs, T), T, 0, s>>>(LU, Y, Y, j, j + 1, n, nrhs, p,
                                                                               st);
    for (int64_t j = n - 1; j >= 0; --j) {
        lu_multi_divide_kernel<W><<<grid_for(nrhs, T), T, 0, s>>>(LU, Y, X, j, nrhs, p, st);
        if (j > 0)
            lu_multi_update_kernel<W><<<grid_for(j * nrhs, T), T, 0, s>>>(LU, X, Y, j, 0, j, nrhs, p, st);
    }
}

// true when the fused column step and the one-launch U12 solve apply
template <int W>
bool lu_fused_ok(int64_t panel)
{
    return W <= 32 && panel <= 128;
}

template <int W>
void launch_lu_column(BMat A, int64_t n, int64_t j0, int64_t k, int64_t je, int64_t ce, int64_t *piv, int p,
                      DevStatus *st, int64_t *cand, unsigned *ticket, cudaStream_t s, bool pivoting)
{
    if constexpr (W <= 32) {
        const int64_t rows = n - k - 1;
        if (rows <= 0) return;
        int64_t g = (rows + LU_COL_WARPS - 1) / LU_COL_WARPS;
        if (g > LU_COL_MAX_CTAS) g = LU_COL_MAX_CTAS;
        lu_column_kernel<W><<<(unsigned)g, LU_COL_WARPS * 32, 0, s>>>(A, n, j0, k, je, ce, piv, p, st, cand,
                                                                     ticket, pivoting ? 1 : 0);
    }
}

template <int W>
void launch_lu_laswp(BMat A, int64_t n, int64_t j0, int64_t je, const int64_t *piv, int p, cudaStream_t s)
{
    const int64_t outside = n - (je - j0);
    if (outside <= 0) return;
    lu_laswp_kernel<W><<<grid_for(outside, 128), 128, 0, s>>>(A, n, j0, je, piv, (p + 63) >> 6);
}

template <int W>
void launch_lu_u12(BMat A, int64_t cend, int64_t j0, int64_t je, int p, DevStatus *st, cudaStream_t s)
{
    if constexpr (W <= 32) {
        const int64_t cols = cend - je;
        if (cols <= 0) return;
        const int64_t g = cols < 152 * 8 ? cols : 152 * 8;
        lu_u12_kernel<W><<<(unsigned)g, 128, 0, s>>>(A, cend, j0, je, p, st);
    }
}

#define MPG_INSTANTIATE_LU(W)                                                                   \
    template void launch_lu_pivot<W>(BMat, int64_t, int64_t, int64_t *, int, DevStatus *,       \
                                     cudaStream_t, int64_t, int64_t, bool);                     \
    template void launch_lu_divide<W>(BMat, int64_t, int64_t, int, cudaStream_t);               \
    template void launch_lu_rank1<W>(BMat, int64_t, int64_t, int64_t, int64_t, int64_t, int,    \
                                     DevStatus *, cudaStream_t);                                \
    template void launch_lu_solve<W>(BMat, int64_t, const int64_t *, BMat, BMat, BMat,          \
                                     int64_t *, int, DevStatus *, cudaStream_t);                \
    template bool lu_fused_ok<W>(int64_t);                                                      \
    template void launch_lu_column<W>(BMat, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t *, \
                                      int, DevStatus *, int64_t *, unsigned *, cudaStream_t, bool); \
    template void launch_lu_laswp<W>(BMat, int64_t, int64_t, int64_t, const int64_t *, int,     \
                                     cudaStream_t);                                             \
    template void launch_lu_u12<W>(BMat, int64_t, int64_t, int64_t, int, DevStatus *, cudaStream_t); \
    template void launch_lu_solve_multi<W>(BMat, int64_t, const int64_t *, BMat, BMat, BMat, int64_t, \
                                           int64_t *, int, DevStatus *, cudaStream_t);

}  // namespace mpg
