// mp_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace mpg {

// capacity class above 2048 bits: 272 words (8704 bits)
constexpr int BIG_W = 272;

// A batch of equally shaped matrices in device memory.  Element (b, r, c):
//   limb k : limb[b * bs_limb + k * plane + r * ld + c]
//   exp    : exp [b * bs_es + r * ld + c],  sign likewise
struct BMat {
    uint64_t *limb;
    int64_t *exp;
    int8_t *sign;
    int64_t ld, plane, bs_limb, bs_es;
};

// device-side status word bits (ORed by kernels, read by mp_sync_status)
enum : unsigned {
    ST_RANGE = 1u,
    ST_DIVZERO = 2u,
    ST_SINGULAR = 4u,
    ST_TIMEOUT = 8u,
    ST_WIDE = 16u,         // exact accumulation: exponent spread beyond the accumulator
};

struct DevStatus {
    unsigned flags;
    unsigned pad;
    long long singular_col;   // smallest column index with a zero pivot
    unsigned long long split_fallbacks;   // split-form outputs recomputed exactly
};

// Launchers, one instantiation per word-capacity class W in {4, 8, 16, 32, 64}.
// All take the precision p (<= 32 W) and the stream; all sizes are elements.
template <int W>
void launch_elementwise(int op, BMat X, BMat Y, BMat R, int64_t rows, int64_t cols, int p,
                        DevStatus *st, cudaStream_t s);

// the same operations with one warp per element (W <= 32; mp_warp.cuh)
template <int W>
void launch_elementwise_warp(int op, BMat X, BMat Y, BMat R, int64_t rows, int64_t cols, int p,
                             DevStatus *st, cudaStream_t s);

template <int W>
void launch_convert(BMat X, int px, BMat R, int pr, int64_t rows, int64_t cols,
                    DevStatus *st, cudaStream_t s);

template <int W>
void launch_gemm_simple(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p,
                        DevStatus *st, cudaStream_t s);

// C_b = A_b B_b for b < batch by the Block kernel (A_b m x l, B_b l x n).
// With tma set and a layout the bulk tensor copies can address (see
// limb_map), the A/B limb tiles are staged in shared memory by TMA;
// otherwise the CTA's threads load them.  Same bits either way.  Returns
// true when the TMA-staged kernel ran.
template <int W>
bool launch_gemm_block(BMat A, BMat B, BMat C, int64_t batch, int64_t m, int64_t l, int64_t n,
                       int p, DevStatus *st, cudaStream_t s, bool tma = false);
// Several batches of equally shaped products (all of one precision) in one
// grouped Block launch: batch g is C_b = A_b B_b for b < batch (strides in
// the BMat batch fields), m x l x n each.  tiles_m/n and first[] are filled
// in by the launcher.
constexpr int LEAF_GROUP_MAX = 32;
struct LeafBatch {
    BMat A, B, C;
    int64_t batch, m, l, n, tiles_m, tiles_n;
};
struct LeafGroup {
    LeafBatch batch[LEAF_GROUP_MAX];
    int64_t first[LEAF_GROUP_MAX + 1];
    int count;
};
template <int W>
void launch_gemm_block_group(LeafGroup grp, int p, DevStatus *st, cudaStream_t s);
// The last level of a Strassen / Winograd recursion with its plain-quadrant
// children left in the parents: child t of node b takes quadrant qa[t] of
// parent b of Ap (1..4 = 11, 12, 21, 22; 0 = the materialised child), and
// likewise qb[t] of Bp.
// The parents are `nodes` matrices of a_rows x a_cols (A side) and
// b_rows x b_cols (B side), their real sizes.
struct LeafViews {
    BMat Ap, Bp;
    int64_t nodes, a_rows, a_cols, b_rows, b_cols;
    uint8_t qa[7], qb[7];
};
template <int W>
bool launch_gemm_leaf_views(BMat A, BMat B, BMat C, const LeafViews &v, int64_t batch, int64_t m, int64_t l,
                            int64_t n, int p, DevStatus *st, cudaStream_t s, bool tma = false);

// Largest class whose Block leaf stages its tiles by TMA.  At 2048 bits
// (b streamed from shared memory by rows, 255 registers) the plane layout
// measured 433 against 290 ms for a 1024^3 Winograd product (cutoff 32), so
// that class keeps the thread-staged records.
constexpr int TMA_MAX_W = 32;

// Tensor map for TMA loads of the limb planes of a batch of `batch`
// rows x cols matrices laid out as M (limb q of element (b, r, c) at
// b * bs + q * plane + r * ld + c, bs = M.bs_limb, or one matrix when
// batch == 1): a 4-D uint64 tensor {cols, rows, L, batch}, boxes of
// box_x x box_y elements over all L planes, zeros past the edges.  False,
// with *map untouched, when the layout is outside what the copies can
// address: a limb base not 16-byte aligned, an odd ld, plane or batch
// stride (byte strides must be multiples of 16), sizes beyond the copy
// unit's limits, or no driver entry point.
bool limb_map(CUtensorMap *map, const BMat &M, int64_t batch, int64_t rows, int64_t cols, int L,
              uint32_t box_x, uint32_t box_y);

// one CTA's bounded wait on an mbarrier that nothing completes (the
// failure-detection self-test): sets ST_TIMEOUT after about `cycles` clocks
void launch_wait_selftest(DevStatus *st, long long cycles, cudaStream_t s);
// one product of a serving group (gemm_group in mp_api.cu): C = A B with
// algorithm algo, device workspace ws of ws_bytes
struct GroupGemm {
    int algo, cutoff;
    int64_t m, l, n;
    BMat A, B, C;
    void *ws;
    size_t ws_bytes;
};
// C := C - A B, each c_ij = RN(c_ij - RN(a_ik b_kj)) for k ascending
template <int W>
void launch_gemm_sub(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p,
                     DevStatus *st, cudaStream_t s);

// one level of the recursion on a batch of `nodes` parents
//   parent A: m x l (real), even sizes M x K, halves h = M/2, k = K/2
//   children: 7 * nodes matrices of h x k, child t of node b at index 7b + t
// skip_plain: the children that are plain quadrants of the parent are not
// written (the leaves read them from the parent: LeafViews)
template <int W>
void launch_operands_a(int algo, BMat P, BMat Ch, int64_t nodes, int64_t m, int64_t l,
                       int64_t h, int64_t k, int p, cudaStream_t s, bool skip_plain = false);
template <int W>
void launch_operands_b(int algo, BMat P, BMat Ch, int64_t nodes, int64_t l, int64_t n,
                       int64_t k, int64_t w, int p, cudaStream_t s, bool skip_plain = false);
// combine 7 child products (h x w) into the parent C (m x n real part mr x nr)
template <int W>
void launch_combine(int algo, BMat Ch, BMat C, int64_t nodes, int64_t h, int64_t w,
                    int64_t mr, int64_t nr, int p, DevStatus *st, cudaStream_t s);
// peel fix-ups on a batch of nodes (A: m x l, B: l x n, C: m x n)
template <int W>
void launch_rank1(BMat A, BMat B, BMat C, int64_t nodes, int64_t mr, int64_t nr, int64_t l,
                  int p, DevStatus *st, cudaStream_t s);
template <int W>
void launch_border(BMat A, BMat B, BMat C, int64_t nodes, int64_t m, int64_t l, int64_t n,
                   int64_t mr, bool last_row, bool last_col, int p, DevStatus *st,
                   cudaStream_t s);

// C = RN_p(exact A B): every dot product exact, rounded once
template <int W>
void launch_gemm_exact(BMat A, BMat B, BMat C, int64_t m, int64_t l, int64_t n, int p,
                       DevStatus *st, cudaStream_t s, const uint8_t *rowsel = nullptr,
                       const uint8_t *colsel = nullptr);

// One thread per listed output t = i n + j (list[0 .. *count)): c_ij by the
// exact limb kernel; *count is added to status->split_fallbacks.
template <int W>
void launch_gemm_exact_list(BMat A, BMat B, BMat C, int64_t n, int64_t l, int p, DevStatus *st,
                            cudaStream_t s, const int64_t *list, const unsigned long long *count);

// split form of C = RN_p(exact A B) (mp_split.cuh): digit planes, slice
// products by weight diagonal, recombination; rows/columns beyond the
// spread budget are recomputed by launch_gemm_exact with rowsel/colsel.
// With truncation the diagonals below s0 are skipped (D holds planes
// s0 .. 2S-2), their sum is below 2^eb in units of the lowest digit, and
// outputs whose rounding that bound leaves open are listed for the exact
// limb kernel (eb < 0: nothing skipped, nothing listed).
int split_digit_count(int p);
// true when ptr is device memory of the calling thread's current device
// (not host, managed or another GPU's memory); the split form's tensor maps
// may only cover such memory
bool on_current_device(const void *ptr);
// flags mpgemm_noalloc recorded on the current device since the last call
// (then cleared); 0 when it has never run there
unsigned noalloc_take_flags();
int64_t split_row_pad(int64_t l);
int split_first_diagonal(int p, int64_t l, int64_t *ebits);
template <int W>
void launch_split_prep(BMat A, BMat B, int64_t m, int64_t l, int64_t n, int p, __half *pa,
                       __half *pb, int64_t *ea, int64_t *eb, uint8_t *wa, uint8_t *wb, cudaStream_t s);
int launch_split_slices(const __half *pa, const __half *pb, int64_t m, int64_t l, int64_t n, int p,
                        int s0, long long *D, DevStatus *st, cudaStream_t s);
template <int W>
void launch_split_finish(const long long *D, int64_t m, int64_t n, int p, int s0, int64_t ebits,
                         const int64_t *ea, const int64_t *eb, const uint8_t *wa, const uint8_t *wb,
                         BMat C, int64_t *list, unsigned long long *count, DevStatus *st, cudaStream_t s);

// LU (Sec. 4): pivot search + row exchange of column k; l_ik = a_ik / a_kk;
// one elimination step a_ij -= a_ik a_kj on [r0, r1) x [c0, c1); solves
template <int W>
void launch_lu_pivot(BMat A, int64_t n, int64_t k, int64_t *piv, int p, DevStatus *st,
                     cudaStream_t s, int64_t c0, int64_t c1, bool pivoting);
template <int W>
void launch_lu_divide(BMat A, int64_t n, int64_t k, int p, cudaStream_t s);
template <int W>
void launch_lu_rank1(BMat A, int64_t k, int64_t r0, int64_t r1, int64_t c0, int64_t c1, int p,
                     DevStatus *st, cudaStream_t s);
template <int W>
void launch_lu_solve(BMat LU, int64_t n, const int64_t *piv, BMat b, BMat y, BMat x,
                     int64_t *perm, int p, DevStatus *st, cudaStream_t s);
// Fused panel column step (l_ik, the panel row updates and the next pivot in
// one launch) and the one-launch U12 solve; up to 1024 bits, panels <= 128.
// cand holds LU_COL_MAX_CTAS row slots; *ticket starts at 0 and is returned
// to 0 by every launch.
constexpr int64_t LU_COL_MAX_CTAS = 152 * 8;
// sub-panel width of the fused panel factorisation above 256 bits (two
// columns per lane of the column step's row warps; 64 measured fastest
// against 32 and 128 at n = 1024, 1024 bits).  Up to 256 bits a multiply-add
// is cheap and the whole panel is one sub-panel: the sub-panel products and
// solves would cost more launches than the column steps' extra rounds.
#ifndef MPG_LU_SUB
#define MPG_LU_SUB 64
#endif
constexpr int64_t LU_SUB = MPG_LU_SUB;
template <int W>
constexpr int64_t lu_sub_width() { return W <= 8 ? 128 : LU_SUB; }
template <int W>
bool lu_fused_ok(int64_t panel);
// column step k of the panel [j0, je): row updates over columns (k, ce)
// with ce <= je, row exchanges over the panel's columns
template <int W>
void launch_lu_column(BMat A, int64_t n, int64_t j0, int64_t k, int64_t je, int64_t ce, int64_t *piv,
                      int p, DevStatus *st, int64_t *cand, unsigned *ticket, cudaStream_t s, bool pivoting);
template <int W>
void launch_lu_laswp(BMat A, int64_t n, int64_t j0, int64_t je, const int64_t *piv, int p, cudaStream_t s);
// rows [j0, je) of the columns [je, cend): U = L^-1 A with the unit lower
// triangle L of rows and columns [j0, je)
template <int W>
void launch_lu_u12(BMat A, int64_t cend, int64_t j0, int64_t je, int p, DevStatus *st, cudaStream_t s);
// X = A^-1 B for the nrhs columns of B from the factors in LU and piv; Y is
// n x nrhs workspace, perm n int64
template <int W>
void launch_lu_solve_multi(BMat LU, int64_t n, const int64_t *piv, BMat B, BMat Y, BMat X, int64_t nrhs,
                           int64_t *perm, int p, DevStatus *st, cudaStream_t s);

}  // namespace mpg
