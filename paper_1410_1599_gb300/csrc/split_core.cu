// split_core.cu -- the slice-product kernel of the split form (see
// mp_split.cuh): D_s(i, j) = sum_{u+v=s} sum_k A_u(i,k) B_v(j,k) exactly, for
// every weight diagonal s, on tensor cores.
//
// CTA tile 128 x 128 outputs, 8 warps of 64 x 32 (4 x 4 mma.m16n8k16 tiles).
// The (pair, k-block) steps of a diagonal form one stream fed by a 4-stage
// cp.async pipeline (k-blocks of 32 halves, operands staged in shared memory,
// fragments loaded with ldmatrix).  Exactness: digit products are integers of
// magnitude <= 2^14; an fp32 accumulator takes at most SPLIT_CHUNK = 512 of
// them (< 2^24: every partial sum is an exact fp32 integer) and is then
// folded into an int32 accumulator; one digit pair contributes at most
// lp * 2^14, so the int32 holds max_pairs = floor((2^31 - 1) / (lp 2^14))
// pairs before it is added into the int64 D_s in global memory.
#include "mp_split.cuh"

namespace mpg {

int split_digit_count(int p) { return split_digits(p); }
int64_t split_row_pad(int64_t l) { return split_lpad(l); }

namespace {

constexpr int TM = 128, TN = 128, TK = SPLIT_TK, STAGES = 4, PADK = TK + 8;
constexpr int THREADS = 256;
constexpr int STAGE_HALVES = (TM + TN) * PADK;
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_HALVES * 2;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    const int sz = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(sz));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                          uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
                 "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

}  // namespace

__global__ void __launch_bounds__(THREADS, 1)
split_slice_kernel(const __half *__restrict__ Ap, const __half *__restrict__ Bp, int64_t m,
                   int64_t n, int64_t lp, int S, int max_pairs, int groups, long long *__restrict__ D)
{
    extern __shared__ __align__(16) __half sm[];
    const int64_t tiles_n = (n + TN - 1) / TN;
    const int64_t tile = blockIdx.x / groups;
    const int grp = (int)(blockIdx.x % groups);      // this CTA's share of the diagonals
    const int64_t i0 = (tile / tiles_n) * TM, j0 = (tile % tiles_n) * TN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 2, wn = warp & 3, g = lane >> 2, tg = lane & 3;
    const int64_t plane_a = m * lp, plane_b = n * lp;
    const int nkb = (int)(lp / TK);

    for (int s = grp; s <= 2 * S - 2; s += groups) {
        const int u0 = s - (S - 1) > 0 ? s - (S - 1) : 0, u1 = s < S - 1 ? s : S - 1;
        const int npairs = u1 - u0 + 1;
        const int total = npairs * nkb;

        // issue the copies of step t into stage buffer t % STAGES
        auto load = [&](int t) {
            if (t < total) {
                const int pu = t / nkb;
                const int u = u0 + pu, kb = t - pu * nkb;
                const __half *Au = Ap + (int64_t)u * plane_a + kb * TK;
                const __half *Bv = Bp + (int64_t)(s - u) * plane_b + kb * TK;
                __half *st = sm + (t % STAGES) * STAGE_HALVES;
#pragma unroll
                for (int q = 0; q < (TM + TN) * TK / 8 / THREADS; ++q) {
                    const int e = tid + q * THREADS;
                    const int r = e / (TK / 8), c8 = (e % (TK / 8)) * 8;
                    if (r < TM) {
                        const bool ok = i0 + r < m;
                        cp_async16(st + r * PADK + c8, Au + (ok ? (i0 + r) : 0) * lp + c8, ok);
                    } else {
                        const int rb = r - TM;
                        const bool ok = j0 + rb < n;
                        cp_async16(st + r * PADK + c8, Bv + (ok ? (j0 + rb) : 0) * lp + c8, ok);
                    }
                }
            }
            cp_commit();
        };

        int acc[4][4][4];
        float f[4][4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) { acc[a][b][c] = 0; f[a][b][c] = 0.f; }
        int pairs_in_acc = 0;
        bool first_flush = true;

        auto flush = [&]() {           // acc (int32) into D_s (int64), then clear
            long long *Ds = D + (int64_t)s * m * n;
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int64_t i = i0 + wm * 64 + mt * 16 + g + (c >= 2 ? 8 : 0);
                        const int64_t j = j0 + wn * 32 + nt * 8 + tg * 2 + (c & 1);
                        if (i < m && j < n) {
                            long long *d = Ds + i * n + j;
                            *d = (first_flush ? 0ll : *d) + (long long)acc[mt][nt][c];
                        }
                        acc[mt][nt][c] = 0;
                    }
            first_flush = false;
            pairs_in_acc = 0;
        };

#pragma unroll
        for (int t = 0; t < STAGES - 1; ++t) load(t);
        for (int t = 0; t < total; ++t) {
            cp_wait<STAGES - 2>();
            __syncthreads();
            load(t + STAGES - 1);
            const __half *st = sm + (t % STAGES) * STAGE_HALVES;
            const __half *As = st, *Bs = st + TM * PADK;
#pragma unroll
            for (int kk = 0; kk < TK; kk += 16) {
                uint32_t af[4][4], bf[2][4];
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
                    ldsm_x4(af[mt], As + (wm * 64 + mt * 16 + (lane & 15)) * PADK + kk + (lane >> 4) * 8);
#pragma unroll
                for (int np = 0; np < 2; ++np)
                    ldsm_x4(bf[np], Bs + (wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3)) * PADK +
                                        kk + ((lane >> 3) & 1) * 8);
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        mma_16816(f[mt][nt], af[mt], bf[nt >> 1][(nt & 1) * 2], bf[nt >> 1][(nt & 1) * 2 + 1]);
            }
            const int kb = t % nkb;
            const bool pair_end = kb == nkb - 1;
            if (((kb + 1) % (SPLIT_CHUNK / TK)) == 0 || pair_end) {
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            acc[a][b][c] += __float2int_rn(f[a][b][c]);
                            f[a][b][c] = 0.f;
                        }
            }
            if (pair_end) {
                ++pairs_in_acc;
                if (pairs_in_acc == max_pairs || t == total - 1) flush();
            }
        }
        cp_wait<0>();
        __syncthreads();
    }
}

void launch_split_slices(const __half *pa, const __half *pb, int64_t m, int64_t l, int64_t n,
                         int p, long long *D, cudaStream_t s)
{
    const int S = split_digits(p);
    const int64_t lp = split_lpad(l);
    const int64_t per_pair = lp * 16384;                     // |one pair's sum| <= lp 2^14
    int max_pairs = (int)((((int64_t)1 << 31) - 1) / per_pair);
    if (max_pairs < 1) max_pairs = 1;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(split_slice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
        attr = true;
    }
    const int64_t tiles = ((m + TM - 1) / TM) * ((n + TN - 1) / TN);
    // spread the diagonals of a tile over several CTAs until about four waves
    int groups = 1;
    while (tiles * groups < 4 * 152 && groups * 2 <= 2 * S - 1) groups *= 2;
    split_slice_kernel<<<(unsigned)(tiles * groups), THREADS, SMEM_BYTES, s>>>(pa, pb, m, n, lp, S,
                                                                               max_pairs, groups, D);
}

}  // namespace mpg
