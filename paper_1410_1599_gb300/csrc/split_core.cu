// split_core.cu -- the slice-product kernel of the split form (tensor cores,
// fp16 digit planes, exact fp32 chunks folded into int64); see mp_split.cuh.
#include "mp_split.cuh"

namespace mpg {

int split_digit_count(int p) { return split_digits(p); }
int64_t split_row_pad(int64_t l) { return split_lpad(l); }

static __device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
                 "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// D[s][i][j] for every diagonal s = 0 .. 2S-2.  CTA: 64 x 64 outputs, four
// warps of 32 x 32 (2 x 4 mma tiles of 16 x 8).
__global__ void __launch_bounds__(128)
split_slice_kernel(const __half *__restrict__ Ap, const __half *__restrict__ Bp, int64_t m,
                   int64_t n, int64_t lp, int S, long long *__restrict__ D)
{
    __shared__ __align__(16) __half As[SPLIT_TM][SPLIT_TK + 8];
    __shared__ __align__(16) __half Bs[SPLIT_TN][SPLIT_TK + 8];
    const int64_t tiles_n = (n + SPLIT_TN - 1) / SPLIT_TN;
    const int64_t i0 = (blockIdx.x / tiles_n) * SPLIT_TM, j0 = (blockIdx.x % tiles_n) * SPLIT_TN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, tg = lane & 3;
    const int64_t plane_a = m * lp, plane_b = n * lp;
    for (int s = 0; s <= 2 * S - 2; ++s) {
        long long acc[2][4][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][b][c] = 0;
        const int u0 = s - (S - 1) > 0 ? s - (S - 1) : 0, u1 = s < S - 1 ? s : S - 1;
        for (int u = u0; u <= u1; ++u) {
            const int v = s - u;
            const __half *Au = Ap + (int64_t)u * plane_a;
            const __half *Bv = Bp + (int64_t)v * plane_b;
            float f[2][4][4];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) f[a][b][c] = 0.f;
            int cnt = 0;
            for (int64_t kb = 0; kb < lp; kb += SPLIT_TK) {
                // stage 64 x 32 halves of A_u and of B_v (16-byte vectors)
                for (int e = tid; e < SPLIT_TM * SPLIT_TK / 8; e += 128) {
                    const int r = e / (SPLIT_TK / 8), c8 = (e % (SPLIT_TK / 8)) * 8;
                    uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
                    if (i0 + r < m) va = *reinterpret_cast<const uint4 *>(Au + (i0 + r) * lp + kb + c8);
                    if (j0 + r < n) vb = *reinterpret_cast<const uint4 *>(Bv + (j0 + r) * lp + kb + c8);
                    *reinterpret_cast<uint4 *>(&As[r][c8]) = va;
                    *reinterpret_cast<uint4 *>(&Bs[r][c8]) = vb;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < SPLIT_TK; kk += 16) {
                    uint32_t af[2][4], bf[4][2];
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        const int r = wm * 32 + mt * 16 + g;
                        af[mt][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + tg * 2]);
                        af[mt][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + tg * 2]);
                        af[mt][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 8 + tg * 2]);
                        af[mt][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 8 + tg * 2]);
                    }
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) {
                        const int c = wn * 32 + nt * 8 + g;
                        bf[nt][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + tg * 2]);
                        bf[nt][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 8 + tg * 2]);
                    }
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt) mma_16816(f[mt][nt], af[mt], bf[nt]);
                }
                __syncthreads();
                cnt += SPLIT_TK;
                if (cnt >= SPLIT_CHUNK || kb + SPLIT_TK >= lp) {
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b)
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                acc[a][b][c] += (long long)__float2ll_rn(f[a][b][c]);
                                f[a][b][c] = 0.f;
                            }
                    cnt = 0;
                }
            }
        }
        // D_s for this thread's 32 outputs
        long long *Ds = D + (int64_t)s * m * n;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int64_t i = i0 + wm * 32 + mt * 16 + g + (c >= 2 ? 8 : 0);
                    const int64_t j = j0 + wn * 32 + nt * 8 + tg * 2 + (c & 1);
                    if (i < m && j < n) Ds[i * n + j] = acc[mt][nt][c];
                }
    }
}

void launch_split_slices(const __half *pa, const __half *pb, int64_t m, int64_t l, int64_t n,
                                int p, long long *D, cudaStream_t s)
{
    const int S = split_digits(p);
    const int64_t tiles = ((m + SPLIT_TM - 1) / SPLIT_TM) * ((n + SPLIT_TN - 1) / SPLIT_TN);
    split_slice_kernel<<<(unsigned)tiles, 128, 0, s>>>(pa, pb, m, n, split_lpad(l), S, D);
}

}  // namespace mpg
