// split_core.cu -- the slice-product kernel of the split form (see
// mp_split.cuh): D_s(i, j) = sum_{u+v=s} sum_k A_u(i,k) B_v(j,k) exactly, for
// every weight diagonal s, on the fifth-generation tensor cores.
//
// A cluster of 2 x 2 CTAs owns a 256 x 512 block of outputs (four 128 x 256
// tiles) and a strided set of diagonals.  CTA (r, c) shares its A tile with
// (r, 1-c) and its B tile with (1-r, c).
//   warp 0     TMA producer: one 64-row half of its 128 x 64 A tile,
//              multicast to its row peer, and one 128-row half of its
//              256 x 64 B tile, multicast to its column peer (fp16, 128-byte
//              swizzle), into a 4-stage shared-memory ring; a stage is
//              refilled once this CTA and both peers have consumed it;
//   warp 1     allocates the tensor memory and issues tcgen05.mma
//              (kind::f16, M = 128, N = 256, K = 16, fp32 accumulation) from
//              one thread; two 256-column accumulators alternate;
//   warps 2-9  drain an accumulator every CHUNK = 512 k-terms: tcgen05.ld,
//              conversion of the exact fp32 integers to int32 and accumulation
//              in registers (each thread one tile row, 128 columns); after at
//              most 255 chunks, and at the end of a diagonal, the int32 sums
//              are stored to (first time) or added into the int64 D_s.
// Exactness: a digit product is an integer of magnitude <= 2^14; an fp32
// accumulator takes at most 512 of them (< 2^24: every partial sum is an
// exact fp32 integer, whatever the tensor core's summation order); an int32
// register takes at most 255 such chunks (< 2^31).  Chunks may cross pair
// boundaries inside a diagonal: all its products carry the same weight.
// Every wait is bounded; a wait that runs out sets ST_TIMEOUT and the CTA
// unwinds (tensor memory is released on every path).
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "mpgemm.h"
#include "mp_split.cuh"
#include "mp_tc.cuh"

namespace mpg {

int split_digit_count(int p) { return split_digits(p); }

bool on_current_device(const void *ptr)
{
    int dev = -1;
    cudaPointerAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}
int64_t split_row_pad(int64_t l) { return split_lpad(l); }

// Lowest diagonal kept by the truncated form and the bound 2^ebits on the
// skipped part (see mp_split.cuh).  A typical output's leading bit lies at
// 2F - 2 or above (its largest products have both factors aligned to the top
// digit); the skipped part is placed SPLIT_GUARD bits under that output's
// round bit at 2F - 2 - p, so an output must sit about SPLIT_GUARD - 32 bits
// lower before its rounding is left open with any real probability.
int split_first_diagonal(int p, int64_t l, int64_t *ebits)
{
    constexpr int SPLIT_GUARD = 72;
    const int S = split_digits(p);
    const int64_t F = p + SPLIT_SB;
    int hb = 0;                                          // ceil(log2(lp S))
    while (((int64_t)1 << hb) < split_lpad(l) * S) ++hb;
    const int64_t room = 2 * F - 2 - p - SPLIT_GUARD - hb - 14;
    int s0 = room > 0 ? (int)(room / 8) : 0;
    if (s0 > 2 * S - 2) s0 = 2 * S - 2;
    *ebits = s0 > 0 ? hb + 14 + 8 * (int64_t)s0 : -1;
    return s0;
}

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
// cluster geometry: CR row tiles share one B tile, CC column tiles one A tile
#ifndef MPG_SPLIT_CR
#define MPG_SPLIT_CR 1
#endif
#ifndef MPG_SPLIT_CC
#define MPG_SPLIT_CC 2
#endif
constexpr int CR = MPG_SPLIT_CR, CC = MPG_SPLIT_CC, CSIZE = CR * CC;
static_assert(CSIZE <= 8 && BM % CC == 0 && BN % CR == 0, "cluster geometry");
constexpr int KB_PER_CHUNK = SPLIT_CHUNK / BK;                 // 8
constexpr int CHUNKS_PER_I32 = 255;
constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;             // 48 KB
constexpr int EPI_WARPS = 8, THREADS = (2 + EPI_WARPS) * 32;
constexpr int EPI_COLS = BN / (EPI_WARPS / 4);                  // columns per epilogue thread
constexpr uint32_t TMEM_COLS = 2 * BN;                          // two accumulators
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024;
constexpr long long WAIT_LIMIT = 4000000000ll;                  // ~2 s of clock

struct Sched {
    int S, s0, groups, nkb;     // diagonals s0 .. 2S-2 are computed
    int64_t m, n, tiles_n2;     // tiles_n2: groups of CC 256-column tiles
    int64_t nitems;             // (2 x 2 tile block, diagonal group) work items
};

// diagonal s of this CTA: pairs u in [u0, u1]; steps = pairs x k-blocks
__device__ __forceinline__ void diag_range(int s, int S, int &u0, int &u1)
{
    u0 = s - (S - 1) > 0 ? s - (S - 1) : 0;
    u1 = s < S - 1 ? s : S - 1;
}

// acc[q] += column q of the accumulator for q < EPI_COLS (16 at a time)
template <int Q>
__device__ __forceinline__ void drain_columns(uint32_t taddr, int32_t (&acc)[EPI_COLS])
{
    if constexpr (Q < EPI_COLS) {
        tc::tmem_ld16_add_i32<Q>(taddr + Q, acc);
        drain_columns<Q + 16>(taddr, acc);
    }
}

// row[q] (int64) = / += acc[q] for q < valid, 16 columns per block
template <int Q>
__device__ __forceinline__ void flush_columns(long long *row, const int32_t (&acc)[EPI_COLS], int valid, bool first)
{
    if constexpr (Q < EPI_COLS) {
        tc::flush16_i64<Q>(row, acc, valid, first);
        flush_columns<Q + 16>(row, acc, valid, first);
    }
}

}  // namespace

__global__ void __launch_bounds__(THREADS, 1)
split_slice_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                      Sched sc, long long *__restrict__ D, DevStatus *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *ring = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = tc::cluster_rank();                   // cr * CC + cc
    const uint32_t cr = rank / CC, cc = rank % CC;
    const uint16_t mask_a = (uint16_t)(((1u << CC) - 1u) << (cr * CC));   // CTAs sharing this A tile
    uint16_t mask_b = 0;                                                  // CTAs sharing this B tile
    for (int r = 0; r < CR; ++r) mask_b |= (uint16_t)(1u << (r * CC + cc));
    // persistent clusters: work items (CR x CC tile block, diagonal group) are
    // taken round-robin; every role walks the same sequence
    const int64_t cl0 = blockIdx.x / CSIZE, ncl = gridDim.x / CSIZE;
    // (quads vary fastest: clusters running at the same time walk the same
    // diagonals on neighbouring blocks and share operand tiles through L2)
    auto item = [&](int64_t it, int64_t &i0, int64_t &j0) -> int {
        const int64_t quads = sc.nitems / sc.groups;
        const int64_t quad = it % quads;
        i0 = (CR * (quad / sc.tiles_n2) + cr) * BM;
        j0 = (CC * (quad % sc.tiles_n2) + cc) * BN;
        return (int)(it / quads);
    };
    const int S = sc.S, nkb = sc.nkb;

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            tc::mbar_init(&full_bar[st], 1);
            tc::mbar_init(&empty_bar[st], CR + CC - 1); // this CTA and its peers consumed it
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&accf_bar[b], 1);
            tc::mbar_init(&acce_bar[b], EPI_WARPS);
        }
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_fence_init();
        abort_flag = 0;
    }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, TMEM_COLS);
    tc::fence_before_sync();
    tc::cluster_sync();                                 // barriers of both CTAs initialised
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    auto fail = [&]() {
        abort_flag = 1;
        if (status) atomicOr(&status->flags, ST_TIMEOUT);
    };

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            tc::prefetch_map(&map_a);
            tc::prefetch_map(&map_b);
            uint32_t g = 0;
            for (int64_t it = cl0; it < sc.nitems && !abort_flag; it += ncl) {
            int64_t i0, j0;
            const int grp = item(it, i0, j0);
            for (int s = sc.s0 + grp; s <= 2 * S - 2 && !abort_flag; s += sc.groups) {
                int u0, u1;
                diag_range(s, S, u0, u1);
                const int total = (u1 - u0 + 1) * nkb;
                for (int t = 0; t < total; ++t, ++g) {
                    const uint32_t st = g % STAGES, ph = (g / STAGES) & 1u;
                    if (!tc::mbar_wait(&empty_bar[st], ph ^ 1u, &abort_flag, WAIT_LIMIT)) { fail(); break; }
                    const int u = u0 + t / nkb, kb = t % nkb;
                    uint8_t *sa = ring + st * STAGE_BYTES, *sb = sa + A_BYTES;
                    tc::mbar_expect_tx(&full_bar[st], STAGE_BYTES);
                    tc::tma_load_2d_mc(sa + cc * (A_BYTES / CC), &map_a, kb * BK,
                                       (int32_t)(u * sc.m + i0 + cc * (BM / CC)), &full_bar[st], mask_a);
                    tc::tma_load_2d_mc(sb + cr * (B_BYTES / CR), &map_b, kb * BK,
                                       (int32_t)((s - u) * sc.n + j0 + cr * (BN / CR)), &full_bar[st], mask_b);
                }
            }
            }
            if (!abort_flag) {
                // both CTAs' consumption of the last fills has reached this CTA
                for (uint32_t k = g > STAGES ? g - STAGES : 0; k < g; ++k)
                    if (!tc::mbar_wait(&empty_bar[k % STAGES], (k / STAGES) & 1u, &abort_flag, WAIT_LIMIT)) {
                        fail();
                        break;
                    }
            }
            if (abort_flag) {
                // unwinding: let the copies still in flight land (bounded)
                for (uint32_t k = g > STAGES ? g - STAGES : 0; k < g; ++k)
                    tc::mbar_wait(&full_bar[k % STAGES], (k / STAGES) & 1u, nullptr, 200000000ll);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16_f32(BM, BN);
            uint32_t g = 0, c = 0;
            for (int64_t it = cl0; it < sc.nitems && !abort_flag; it += ncl) {
            int64_t i0, j0;
            const int grp = item(it, i0, j0);
            for (int s = sc.s0 + grp; s <= 2 * S - 2 && !abort_flag; s += sc.groups) {
                int u0, u1;
                diag_range(s, S, u0, u1);
                const int total = (u1 - u0 + 1) * nkb;
                bool ok = true;
                for (int t = 0; t < total && ok; ++t, ++g) {
                    const uint32_t buf = c & 1u;
                    const bool first = (t % KB_PER_CHUNK) == 0;
                    const bool last = (t % KB_PER_CHUNK) == KB_PER_CHUNK - 1 || t == total - 1;
                    if (first) {
                        if (!tc::mbar_wait(&acce_bar[buf], ((c >> 1) & 1u) ^ 1u, &abort_flag, WAIT_LIMIT)) {
                            fail();
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                    }
                    const uint32_t st = g % STAGES, ph = (g / STAGES) & 1u;
                    if (!tc::mbar_wait(&full_bar[st], ph, &abort_flag, WAIT_LIMIT)) { fail(); ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t sa = tc::saddr(ring + st * STAGE_BYTES), sb = sa + A_BYTES;
                    const uint32_t d = tmem + buf * BN;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        tc::mma_f16(d, tc::desc_k128(sa + 32 * k), tc::desc_k128(sb + 32 * k), idesc,
                                    (first && k == 0) ? 0u : 1u);
                    tc::mma_commit_mc(&empty_bar[st], mask_a | mask_b);   // self and its peers
                    if (last) {
                        tc::mma_commit(&accf_bar[buf]);             // the chunk is complete
                        ++c;
                    }
                }
                if (!ok) break;
            }
            }
            if (abort_flag) {
                // unwinding: every MMA issued so far completes before the
                // tensor memory is released (bounded)
                tc::mma_commit(&drain_bar);
                tc::mbar_wait(&drain_bar, 0u, nullptr, 200000000ll);
            }
        }
    } else {
        // --------------------------------------------------------- epilogue
        const int ew = warp - 2;
        const int quarter = warp & 3;                               // TMEM lanes of this warp
        const int part = ew >> 2;                                   // column range of the tile
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        int32_t acc[EPI_COLS];
        uint32_t c = 0;
        for (int64_t it = cl0; it < sc.nitems && !abort_flag; it += ncl) {
        int64_t i0, j0;
        const int grp = item(it, i0, j0);
        const int64_t i = i0 + quarter * 32 + lane;
        for (int s = sc.s0 + grp; s <= 2 * S - 2 && !abort_flag; s += sc.groups) {
            int u0, u1;
            diag_range(s, S, u0, u1);
            const int total = (u1 - u0 + 1) * nkb;
            const int nch = (total + KB_PER_CHUNK - 1) / KB_PER_CHUNK;
            long long *Ds = D + (int64_t)(s - sc.s0) * sc.m * sc.n;
            // segments of at most 255 chunks: int32 sums, then one int64 flush
            for (int seg = 0; seg < nch && !abort_flag; seg += CHUNKS_PER_I32) {
                const int seg_end = seg + CHUNKS_PER_I32 < nch ? seg + CHUNKS_PER_I32 : nch;
#pragma unroll
                for (int q = 0; q < EPI_COLS; ++q) acc[q] = 0;
                for (int ch = seg; ch < seg_end; ++ch, ++c) {
                    const uint32_t buf = c & 1u;
                    if (!tc::mbar_wait(&accf_bar[buf], (c >> 1) & 1u, &abort_flag, WAIT_LIMIT)) { fail(); break; }
                    tc::fence_after_sync();
                    drain_columns<0>(tmem + lane_addr + buf * BN + part * EPI_COLS, acc);
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&acce_bar[buf]);
                }
                if (abort_flag) break;
                if (i < sc.m) {
                    // first flush of the diagonal stores, later ones add (no read-back)
                    const int64_t jb = j0 + part * EPI_COLS;
                    const int64_t left = sc.n - jb;
                    flush_columns<0>(Ds + i * sc.n + jb, acc, (int)(left < EPI_COLS ? left : EPI_COLS), seg == 0);
                }
            }
        }
        }
    }

    tc::fence_before_sync();
    tc::cluster_sync();                                 // no multicast or arrival still bound for this CTA
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_free(tmem, TMEM_COLS);
    }
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// rows x lp fp16 matrix (K contiguous), boxes of box_rows x 64 with the
// 128-byte swizzle; reads past the edges return zeros
bool make_map(CUtensorMap *map, const __half *base, int64_t rows, int64_t lp, uint32_t box_rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)lp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)lp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    const cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// One CTA waits, through the bounded wait every mbarrier wait of the split
// and TMA-staged Block kernels uses, on an mbarrier that nothing completes:
// the wait gives up after about `limit` clock cycles, the timeout goes to
// the status word, and the CTA ends (nothing was issued, nothing is in
// flight).
__global__ void wait_selftest_kernel(DevStatus *status, long long limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    const bool got = tc::mbar_wait(&bar, 0u, nullptr, limit);
    if (__syncthreads_or(!got) && threadIdx.x == 0) atomicOr(&status->flags, ST_TIMEOUT);
}

void launch_wait_selftest(DevStatus *st, long long cycles, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 128, 0, s>>>(st, cycles);
}

bool limb_map(CUtensorMap *map, const BMat &M, int64_t batch, int64_t rows, int64_t cols, int L,
              uint32_t box_x, uint32_t box_y)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || batch < 1 || rows < 1 || cols < 1 || L < 1 || L > 256) return false;
    if (((uintptr_t)M.limb & 15) || (M.ld & 1) || (M.plane & 1)) return false;
    if (batch > 1 && M.bs_limb <= 0) return false;
    const int64_t bs = batch > 1 ? M.bs_limb : M.plane * L;
    if (bs & 1) return false;
    const int64_t lim = (int64_t)1 << 37;               // byte strides below 2^40
    if (M.ld >= lim || M.plane >= lim || bs >= lim) return false;
    if (cols > 0xffffffffll || rows > 0xffffffffll || batch > 0xffffffffll) return false;
    if (box_x == 0 || box_y == 0 || box_x > 256 || box_y > 256 || (box_x * 8) % 16) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)L, (cuuint64_t)batch};
    const cuuint64_t strides[3] = {(cuuint64_t)M.ld * 8, (cuuint64_t)M.plane * 8, (cuuint64_t)bs * 8};
    const cuuint32_t box[4] = {box_x, box_y, (cuuint32_t)L, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUtensorMap tmp;
    if (enc(&tmp, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, M.limb, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    *map = tmp;
    return true;
}

int launch_split_slices(const __half *pa, const __half *pb, int64_t m, int64_t l, int64_t n, int p,
                        int s0, long long *D, DevStatus *st, cudaStream_t s)
{
    const int S = split_digits(p);
    if (s0 < 0 || s0 > 2 * S - 2) return MP_ERR_ARG;
    const int64_t lp = split_lpad(l);
    // TMA: 16-byte aligned bases and row strides (lp is a multiple of 32)
    if (((uintptr_t)pa & 15) || ((uintptr_t)pb & 15) || (lp * 2) % 16) return MP_ERR_ARG;
    if ((int64_t)S * m > 0x7fffffff || (int64_t)S * n > 0x7fffffff) return MP_ERR_ARG;
    // the TMA loads below are multicast within a cluster: only this GPU's
    // own device memory may sit under the tensor maps
    if (!on_current_device(pa) || !on_current_device(pb)) return MP_ERR_ARG;
    CUtensorMap ma, mb;
    if (!make_map(&ma, pa, (int64_t)S * m, lp, BM / CC) || !make_map(&mb, pb, (int64_t)S * n, lp, BN / CR)) {
        if (std::getenv("MPGEMM_DEBUG")) std::fprintf(stderr, "split: tensor map encoding failed\n");
        return MP_ERR_UNSUPPORTED;
    }
    // once per process (one GPU per process): the shared-memory opt-in and
    // the number of clusters resident at once
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int resident = 0;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(split_slice_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SMEM_BYTES);
        if (attr_err != cudaSuccess) return;
        cudaLaunchConfig_t q = {};
        q.blockDim = dim3(THREADS);
        q.dynamicSmemBytes = SMEM_BYTES;
        q.gridDim = dim3(CSIZE * (152 / CSIZE));
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = CSIZE;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&resident, split_slice_tc_kernel, &q) != cudaSuccess || resident <= 0) {
            (void)cudaGetLastError();                   // clear a failed query
            resident = 144 / CSIZE;
        }
    });
    if (attr_err != cudaSuccess) {
        if (std::getenv("MPGEMM_DEBUG"))
            std::fprintf(stderr, "split: shared memory attribute: %s\n", cudaGetErrorString(attr_err));
        return MP_ERR_CUDA;
    }
    Sched sc;
    sc.S = S;
    sc.s0 = s0;
    sc.nkb = (int)((lp + BK - 1) / BK);
    sc.m = m;
    sc.n = n;
    sc.tiles_n2 = (n + CC * BN - 1) / (CC * BN);
    const int64_t quads = ((m + CR * BM - 1) / (CR * BM)) * sc.tiles_n2;   // CR x CC tile blocks
    // One resident cluster of CSIZE CTAs per CSIZE SMs (as many as fit at once); the
    // diagonals of a block are spread over groups until there are about
    // eight work items per cluster, so that the round-robin leaves little
    // imbalance at the end.
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr_cl[1];
    attr_cl[0].id = cudaLaunchAttributeClusterDimension;
    attr_cl[0].val.clusterDim.x = CSIZE;
    attr_cl[0].val.clusterDim.y = 1;
    attr_cl[0].val.clusterDim.z = 1;
    cfg.attrs = attr_cl;
    cfg.numAttrs = 1;
    const int64_t clusters = resident;
    int groups = 1;
    while (quads * groups < 8 * clusters && groups * 2 <= 2 * S - 1 - s0) groups *= 2;
    sc.groups = groups;
    sc.nitems = quads * groups;
    const int64_t ncl = sc.nitems < clusters ? sc.nitems : clusters;
    cfg.gridDim = dim3((unsigned)(CSIZE * ncl));
    cudaLaunchKernelEx(&cfg, split_slice_tc_kernel, ma, mb, sc, D, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && std::getenv("MPGEMM_DEBUG"))
        std::fprintf(stderr, "split: slice kernel launch failed: %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? MP_OK : MP_ERR_CUDA;
}

}  // namespace mpg
