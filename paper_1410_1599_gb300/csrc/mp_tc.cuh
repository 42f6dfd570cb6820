// mp_tc.cuh -- Blackwell primitives in inline PTX for the split form's slice
// products: mbarriers with bounded waits, TMA tile loads, TMEM allocation,
// tcgen05.mma (kind::f16, fp32 accumulation in tensor memory) and
// tcgen05.ld.  Nothing here waits without a limit: a wait that runs out
// reports failure to the caller, which sets an error flag and unwinds.
#pragma once
#include <cstdint>
#include <cuda.h>

namespace mpg {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------------ mbarriers
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Wait for the phase with the given parity to complete; false after about
// `limit` clock cycles or when *abort (if given) is set by another thread.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const volatile int *abort,
                                          long long limit)
{
    const long long t0 = clock64();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 63u) {
            if (abort && *abort) return false;
            if (clock64() - t0 > limit) return false;
        }
    }
}

// ------------------------------------------------------------------ TMA
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

// a 4-D box (x innermost) of this CTA's tensor map into shared memory
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int32_t x, int32_t y, int32_t z,
                                            int32_t w, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(saddr(bar))
        : "memory");
}

// the same tile into the same shared-memory offset of every CTA in `mask`
// (cluster ranks); each destination's mbarrier at `bar`'s offset receives
// the byte count
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                               uint64_t *bar, uint16_t mask)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar)), "h"(mask)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// all threads of all CTAs of the cluster
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ----------------------------------------------------------------- TMEM
// Allocation by one whole warp; the base address lands in *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ------------------------------------------------------------- tcgen05.mma
// Shared-memory matrix descriptor of a K-major operand tile stored by TMA
// with the 128-byte swizzle: rows of 64 halves (128 B), 8-row swizzle atoms
// 1024 B apart (stride byte offset), start address advanced by 32 B per
// K = 16 step inside the atom.  Field layout: start >> 4 in [0,14), leading
// byte offset >> 4 in [16,30), stride byte offset >> 4 in [32,46), the
// descriptor version 1 in [46,48), base offset 0, swizzle mode 2 (128 B) in
// [61,64).
__device__ __forceinline__ uint64_t desc_k128(uint32_t smem_byte_addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_byte_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1), A and
// B fp16 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A * B^T for one M x N x 16 step, issued by one thread
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the mbarrier completes (one arrival) once every MMA issued so far by this
// thread has finished
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     saddr(bar))
                 : "memory");
}

// as mma_commit, arriving on the mbarrier at `bar`'s offset in every CTA of
// `mask`
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            saddr(bar)),
        "h"(mask)
        : "memory");
}

// 32 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// acc[O + e] += (int32) fp32 column e of 16 consecutive columns of this
// thread's TMEM lane, for e < 16; the values are exact integers, converted
// with round-to-nearest (a no-op on them).  Load, wait and accumulate in one
// block, so the loaded columns are consumed before the next load is issued.
template <int O, int N>
__device__ __forceinline__ void tmem_ld16_add_i32(uint32_t taddr, int32_t (&acc)[N])
{
    static_assert(O + 16 <= N, "range");
    asm volatile(
        "{\n\t.reg .f32 f<16>;\n\t.reg .s32 t;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{f0,f1,f2,f3,f4,f5,f6,f7,f8,f9,f10,f11,f12,f13,f14,f15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t"
        "cvt.rni.s32.f32 t, f0;  add.s32 %0, %0, t;\n\t"
        "cvt.rni.s32.f32 t, f1;  add.s32 %1, %1, t;\n\t"
        "cvt.rni.s32.f32 t, f2;  add.s32 %2, %2, t;\n\t"
        "cvt.rni.s32.f32 t, f3;  add.s32 %3, %3, t;\n\t"
        "cvt.rni.s32.f32 t, f4;  add.s32 %4, %4, t;\n\t"
        "cvt.rni.s32.f32 t, f5;  add.s32 %5, %5, t;\n\t"
        "cvt.rni.s32.f32 t, f6;  add.s32 %6, %6, t;\n\t"
        "cvt.rni.s32.f32 t, f7;  add.s32 %7, %7, t;\n\t"
        "cvt.rni.s32.f32 t, f8;  add.s32 %8, %8, t;\n\t"
        "cvt.rni.s32.f32 t, f9;  add.s32 %9, %9, t;\n\t"
        "cvt.rni.s32.f32 t, f10; add.s32 %10, %10, t;\n\t"
        "cvt.rni.s32.f32 t, f11; add.s32 %11, %11, t;\n\t"
        "cvt.rni.s32.f32 t, f12; add.s32 %12, %12, t;\n\t"
        "cvt.rni.s32.f32 t, f13; add.s32 %13, %13, t;\n\t"
        "cvt.rni.s32.f32 t, f14; add.s32 %14, %14, t;\n\t"
        "cvt.rni.s32.f32 t, f15; add.s32 %15, %15, t;\n\t}"
        : "+r"(acc[O + 0]), "+r"(acc[O + 1]), "+r"(acc[O + 2]), "+r"(acc[O + 3]), "+r"(acc[O + 4]),
          "+r"(acc[O + 5]), "+r"(acc[O + 6]), "+r"(acc[O + 7]), "+r"(acc[O + 8]), "+r"(acc[O + 9]),
          "+r"(acc[O + 10]), "+r"(acc[O + 11]), "+r"(acc[O + 12]), "+r"(acc[O + 13]), "+r"(acc[O + 14]),
          "+r"(acc[O + 15])
        : "r"(taddr));
}

// Columns O .. O+15 of a row of int32 sums to int64 memory row[O + e]
// (e < valid - O only): stored when `first`, else added with a reduction
// (no read-back).  One asm block per 16 columns keeps the 64-bit temporaries
// out of the register budget.
template <int O, int N>
__device__ __forceinline__ void flush16_i64(long long *row, const int32_t (&acc)[N], int valid, bool first)
{
    static_assert(O + 16 <= N, "range");
    long long *r = row + O;
    const int v = valid - O;
    if (first)
        asm volatile(
            "{\n\t.reg .pred p;\n\t.reg .s64 t;\n\t"
        "setp.gt.s32 p, %17, 0; cvt.s64.s32 t, %0; @p st.global.s64 [%16+0], t;\n\t"
        "setp.gt.s32 p, %17, 1; cvt.s64.s32 t, %1; @p st.global.s64 [%16+8], t;\n\t"
        "setp.gt.s32 p, %17, 2; cvt.s64.s32 t, %2; @p st.global.s64 [%16+16], t;\n\t"
        "setp.gt.s32 p, %17, 3; cvt.s64.s32 t, %3; @p st.global.s64 [%16+24], t;\n\t"
        "setp.gt.s32 p, %17, 4; cvt.s64.s32 t, %4; @p st.global.s64 [%16+32], t;\n\t"
        "setp.gt.s32 p, %17, 5; cvt.s64.s32 t, %5; @p st.global.s64 [%16+40], t;\n\t"
        "setp.gt.s32 p, %17, 6; cvt.s64.s32 t, %6; @p st.global.s64 [%16+48], t;\n\t"
        "setp.gt.s32 p, %17, 7; cvt.s64.s32 t, %7; @p st.global.s64 [%16+56], t;\n\t"
        "setp.gt.s32 p, %17, 8; cvt.s64.s32 t, %8; @p st.global.s64 [%16+64], t;\n\t"
        "setp.gt.s32 p, %17, 9; cvt.s64.s32 t, %9; @p st.global.s64 [%16+72], t;\n\t"
        "setp.gt.s32 p, %17, 10; cvt.s64.s32 t, %10; @p st.global.s64 [%16+80], t;\n\t"
        "setp.gt.s32 p, %17, 11; cvt.s64.s32 t, %11; @p st.global.s64 [%16+88], t;\n\t"
        "setp.gt.s32 p, %17, 12; cvt.s64.s32 t, %12; @p st.global.s64 [%16+96], t;\n\t"
        "setp.gt.s32 p, %17, 13; cvt.s64.s32 t, %13; @p st.global.s64 [%16+104], t;\n\t"
        "setp.gt.s32 p, %17, 14; cvt.s64.s32 t, %14; @p st.global.s64 [%16+112], t;\n\t"
        "setp.gt.s32 p, %17, 15; cvt.s64.s32 t, %15; @p st.global.s64 [%16+120], t;\n\t"
            "}" ::"r"(acc[O + 0]), "r"(acc[O + 1]), "r"(acc[O + 2]), "r"(acc[O + 3]), "r"(acc[O + 4]),
            "r"(acc[O + 5]), "r"(acc[O + 6]), "r"(acc[O + 7]), "r"(acc[O + 8]), "r"(acc[O + 9]),
            "r"(acc[O + 10]), "r"(acc[O + 11]), "r"(acc[O + 12]), "r"(acc[O + 13]), "r"(acc[O + 14]),
            "r"(acc[O + 15]), "l"(r), "r"(v)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t.reg .s64 t;\n\t"
        "setp.gt.s32 p, %17, 0; cvt.s64.s32 t, %0; @p red.global.add.u64 [%16+0], t;\n\t"
        "setp.gt.s32 p, %17, 1; cvt.s64.s32 t, %1; @p red.global.add.u64 [%16+8], t;\n\t"
        "setp.gt.s32 p, %17, 2; cvt.s64.s32 t, %2; @p red.global.add.u64 [%16+16], t;\n\t"
        "setp.gt.s32 p, %17, 3; cvt.s64.s32 t, %3; @p red.global.add.u64 [%16+24], t;\n\t"
        "setp.gt.s32 p, %17, 4; cvt.s64.s32 t, %4; @p red.global.add.u64 [%16+32], t;\n\t"
        "setp.gt.s32 p, %17, 5; cvt.s64.s32 t, %5; @p red.global.add.u64 [%16+40], t;\n\t"
        "setp.gt.s32 p, %17, 6; cvt.s64.s32 t, %6; @p red.global.add.u64 [%16+48], t;\n\t"
        "setp.gt.s32 p, %17, 7; cvt.s64.s32 t, %7; @p red.global.add.u64 [%16+56], t;\n\t"
        "setp.gt.s32 p, %17, 8; cvt.s64.s32 t, %8; @p red.global.add.u64 [%16+64], t;\n\t"
        "setp.gt.s32 p, %17, 9; cvt.s64.s32 t, %9; @p red.global.add.u64 [%16+72], t;\n\t"
        "setp.gt.s32 p, %17, 10; cvt.s64.s32 t, %10; @p red.global.add.u64 [%16+80], t;\n\t"
        "setp.gt.s32 p, %17, 11; cvt.s64.s32 t, %11; @p red.global.add.u64 [%16+88], t;\n\t"
        "setp.gt.s32 p, %17, 12; cvt.s64.s32 t, %12; @p red.global.add.u64 [%16+96], t;\n\t"
        "setp.gt.s32 p, %17, 13; cvt.s64.s32 t, %13; @p red.global.add.u64 [%16+104], t;\n\t"
        "setp.gt.s32 p, %17, 14; cvt.s64.s32 t, %14; @p red.global.add.u64 [%16+112], t;\n\t"
        "setp.gt.s32 p, %17, 15; cvt.s64.s32 t, %15; @p red.global.add.u64 [%16+120], t;\n\t"
            "}" ::"r"(acc[O + 0]), "r"(acc[O + 1]), "r"(acc[O + 2]), "r"(acc[O + 3]), "r"(acc[O + 4]),
            "r"(acc[O + 5]), "r"(acc[O + 6]), "r"(acc[O + 7]), "r"(acc[O + 8]), "r"(acc[O + 9]),
            "r"(acc[O + 10]), "r"(acc[O + 11]), "r"(acc[O + 12]), "r"(acc[O + 13]), "r"(acc[O + 14]),
            "r"(acc[O + 15]), "l"(r), "r"(v)
            : "memory");
}

__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace tc
}  // namespace mpg
