// am_tcgen05.cuh -- inline-PTX building blocks of the tcgen05 kernels (sm_103a): mbarriers
// with bounded waits, 2-D TMA loads, shared-memory matrix descriptors for 128-byte-swizzled
// K-major tiles, the BF16 UMMA instruction descriptor, tcgen05.mma / commit / fences and TMEM
// loads.  Written from the PTX ISA's descriptions of these instructions.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace am {
namespace tc {

constexpr long long kWaitNs = 2000000000ll;    // 2 s limit on any pipeline wait
constexpr long long kDrainNs = 200000000ll;    // 0.2 s limit on the drain after an abort

__device__ __forceinline__ unsigned long long oz_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete, for at most `limit` ns, or until another
// role of the CTA has aborted.  On a time-out the CTA aborts and the host sees *err = 1.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *err,
                                          long long limit = kWaitNs)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = oz_now();
    while (!mbar_test(bar, parity)) {
        if (*abort) return false;
        if ((long long)(oz_now() - t0) > limit) {
            *abort = 1;
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// Wait without an abort check (after an abort: let what is in flight finish), at most `limit` ns.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, long long limit)
{
    const unsigned long long t0 = oz_now();
    while (!mbar_test(bar, parity))
        if ((long long)(oz_now() - t0) > limit) return;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile whose rows are 128 bytes, written by TMA
// with the 128-byte swizzle: 8-row groups 1024 bytes apart (stride byte offset), descriptor
// version 1 (the tcgen05 family), layout type 2 = 128-byte swizzle.  The leading byte offset is
// not used by swizzled K-major layouts; successive K = 16 steps advance the start address by
// 32 bytes inside the swizzle atom.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The same product with the A operand kept in the tensor core's collector buffer: kind 1 reads A
// from shared memory and keeps it (fill), 2 reuses the kept A (use), 3 reuses it for the last
// time (lastuse).  Consecutive products with one A tile read it from shared memory once.
template <int KIND>
__device__ __forceinline__ void umma_bf16_collect(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                  uint32_t accumulate)
{
    if constexpr (KIND == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if constexpr (KIND == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// The products of one W_l plane s (its A tile at adesc) with the operand planes t = 0 .. NT - 1
// (B tiles bplane bytes apart from bdesc) into the accumulators of diagonals s + t, for the 4
// K = 16 steps of a staged chunk.  Per K step the A slice is read into the collector once and
// reused by the NT products.  Descriptor start addresses advance in 16-byte units.
template <int NT, int NCOL, int BPLANE>
__device__ __forceinline__ void issue_plane(uint32_t tmem, int s, uint64_t adesc, uint64_t bdesc, uint32_t acc0)
{
    constexpr uint32_t idesc = umma_idesc_bf16(128, NCOL);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = adesc + (uint64_t)(2 * kk);
        const uint32_t acc = (acc0 | kk) != 0 ? 1u : 0u;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const uint64_t bd = bdesc + (uint64_t)((t * BPLANE + 32 * kk) >> 4);
            const uint32_t d = tmem + (uint32_t)((s + t) * NCOL);
            if constexpr (NT == 1) umma_bf16(d, ad, bd, idesc, acc);
            else if (t == 0) umma_bf16_collect<1>(d, ad, bd, idesc, acc);
            else if (t + 1 < NT) umma_bf16_collect<2>(d, ad, bd, idesc, acc);
            else umma_bf16_collect<3>(d, ad, bd, idesc, acc);
        }
    }
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes; the caller waits (tcgen05.wait::ld)
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

}  // namespace tc
}  // namespace am
