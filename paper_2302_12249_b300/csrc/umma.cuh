// umma.cuh -- the sm_100-family primitives used by the deferred MLP: tcgen05.mma (one elected
// thread issues a CTA-wide M = 128 MMA), its A operand and accumulator in tensor memory (TMEM,
// written by tcgen05.st and read back by tcgen05.ld), the mbarrier that tcgen05.commit signals
// when the MMAs are done, and the bulk (TMA) copy that brings the weights into shared memory.
//
// The B operand (the weights) lives in shared memory in the canonical K-major layout without
// swizzle: an R x K tile of 16-bit elements is made of 8-row x 16-byte "core matrices"; element
// (r, k) sits at
//     (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2
// with LBO = 128 (core matrices adjacent along K) and SBO = (K / 8) * 128 (the next 8 rows).
// The accumulator of an M = 128 MMA (cta_group::1) holds row m in TMEM lane m and column n in
// TMEM column n; warp w of the CTA reads lanes 32 w .. 32 w + 31.
#pragma once

#include <stdint.h>

namespace merf {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) in a K-major no-swizzle tile of K columns.
__device__ __forceinline__ constexpr int kmajor_offset(int r, int k, int K)
{
    return (r / 8) * (K / 8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor version 1,
// base offset 0, no swizzle.
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both FP16 (bf16 = false) or
// both BF16, K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N, bool bf16)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Whole warp: allocate `ncols` TMEM columns (a power of two >= 32); the address lands in *slot.
template <int ncols>
__device__ __forceinline__ void tmem_alloc(uint32_t *slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "n"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

template <int ncols>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(ncols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Orders this thread's generic-proxy shared-memory accesses before later async-proxy ones: operand
// writes before the tensor cores read them, earlier reads before a bulk copy overwrites them.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (TMEM) = A B (+ D if accumulate), with A in tensor memory (row m of A in TMEM lane m, its
// 16-bit elements (k, k + 1) in one 32-bit column, element k in the low half; a_tmem: the column
// of element 0) and B in shared memory (descriptor b_desc); one thread issues it for the CTA.
__device__ __forceinline__ void umma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// The mbarrier gets one arrival when every MMA this thread issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with parity `parity` to complete; false once `limit_ns` nanoseconds of the
// global timer have passed without it (each try_wait may suspend the thread for a while before it
// reports, so the clock is read after every poll), or after `max_polls` polls should the timer
// not advance.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t limit_ns, int max_polls = 1 << 26)
{
    const uint64_t t0 = globaltimer_ns();
    for (int it = 0; it < max_polls; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_addr(mbar)), "r"(parity)
                     : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// One bulk (TMA, untiled) copy of `bytes` from global to shared memory, completing on `mbar`
// (count 1: this thread's arrival plus the bytes).  Both addresses 16-byte aligned, bytes a
// multiple of 16.  One thread calls it.
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gsrc, uint32_t bytes, uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(smem_dst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

// Columns col .. col + 15 of this thread's TMEM lane (warp w: lanes 32 w + lane).
__device__ __forceinline__ void tmem_ld16(uint32_t tmem, int col, float v[16])
{
    const uint32_t addr = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16) + (uint32_t)col;
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// Columns col .. col + 7 of this thread's TMEM lane from registers; tmem_st_wait() makes the
// thread's stores complete (before the barrier that precedes an MMA reading them).
__device__ __forceinline__ void tmem_st8(uint32_t tmem, int col, const uint32_t r[8])
{
    const uint32_t addr = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16) + (uint32_t)col;
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld4(uint32_t tmem, int col, float v[4])
{
    const uint32_t addr = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16) + (uint32_t)col;
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = __uint_as_float(r[c]);
}

}  // namespace merf
