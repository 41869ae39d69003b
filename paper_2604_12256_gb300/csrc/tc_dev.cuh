// tc_dev.cuh -- inline-PTX helpers of the tensor-core kernels (k_dense5.cu,
// k_dense_chunk.cu): shared-memory operand layout and descriptors for
// tcgen05.mma kind::tf32, TF32 rounding, bounded mbarrier polling, TMEM loads
// and bulk global -> shared copies completing on an mbarrier.
#pragma once

#include <cstdint>

namespace svs {

// Shared-memory operand layout: K-major, no swizzle.  A "core matrix" is 8
// rows x 16 bytes (4 TF32), stored as 128 contiguous bytes; core matrices are
// ordered with the row (M or N) direction fastest, so the row-direction step
// (SBO) is 128 B and the K-direction step (LBO) is rows/8 * 128 B.
__host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int k, int rows)
{
    return (uint32_t)(((k >> 2) * (rows >> 3) + (row >> 3)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version for tcgen05
    // base offset 0, lbo mode 0, layout type 0 (no swizzle)
    return d;
}

// instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_of(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(phase)
        : "memory");
    return ok != 0;
}

// poll an mbarrier phase at most `limit` times; false when the wait ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t phase, uint32_t limit)
{
    for (uint32_t it = 0; it <= limit; it++) {
        if (mbar_try_wait(addr, phase)) return true;
        __nanosleep(32);
    }
    return false;
}

// One try_wait that may suspend the thread until the phase completes or
// about `hint_ns` nanoseconds have passed (the hardware wakes it on
// completion, without a sleep-and-poll delay).
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t addr, uint32_t phase, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(phase), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// at most `limit` suspended tries of at most ~1 us each; false when the wait ran out
__device__ __forceinline__ bool mbar_wait_suspend(uint32_t addr, uint32_t phase, uint32_t limit)
{
    for (uint32_t it = 0; it <= limit; it++)
        if (mbar_try_wait_hint(addr, phase, 1000u)) return true;
    return false;
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count));
}

// One thread: announce `bytes` of bulk copies on the barrier's current phase
// and copy `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory in pieces of at most 8 KB.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    for (uint32_t o = 0; o < bytes; o += 8192) {
        const uint32_t len = bytes - o < 8192 ? bytes - o : 8192;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst + o),
            "l"((const char *)src + o), "r"(len), "r"(mbar)
            : "memory");
    }
}

// 32 consecutive TMEM columns of this warp's 32 lanes -> 32 registers
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&y)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]), "=r"(y[7]),
          "=r"(y[8]), "=r"(y[9]), "=r"(y[10]), "=r"(y[11]), "=r"(y[12]), "=r"(y[13]), "=r"(y[14]), "=r"(y[15]),
          "=r"(y[16]), "=r"(y[17]), "=r"(y[18]), "=r"(y[19]), "=r"(y[20]), "=r"(y[21]), "=r"(y[22]),
          "=r"(y[23]), "=r"(y[24]), "=r"(y[25]), "=r"(y[26]), "=r"(y[27]), "=r"(y[28]), "=r"(y[29]),
          "=r"(y[30]), "=r"(y[31])
        : "r"(taddr));
}

// 16 consecutive TMEM columns of this warp's 32 lanes -> 16 registers
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&y)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]), "=r"(y[7]),
          "=r"(y[8]), "=r"(y[9]), "=r"(y[10]), "=r"(y[11]), "=r"(y[12]), "=r"(y[13]), "=r"(y[14]), "=r"(y[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (TMEM) [+]= A (shared) . B (shared)^T, one tcgen05.mma issued by the
// calling thread
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            int accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// the MMAs issued so far by this thread arrive on the mbarrier when complete
__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

}  // namespace svs
