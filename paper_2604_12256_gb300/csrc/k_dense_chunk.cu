// k_dense_chunk.cu -- fused dense 5-qubit blocks applied inside the
// cache-blocked sweep (K6 inside K4): a chunk of 2^12 complex64 amplitudes is
// read from HBM once, takes every block of its sweep on the tensor cores
// while it stays in shared memory, and is written back once.  This is the
// all-in-one branch of Algorithm 5 for the dense blocks of Algorithm 4's
// fusion mode; the paper's argument against leaving the cached state for a
// separate GEMM (its hybrid BatchMV scheme, Algorithm 3) is what it follows.
//
// Per block, the chunk is a 32 x 128 complex matrix X (rows: the block's five
// target bits; columns: the other seven chunk bits) and Y = U X is the real
// GEMM D(128 x 64) = A(128 x 64) B(64 x 64)^T with A = [Xr Xi]^T and B the
// real embedding [[Ur, -Ui], [Ui, Ur]], in split-TF32 (A = Ahi + Alo,
// B = Bhi + Blo; Ahi.Bhi into one TMEM accumulator, Ahi.Blo + Alo.Bhi into a
// second, summed in FP32 at the end; Ahi.Bhi and Ahi.Blo are one product of
// N = 128 against the stacked [Bhi; Blo], so Ahi is read once).  Thread t
// owns column t: it gathers the column from the chunk, writes its split row
// of A, and after the MMAs reads row t of D from TMEM (its lane) and scatters
// it back into the chunk.
//
// Shared memory per CTA (two CTAs of 128 threads per SM): A hi (32 KB), A lo (32 KB, which
// also holds the chunk itself between blocks: 4096 complex64 amplitudes in
// the swizzled slot layout of dense_prog.h), the block's B image (32 KB,
// brought in by a bulk copy while the previous block's epilogue runs), two
// mbarriers.  TMEM: 128 columns (the two accumulators of 64).  Every wait is
// bounded: a wait that runs out sets *status = 1, lets the copies and MMAs in
// flight finish (again bounded), frees TMEM and returns.
#include <algorithm>
#include <cstdint>

#include "dense_prog.h"
#include "kernels.h"
#include "tc_dev.cuh"

namespace svs {
using namespace dprog;

namespace {

constexpr int kThreads = kCols;               // one thread per column
constexpr int kTmemCols = 128;                // two accumulators of N = 64
constexpr uint32_t kWaitPolls = 1u << 20;      // suspended tries of <= ~1 us

struct DcSmem {
    uint32_t a_hi[kCols * 64];
    uint32_t a_lo[kCols * 64];   // also the chunk: float2 slots 0..4095
    uint32_t b[2 * 64 * 64];     // B hi (rows 0..63) over B lo (rows 64..127)
    uint32_t rec[kMaxBlocks * kBlkWords];   // the sweep's block records
    uint64_t mbar_mma;
    uint64_t mbar_b;
    uint32_t tmem_addr;
    int abort_;
};

__device__ __forceinline__ uint64_t deposit_free(uint64_t v, uint64_t mask)
{
    uint64_t r = 0;
    while (mask) {
        const uint64_t low = mask & (~mask + 1);
        if (v & 1) r |= low;
        v >>= 1;
        mask ^= low;
    }
    return r;
}

}  // namespace

// Thread t serves column t (MMA row and TMEM lane t: warp w reads lanes
// 32 w ... 32 w + 31).
__global__ void __launch_bounds__(kThreads, 2) k_dense_chunk_tc(float2 *__restrict__ a, int n,
                                                                 const uint32_t *__restrict__ prog, int *status,
                                                                 uint32_t wait_limit, int skip_mma)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    DcSmem &sm = *reinterpret_cast<DcSmem *>(smraw);
    float2 *chunk = reinterpret_cast<float2 *>(sm.a_lo);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int t = tid;
    const int nblk = (int)prog[H_NBLK];
    const uint32_t *bimg = prog + prog[H_BOFF];
    const uint64_t freem = (uint64_t)prog[H_FREE_LO] | ((uint64_t)prog[H_FREE_HI] << 32);

    // this thread's share of a chunk: pieces P = 128 p + tid (p = 0..15) of
    // two amplitudes each, chunk index 2P: chunk bits 1..7 from tid, 8..11
    // from p; lanes 0..7 read one 128-byte segment.  The swizzle is linear,
    // so slot(2P) = slot(2 tid) ^ slot(256 p) = slot(2 tid) ^ 257 p.
    uint64_t tglob = 0;
#pragma unroll
    for (int i = 0; i < 7; i++)
        if ((tid >> i) & 1) tglob |= 1ull << prog[H_QIN + 1 + i];
    uint64_t pq[4];
#pragma unroll
    for (int i = 0; i < 4; i++) pq[i] = 1ull << prog[H_QIN + 8 + i];
    auto poff = [&](int p) {
        return ((p & 1) ? pq[0] : 0ull) | ((p & 2) ? pq[1] : 0ull) | ((p & 4) ? pq[2] : 0ull) |
               ((p & 8) ? pq[3] : 0ull);
    };
    const uint32_t tslot = slot(2u * (uint32_t)tid);

    for (int i = tid; i < nblk * kBlkWords; i += kThreads) sm.rec[i] = prog[H_SIZE + i];
    if (tid == 0) {
        sm.abort_ = 0;
        mbar_init((uint32_t)__cvta_generic_to_shared(&sm.mbar_mma), 1);
        mbar_init((uint32_t)__cvta_generic_to_shared(&sm.mbar_b), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&sm.tmem_addr)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_addr;
    const uint32_t mbar_mma = (uint32_t)__cvta_generic_to_shared(&sm.mbar_mma);
    const uint32_t mbar_b = (uint32_t)__cvta_generic_to_shared(&sm.mbar_b);
    // the B image holds 128 rows: Bhi (rows 0..63) then Blo (64..127)
    constexpr uint32_t idesc128 = tf32_idesc(kCols, 128), idesc64 = tf32_idesc(kCols, 64);
    constexpr uint32_t lbo_a = (kCols / 8) * 128, lbo_b = (128 / 8) * 128, sbo = 128;
    // operand descriptors; a K-step of 8 moves the start address by two
    // core-matrix columns (2 LBO, in 16-byte units in the low field)
    const uint64_t d_ahi = smem_desc((uint32_t)__cvta_generic_to_shared(sm.a_hi), lbo_a, sbo);
    const uint64_t d_alo = smem_desc((uint32_t)__cvta_generic_to_shared(sm.a_lo), lbo_a, sbo);
    const uint32_t b_smem = (uint32_t)__cvta_generic_to_shared(sm.b);
    const uint64_t d_b = smem_desc(b_smem, lbo_b, sbo);

    // thread 0 waits on the barriers and tracks what it has in flight
    uint32_t b_phase = 0, mma_phase = 0;
    bool b_inflight = false, mma_inflight = false;
    if (tid == 0) {
        bulk_g2s(b_smem, bimg, kBImgWords * 4, mbar_b);
        b_inflight = true;
    }

    const int64_t nch = (int64_t)1 << (n - kC);
    float4 nx[16];
    auto load_chunk = [&](int64_t ch) {
        const float4 *g = reinterpret_cast<const float4 *>(a);
        const uint64_t base = deposit_free((uint64_t)ch, freem) | tglob;
#pragma unroll
        for (int p = 0; p < 16; p++) nx[p] = __ldcs(g + ((base | poff(p)) >> 1));
    };
    if ((int64_t)blockIdx.x < nch) load_chunk(blockIdx.x);

    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const uint64_t base = deposit_free((uint64_t)ch, freem) | tglob;
        // the loaded chunk into its slots (pairs stay in one 16-byte unit,
        // swapped when the swizzle moves amplitude 2P to an odd slot)
#pragma unroll
        for (int p = 0; p < 16; p++) {
            const uint32_t s = tslot ^ (uint32_t)(257 * p);
            const float4 v = nx[p];
            *reinterpret_cast<float4 *>(&chunk[s & ~1u]) = (s & 1) ? make_float4(v.z, v.w, v.x, v.y) : v;
        }
        __syncthreads();
        if (ch + gridDim.x < nch) load_chunk(ch + gridDim.x);   // in flight through the blocks

        for (int blk = 0; blk < nblk; blk++) {
            const uint32_t *rec = sm.rec + blk * kBlkWords;
            uint32_t rowbase = 0;
            {
                const uint4 r0 = *reinterpret_cast<const uint4 *>(rec);       // tmask, rowslot 0..2
                const uint4 r1 = *reinterpret_cast<const uint4 *>(rec + 4);   // rowslot 3..6
                const uint32_t rs[7] = {r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
                for (int i = 0; i < 7; i++)
                    if ((t >> i) & 1) rowbase ^= rs[i];
            }
            // slot of (column t, target index j) = rowbase ^ toff[j]; the
            // offsets are read four at a time (broadcast 128-bit loads)
            const uint4 *toff4 = reinterpret_cast<const uint4 *>(rec + B_TOFF);
            // ---- gather column t, split into TF32 hi + lo, write row t of A
            {
                float xr[32], xi[32];
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const uint4 o = toff4[q];
                    const float2 v0 = chunk[rowbase ^ o.x], v1 = chunk[rowbase ^ o.y];
                    const float2 v2 = chunk[rowbase ^ o.z], v3 = chunk[rowbase ^ o.w];
                    xr[4 * q] = v0.x, xi[4 * q] = v0.y, xr[4 * q + 1] = v1.x, xi[4 * q + 1] = v1.y;
                    xr[4 * q + 2] = v2.x, xi[4 * q + 2] = v2.y, xr[4 * q + 3] = v3.x, xi[4 * q + 3] = v3.y;
                }
                __syncthreads();   // every column read before A (over the chunk) is written
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    // K = 4 q .. 4 q + 3: real parts (q < 8), then imaginary
                    uint32_t hv[4], lv[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const float x = q < 8 ? xr[4 * q + e] : xi[4 * (q - 8) + e];
                        // hi: x truncated to TF32; lo = x - hi exactly (the
                        // tensor core reads its leading 11 bits)
                        hv[e] = __float_as_uint(x) & 0xffffe000u;
                        lv[e] = __float_as_uint(x - __uint_as_float(hv[e]));
                    }
                    const uint32_t o = kmajor_off(t, 4 * q, kCols) >> 2;
                    *reinterpret_cast<uint4 *>(&sm.a_hi[o]) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                    *reinterpret_cast<uint4 *>(&sm.a_lo[o]) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                // (a sweep of one block keeps its B image for every chunk)
                const bool ok = !b_inflight || mbar_wait_suspend(mbar_b, b_phase, wait_limit);
                if (ok) {
                    if (b_inflight) b_phase ^= 1;
                    b_inflight = false;
                }
                if (ok && !skip_mma) {
                    // Ahi [Bhi; Blo]^T in one N = 128 product: big = Ahi Bhi^T
                    // (columns 0..63), Ahi Blo^T (64..127); then Alo Bhi^T
                    // added to columns 64..127 (the small terms, kept apart
                    // from the big ones); 8 K-steps of 8 each
#pragma unroll
                    for (int ks = 0; ks < 8; ks++)
                        tc_mma_tf32(tmem, d_ahi + (uint64_t)((ks * 2 * lbo_a) >> 4),
                                    d_b + (uint64_t)((ks * 2 * lbo_b) >> 4), idesc128, ks > 0 ? 1 : 0);
#pragma unroll
                    for (int ks = 0; ks < 8; ks++)
                        tc_mma_tf32(tmem + 64, d_alo + (uint64_t)((ks * 2 * lbo_a) >> 4),
                                    d_b + (uint64_t)((ks * 2 * lbo_b) >> 4), idesc64, 1);
                    tc_commit(mbar_mma);
                    mma_inflight = true;
                }
                // ---- wait for the products (bounded); only this thread waits
                bool done = false;
                if (ok) {
                    done = mbar_wait_suspend(mbar_mma, mma_phase, wait_limit);
                    if (done) {
                        mma_phase ^= 1;
                        mma_inflight = false;
                    }
                }
                if (!done) {
                    sm.abort_ = 1;
                } else {
                    // the next block's B (the first one again for the next
                    // chunk) comes in while this block's epilogue runs
                    const bool more = blk + 1 < nblk || ch + gridDim.x < nch;
                    if (nblk > 1 && more) {
                        bulk_g2s(b_smem, bimg + (size_t)((blk + 1) % nblk) * kBImgWords, kBImgWords * 4, mbar_b);
                        b_inflight = true;
                    }
                }
                tc_fence_after();
                tc_fence_before();
            }
            __syncthreads();
            tc_fence_after();
            if (sm.abort_) goto finish;
            // ---- epilogue: row t of D (TMEM lane t) back into the chunk
            {
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
                float yre[32];
                uint32_t bg[32], sm_[32];
                tmem_ld32(taddr, bg);
                tmem_ld32(taddr + 64, sm_);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int r = 0; r < 32; r++) yre[r] = __uint_as_float(bg[r]) + __uint_as_float(sm_[r]);
                tmem_ld32(taddr + 32, bg);
                tmem_ld32(taddr + 96, sm_);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const uint4 o = toff4[q];
                    const uint32_t so[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int r = 4 * q + e;
                        chunk[rowbase ^ so[e]] = make_float2(yre[r], __uint_as_float(bg[r]) + __uint_as_float(sm_[r]));
                    }
                }
            }
            // the chunk is complete, and every TMEM read is ordered before
            // the next block's MMAs
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
        // ---- the chunk back to HBM
        {
            float4 *g = reinterpret_cast<float4 *>(a);
#pragma unroll
            for (int p = 0; p < 16; p++) {
                const uint32_t s = tslot ^ (uint32_t)(257 * p);
                const float4 v = *reinterpret_cast<const float4 *>(&chunk[s & ~1u]);
                __stcs(g + ((base | poff(p)) >> 1), (s & 1) ? make_float4(v.z, v.w, v.x, v.y) : v);
            }
        }
        __syncthreads();   // every slot read before the next chunk is written
    }

finish:
    if (sm.abort_ && tid == 0) {
        atomicExch(status, 1);
        // let the copy and the products in flight land before TMEM and the
        // shared memory go away (bounded as well)
        if (b_inflight) mbar_wait_suspend(mbar_b, b_phase, wait_limit);
        if (mma_inflight) mbar_wait_suspend(mbar_mma, mma_phase, wait_limit);
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ------------------------------------------------------------ launchers
static cudaError_t dense_chunk_launch(void *a, int n, const uint32_t *prog, int *status, uint32_t wait_limit,
                                      int skip_mma, cudaStream_t st)
{
    if (n < kC || n > 40) return cudaErrorInvalidValue;
    if (((uintptr_t)prog & 15) != 0 || ((uintptr_t)a & 15) != 0) return cudaErrorMisalignedAddress;
    static bool attr = false;
    const size_t smem = sizeof(DcSmem);
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k_dense_chunk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // two CTAs per SM: 2 x 96 KB of shared memory, 2 x 128 TMEM columns
    const int64_t nch = (int64_t)1 << (n - kC);
    const int grid = (int)std::min<int64_t>(nch, (int64_t)device_sm_count() * 2);
    k_dense_chunk_tc<<<grid, kThreads, smem, st>>>((float2 *)a, n, prog, status, wait_limit, skip_mma);
    return counted(cudaGetLastError(), 1);
}

cudaError_t launch_dense_chunk(void *a, int n, const uint32_t *prog, int *status, cudaStream_t st)
{
    return dense_chunk_launch(a, n, prog, status, kWaitPolls, 0, st);
}

// Self-test of the bounded waits: no MMA is issued, so the first wait on the
// products runs out after wait_limit polls; *status becomes 1 and the state
// is not written (a chunk is stored only after its last block).
cudaError_t launch_dense_chunk_wait_selftest(void *a, int n, const uint32_t *prog, int *status, uint32_t wait_limit,
                                             cudaStream_t st)
{
    return dense_chunk_launch(a, n, prog, status, wait_limit, 1, st);
}

}  // namespace svs
