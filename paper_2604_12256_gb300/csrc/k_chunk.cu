// k_chunk.cu -- the cache-blocked chunk sweep (K4, the all-in-one branch of
// Algorithm 5 / the block-by-block scheme of Algorithm 2) and the fused
// diagonal phase sweep (K3, the diagonal branch of Algorithm 5).
//
// K4: each CTA takes chunks of 2^C amplitudes (C = 12 complex64, 11
// complex128): the low chunk bits are contiguous qubits (coalesced 128-bit
// loads), the others strided high qubits (direct indexing, no permutation
// pass).  The chunk is staged through shared memory (interleaved complex,
// XOR-swizzled) and processed in register stages: in each stage every thread
// holds 2^RB amplitudes whose index bits are the stage's register bits; gates
// on those bits are register arithmetic, diagonal phases may use any bit.
// One HBM read and one write per chunk, whatever the number of gates.
//
// Phases: a diagonal segment is a phase polynomial in fixed-point turns.
// Per thread it reduces to base + sum_j m_j lin_j + tab[m] (+ rare terms with
// several register bits) over the register index m, evaluated with integer
// adds; one sin/cos per amplitude turns it into a complex factor.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "chunk_dev.cuh"
#include "kernels.h"

namespace svs {
using namespace prog;

// ------------------------------------------------------------ K4 chunk sweep (interpreter)
template <typename R, int C, int RB>
__global__ void __launch_bounds__(1 << (C - RB), (C - RB) >= 7 ? 3 : 8) k_chunk(typename CT<R>::G2 *__restrict__ a,
                                                         const uint32_t *__restrict__ gprog, int n,
                                                         TSrc<typename CT<R>::G2> src)
{
    chunk_sweep<R, C, RB, InterpOps>(a, gprog, n, src);
}

// ------------------------------------------------------------ K3 diagonal sweep
// tile of 2^C consecutive amplitudes, C = 7 + RB: thread t holds amplitudes
// tile + t + m * 128 (register bits on top -> each warp load is contiguous)
template <typename R, int RB>
__global__ void __launch_bounds__(128) k_diag(typename CT<R>::G2 *__restrict__ a, const uint32_t *__restrict__ gprog,
                                              int n, TSrc<typename CT<R>::G2> src)
{
    using T2 = typename CT<R>::T2;
    using G2 = typename CT<R>::G2;
    using W = typename CT<R>::W;
    constexpr int NR = 1 << RB;
    constexpr int C = 7 + RB;
    constexpr int S = 1 + RB;
    constexpr int SCP = (int)cta_stride(RB, 7, sizeof(typename CT<R>::W));
    extern __shared__ __align__(16) unsigned char smraw[];
    uint32_t *prog = (uint32_t *)smraw;
    const int tid = threadIdx.x;
    stage_program<128>(gprog, prog, tid);
    __syncthreads();
    const int nd = (int)ldw(prog + H_NDSEG);
    const int nhoist = (int)ldw(prog + H_NHOIST);
    W *cta_buf = (W *)(prog + ((ldw(prog + H_WORDS) + 3) & ~3u));
    const int cbw = (int)(cta_buffer_bytes(nd, RB, 7, sizeof(W)) / sizeof(W));   // words of one buffer
    W *thr_ph = cta_buf + kCtaBuffers * cbw;
    const uint32_t *sp = prog + ldw(prog + H_STAGE_OFF);
    const uint32_t *op = sp + S_SIZE + O_BODY;
    thread_sums<R, 128>(prog, thr_ph, nhoist * S, tid);
    const int64_t ntiles = (int64_t)1 << (n - C);
    cta_zero<R, 128>(cta_buf, 2 * cbw, tid);
    __syncthreads();
    if (blockIdx.x < ntiles) cta_accum<R, 128>(prog, cta_buf, (uint64_t)blockIdx.x << C, tid);
    __syncthreads();
    // one barrier per tile: tile i reads CTA buffer i mod 3 while the next
    // tile's sums go to (i + 1) mod 3 (cleared during tile i - 1) and buffer
    // (i + 2) mod 3, last read by tile i - 1, is cleared
    int cb = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t base = (uint64_t)tile << C;
        const W *cta_ph = cta_buf + cb * cbw;
        cta_zero<R, 128>(cta_buf + (cb == 0 ? 2 : cb - 1) * cbw, nd * SCP, tid);
        if (tile + gridDim.x < ntiles)
            cta_accum<R, 128>(prog, cta_buf + (cb == 2 ? 0 : cb + 1) * cbw, (uint64_t)(tile + gridDim.x) << C, tid);
        const uint64_t x0 = base | (uint64_t)tid;
        T2 v[NR];
        // the tile's 2^C amplitudes share one hi factor when n_lo >= C:
        // converted once, multiplied in the register precision
        const bool shared_hi = src.hi && src.n_lo >= C;
        const T2 h = shared_hi ? to_reg(__ldg(&src.hi[base >> src.n_lo])) : T2{};
#pragma unroll
        for (int m = 0; m < NR; m++) {
            if (!src.hi) {
                v[m] = to_reg(__ldcs(a + x0 + ((uint64_t)m << 7)));
            } else if (shared_hi) {
                const G2 l = __ldg(&src.lo[(x0 + ((uint64_t)m << 7)) & ((1ull << src.n_lo) - 1)]);
                v[m] = cmul(h, to_reg(l));
            } else {
                v[m] = to_reg(tensor_amp(src, x0 + ((uint64_t)m << 7)));
            }
        }
        dseg_apply<R, RB, 128>(v, x0, op, cta_ph, thr_ph, nhoist, tid);
#pragma unroll
        for (int m = 0; m < NR; m++) __stcs(a + x0 + ((uint64_t)m << 7), to_glob(v[m]));
        __syncthreads();
        cb = cb == 2 ? 0 : cb + 1;
    }
}

// ------------------------------------------------------------ launchers
static constexpr int kMaxSmem = 200 * 1024;

// `attr` is per kernel instantiation (kernels of one signature share K)
template <typename K>
static cudaError_t sized_grid(K kern, bool &attr, int threads, size_t smem, int64_t work, int &grid)
{
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    int64_t g = (int64_t)device_sm_count() * occ;
    grid = (int)(g < work ? g : work);
    return cudaSuccess;
}

template <typename R, int C, int RB>
static cudaError_t chunk_t(void *a, int n, const uint32_t *prog, size_t smem, TensorSrc src, cudaStream_t st)
{
    using G2 = typename CT<R>::G2;
    constexpr int T = 1 << (C - RB);
    static bool attr = false;
    int grid = 0;
    cudaError_t e = sized_grid(k_chunk<R, C, RB>, attr, T, smem, (int64_t)1 << (n - C), grid);
    if (e != cudaSuccess) return e;
    const TSrc<G2> ts{(const G2 *)src.hi, (const G2 *)src.lo, src.n_lo};
    k_chunk<R, C, RB><<<grid, T, smem, st>>>((G2 *)a, prog, n, ts);
    return counted(cudaGetLastError(), 1);
}

// Fill g_cis64 on the current device once (before its first complex128
// sweep).  cudaMemcpyToSymbol from pageable memory returns when the copy is
// done, so kernels enqueued afterwards on any stream see the tables.
static cudaError_t set_cis64_tables()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    std::vector<dfc> t(3 * 256);
    const long double two_pi = 6.283185307179586476925286766559L;
    auto split = [](long double v, float &h, float &l) {
        h = (float)v;
        l = (float)(v - (long double)h);
    };
    for (int k = 0; k < 3; k++)
        for (int b = 0; b < 256; b++) {
            const long double x = two_pi * (long double)b / (long double)(1ull << (8 * k + 8));
            dfc &c = t[256 * k + b];
            split(cosl(x), c.rh, c.rl);
            split(sinl(x), c.ih, c.il);
        }
    e = cudaMemcpyToSymbol(g_cis64, t.data(), t.size() * sizeof(dfc));
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

cudaError_t launch_chunk(void *a, int n, bool f64, int C, int RB, const uint32_t *prog, size_t smem,
                         TensorSrc src, cudaStream_t st)
{
    if (f64) {
        cudaError_t e = set_cis64_tables();
        if (e != cudaSuccess) return e;
    }
    if (smem > (size_t)kMaxSmem) return cudaErrorInvalidValue;
    if (src.hi && (src.n_lo < 0 || src.n_lo > n || !src.lo)) return cudaErrorInvalidValue;
    if (!f64) {
        if (C == 12 && RB == 5 && n >= 12) return chunk_t<float, 12, 5>(a, n, prog, smem, src, st);
        if (C == 12 && RB == 4 && n >= 12) return chunk_t<float, 12, 4>(a, n, prog, smem, src, st);
        if (C == 10 && RB == 5 && n >= 10) return chunk_t<float, 10, 5>(a, n, prog, smem, src, st);
    } else {
        if (C == 11 && RB == 4 && n >= 11) return chunk_t<double, 11, 4>(a, n, prog, smem, src, st);
        if (C == 9 && RB == 4 && n >= 9) return chunk_t<double, 9, 4>(a, n, prog, smem, src, st);
    }
    return cudaErrorInvalidValue;
}

template <typename R, int RB>
static cudaError_t diag_t(void *a, int n, const uint32_t *prog, size_t smem, TensorSrc src, cudaStream_t st)
{
    using G2 = typename CT<R>::G2;
    constexpr int C = 7 + RB;
    if (n < C) return cudaErrorInvalidValue;
    static bool attr = false;
    int grid = 0;
    cudaError_t e = sized_grid(k_diag<R, RB>, attr, 128, smem, (int64_t)1 << (n - C), grid);
    if (e != cudaSuccess) return e;
    const TSrc<G2> ts{(const G2 *)src.hi, (const G2 *)src.lo, src.n_lo};
    k_diag<R, RB><<<grid, 128, smem, st>>>((G2 *)a, prog, n, ts);
    return counted(cudaGetLastError(), 1);
}

cudaError_t launch_diag_sweep(void *a, int n, bool f64, const uint32_t *prog, size_t smem, TensorSrc src,
                              cudaStream_t st)
{
    if (f64) {
        cudaError_t e = set_cis64_tables();
        if (e != cudaSuccess) return e;
    }
    if (smem > (size_t)kMaxSmem) return cudaErrorInvalidValue;
    if (src.hi && (src.n_lo < 0 || src.n_lo > n || !src.lo)) return cudaErrorInvalidValue;
    return f64 ? diag_t<double, 4>(a, n, prog, smem, src, st) : diag_t<float, 4>(a, n, prog, smem, src, st);
}

}  // namespace svs
