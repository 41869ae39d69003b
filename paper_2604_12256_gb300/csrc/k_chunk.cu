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
// Registers for three CTAs per SM (2^12 chunks: 256 threads of 16 amplitudes
// fit in 80 registers), one for 2^13 chunks.
template <typename R, int C, int RB>
__global__ void __launch_bounds__(1 << (C - RB), C >= 13 ? 1 : (C - RB) >= 7 ? 3 : 8) k_chunk(typename CT<R>::G2 *__restrict__ a,
                                                         const uint32_t *__restrict__ gprog, int n,
                                                         TSrc<typename CT<R>::G2> src)
{
    chunk_sweep<R, C, RB, InterpOps>(a, gprog, n, src, NoParams{});
}

// ------------------------------------------------------------ K3 diagonal sweep (interpreter)
template <typename R, int RB>
__global__ void __launch_bounds__(128) k_diag(typename CT<R>::G2 *__restrict__ a, const uint32_t *__restrict__ gprog,
                                              int n, TSrc<typename CT<R>::G2> src)
{
    diag_sweep<R, RB, DiagInterp>(a, gprog, n, src, NoParams{});
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
        if (C == 13 && RB == 5 && n >= 13) return chunk_t<float, 13, 5>(a, n, prog, smem, src, st);
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
