// k_dense5.cu -- a fused dense 5-qubit block (32 x 32 complex unitary U) applied
// to the whole state as a GEMM over the 2^(n-5) strided columns (the BatchMV
// idea of the hybrid scheme, Algorithm 3, done in-house instead of through a
// library + transpose).  Column j of X is the 32 amplitudes a[b_j | off(c)]
// of base index b_j (target bits zero); Y = U X is written back in place.
//
// Three arithmetic variants:
//   * k_dense5_tc: tcgen05 tensor cores, split-TF32 (x = hi + lo, three
//     products hi.hi + hi.lo + lo.hi accumulated in FP32 in TMEM) for
//     complex64 states.  Real embedding [Yr; Yi] = [[Ur, -Ui], [Ui, Ur]] [Xr; Xi]
//     as D(128 x 64) = A(128 x 64) B(64 x 64)^T with A = X^T of a 128-column
//     tile (one CTA thread per column) and B = the 64 x 64 embedding.
//   * k_dense5_fma<float>: FP32 CUDA cores (complex64 states).
//   * k_dense5_df: double-float on the FP32 pipe (complex128 states, default).
//   * k_dense5_fma<double>: FP64 on the FP64 pipe (complex128 states asked
//     for SIM_DENSE_FP64; this GPU's FP64 rate is 1/64 of its FP32 rate).
#include <cstdint>

#include "dfloat.h"
#include "kernels.h"
#include "tc_dev.cuh"

namespace svs {

struct Dense5Args {
    int sq[5];           // target qubits, ascending
    uint64_t off[32];    // global offset of target index c
};

__device__ __forceinline__ uint64_t d5_base(uint64_t col, const Dense5Args &g)
{
    uint64_t b = col;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const uint64_t low = b & ((1ull << g.sq[i]) - 1);
        b = ((b >> g.sq[i]) << (g.sq[i] + 1)) | low;
    }
    return b;
}

// ------------------------------------------------------------ CUDA cores
template <typename R> struct D5T;
template <> struct D5T<float> { using T2 = float2; };
template <> struct D5T<double> { using T2 = double2; };

// complex128 states: the block in double-float on the FP32 pipe (the FP64
// rate of this GPU is 1/64 of FP32's).  Each output component is a
// double-float dot product of 64 real products; the matrix is split into
// double-float pairs in shared memory, the column is converted once.
__global__ void __launch_bounds__(128) k_dense5_df(double2 *__restrict__ a, int n, Dense5Args g,
                                                   const double2 *__restrict__ U)
{
    __shared__ dfc su[32 * 32];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        const double2 u = U[i];
        dfc m;
        m.rh = __double2float_rn(u.x);
        m.rl = __double2float_rn(u.x - (double)m.rh);
        m.ih = __double2float_rn(u.y);
        m.il = __double2float_rn(u.y - (double)m.ih);
        su[i] = m;
    }
    __syncthreads();
    const int64_t ncol = (int64_t)1 << (n - 5);
    for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncol;
         col += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = d5_base((uint64_t)col, g);
        dfc x[32];
#pragma unroll
        for (int c = 0; c < 32; c++) x[c] = to_reg(a[b | g.off[c]]);
        for (int r = 0; r < 32; r++) {
            float rs = 0.f, re = 0.f, is = 0.f, ie = 0.f;
#pragma unroll
            for (int c = 0; c < 32; c++) {
                const dfc u = su[r * 32 + c];
                df_fma_acc(u.rh, u.rl, x[c].rh, x[c].rl, rs, re);
                df_fma_acc(-u.ih, -u.il, x[c].ih, x[c].il, rs, re);
                df_fma_acc(u.rh, u.rl, x[c].ih, x[c].il, is, ie);
                df_fma_acc(u.ih, u.il, x[c].rh, x[c].rl, is, ie);
            }
            dfc y;
            quick_two_sum(rs, re, y.rh, y.rl);
            quick_two_sum(is, ie, y.ih, y.il);
            a[b | g.off[r]] = to_glob(y);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(128) k_dense5_fma(typename D5T<R>::T2 *__restrict__ a, int n, Dense5Args g,
                                                    const double2 *__restrict__ U)
{
    using T2 = typename D5T<R>::T2;
    __shared__ T2 su[32 * 32];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        const double2 u = U[i];
        su[i].x = (R)u.x;
        su[i].y = (R)u.y;
    }
    __syncthreads();
    const int64_t ncol = (int64_t)1 << (n - 5);
    for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncol;
         col += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = d5_base((uint64_t)col, g);
        T2 x[32];
#pragma unroll
        for (int c = 0; c < 32; c++) x[c] = a[b | g.off[c]];
        for (int r = 0; r < 32; r++) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < 32; c++) {
                const T2 u = su[r * 32 + c];
                re = fma(u.x, x[c].x, re);
                re = fma(-u.y, x[c].y, re);
                im = fma(u.x, x[c].y, im);
                im = fma(u.y, x[c].x, im);
            }
            T2 y;
            y.x = re;
            y.y = im;
            a[b | g.off[r]] = y;
        }
    }
}

// ------------------------------------------------------------ tensor cores
constexpr int kTcCols = 128;                  // columns per tile (MMA M)
constexpr int kTmemCols = 64;                 // columns of one accumulator (MMA N)
constexpr int kTmemAlloc = 128;               // two accumulators: hi.hi and the hi.lo + lo.hi corrections
constexpr uint32_t kWaitLimit = 1u << 22;     // bounded mbarrier polling

// A: X^T tile (128 x 64) hi/lo; B: embedded U (64 x 64) hi/lo
struct TcSmem {
    uint32_t a_hi[kTcCols * 64];
    uint32_t a_lo[kTcCols * 64];
    uint32_t b_hi[64 * 64];
    uint32_t b_lo[64 * 64];
    uint64_t mbar;
    uint32_t tmem_addr;
    int abort_;
};

// wait_limit: mbarrier polls before a wait gives up (kWaitLimit in normal
// use).  skip_mma != 0 (self-test only): the elected thread issues no MMA and
// no commit, so the first wait runs out and the abort path is taken with
// nothing in flight.
__global__ void __launch_bounds__(kTcCols) k_dense5_tc(float2 *__restrict__ a, int n, Dense5Args g,
                                                        const double2 *__restrict__ U, int *status,
                                                        uint32_t wait_limit, int skip_mma)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smraw);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    // B = [[Ur, -Ui], [Ui, Ur]] split into TF32 hi + lo (from the FP64 matrix)
    for (int e = tid; e < 64 * 64; e += kTcCols) {
        const int nn = e >> 6, kk = e & 63;
        const int r = nn & 31, c = kk & 31;
        const double2 u = U[r * 32 + c];
        double v;
        if (nn < 32) v = kk < 32 ? u.x : -u.y;
        else v = kk < 32 ? u.y : u.x;
        const uint32_t hi = tf32_of((float)v);
        const uint32_t lo = tf32_of((float)(v - (double)__uint_as_float(hi)));
        const uint32_t o = kmajor_off(nn, kk, 64) >> 2;
        sm.b_hi[o] = hi;
        sm.b_lo[o] = lo;
    }
    if (tid == 0) {
        sm.abort_ = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&sm.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&sm.tmem_addr)),
                     "r"(kTmemAlloc));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sm.tmem_addr;
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&sm.mbar);
    const uint32_t a_hi = (uint32_t)__cvta_generic_to_shared(sm.a_hi);
    const uint32_t a_lo = (uint32_t)__cvta_generic_to_shared(sm.a_lo);
    const uint32_t b_hi = (uint32_t)__cvta_generic_to_shared(sm.b_hi);
    const uint32_t b_lo = (uint32_t)__cvta_generic_to_shared(sm.b_lo);
    // kind::tf32, D = F32, A = B = TF32, both K-major, N = 64, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTmemCols >> 3) << 17) |
                           ((uint32_t)(kTcCols >> 4) << 24);
    const uint32_t lbo_a = (kTcCols / 8) * 128, lbo_b = (64 / 8) * 128, sbo = 128;

    const int64_t ncol = (int64_t)1 << (n - 5);
    const int64_t ntiles = (ncol + kTcCols - 1) / kTcCols;
    uint32_t phase = 0;
    // this thread's column of a tile: its 32 amplitudes into registers
    float xr[32], xi[32];
    auto load_col = [&](int64_t t, uint64_t &base, bool &ok) {
        const int64_t col = t * kTcCols + tid;
        ok = t < ntiles && col < ncol;
        base = ok ? d5_base((uint64_t)col, g) : 0;
#pragma unroll
        for (int c = 0; c < 32; c++) {
            float2 v = ok ? a[base | g.off[c]] : make_float2(0.f, 0.f);
            xr[c] = v.x;
            xi[c] = v.y;
        }
    };
    uint64_t b = 0;
    bool valid = false;
    load_col(blockIdx.x, b, valid);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // ---- A tile: this thread's column, split into TF32 hi + lo
#pragma unroll
        for (int k4 = 0; k4 < 16; k4++) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int k = k4 * 4 + e;
                const float x = k < 32 ? xr[k] : xi[k - 32];
                h[e] = tf32_of(x);
                l[e] = tf32_of(x - __uint_as_float(h[e]));
            }
            const uint32_t o = kmajor_off(tid, k4 * 4, kTcCols) >> 2;
            *reinterpret_cast<uint4 *>(&sm.a_hi[o]) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(&sm.a_lo[o]) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        // make the generic-proxy writes visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0 && !skip_mma) {
            // big = Ahi Bhi^T (columns 0..63); small = Ahi Blo^T + Alo Bhi^T
            // (columns 64..127), kept apart so that the accumulator does not
            // drop the small terms; 8 K-steps of 8 each
            for (int pass = 0; pass < 3; pass++) {
                const uint32_t A = pass == 2 ? a_lo : a_hi;
                const uint32_t B = pass == 1 ? b_lo : b_hi;
                const uint32_t D = pass == 0 ? tmem : tmem + kTmemCols;
                for (int ks = 0; ks < 8; ks++) {
                    const uint64_t ad = smem_desc(A + ks * 2 * lbo_a, lbo_a, sbo);
                    const uint64_t bd = smem_desc(B + ks * 2 * lbo_b, lbo_b, sbo);
                    const int acc = (pass == 2 || ks > 0) ? 1 : 0;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(D),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                         : "memory");
        }
        // ---- the next tile's loads go out now and stay in flight through the
        // wait and the epilogue (its columns are disjoint from this tile's)
        uint64_t b_next;
        bool valid_next;
        load_col(tile + gridDim.x, b_next, valid_next);
        // ---- wait for the products (bounded), then read this thread's row
        uint32_t it = 0;
        while (!mbar_try_wait(mbar, phase)) {
            if (++it > wait_limit) break;
            __nanosleep(64);
        }
        if (it > wait_limit) sm.abort_ = 1;
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (sm.abort_) break;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        float yre[32], yim[32];
        {
            uint32_t bg[32], sm_[32];
            tmem_ld32(taddr, bg);
            tmem_ld32(taddr + kTmemCols, sm_);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int r = 0; r < 32; r++) yre[r] = __uint_as_float(bg[r]) + __uint_as_float(sm_[r]);
            tmem_ld32(taddr + 32, bg);
            tmem_ld32(taddr + kTmemCols + 32, sm_);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int r = 0; r < 32; r++) yim[r] = __uint_as_float(bg[r]) + __uint_as_float(sm_[r]);
        }
        if (valid) {
#pragma unroll
            for (int r = 0; r < 32; r++) a[b | g.off[r]] = make_float2(yre[r], yim[r]);
        }
        // the next tile's MMAs overwrite the accumulator and read A: every
        // thread's TMEM reads and A writes must be ordered around them
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        b = b_next;
        valid = valid_next;
    }
    if (sm.abort_ && tid == 0) {
        atomicExch(status, 1);
        // give the products in flight one more bounded wait before freeing TMEM
        for (uint32_t it = 0; it < wait_limit && !mbar_try_wait(mbar, phase ^ 1); it++) __nanosleep(64);
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemAlloc));
}

// ------------------------------------------------------------ launcher
static Dense5Args d5_args(const int *q)
{
    Dense5Args g;
    int sq[5];
    for (int i = 0; i < 5; i++) sq[i] = q[i];
    for (int i = 1; i < 5; i++)
        for (int j = i; j > 0 && sq[j - 1] > sq[j]; j--) { int t = sq[j]; sq[j] = sq[j - 1]; sq[j - 1] = t; }
    for (int i = 0; i < 5; i++) g.sq[i] = sq[i];
    for (int c = 0; c < 32; c++) {
        uint64_t o = 0;
        for (int i = 0; i < 5; i++) if ((c >> i) & 1) o |= 1ull << q[i];
        g.off[c] = o;
    }
    return g;
}

cudaError_t launch_dense5(void *a, int n, bool f64, int precision, const int *q, const void *U64, int *status,
                          cudaStream_t st)
{
    if (n < 5) return cudaErrorInvalidValue;
    const Dense5Args g = d5_args(q);
    const int64_t ncol = (int64_t)1 << (n - 5);
    if (f64) {
        int grid = (int)std::min<int64_t>((ncol + 127) / 128, (int64_t)device_sm_count() * 8);
        if (precision == 2)   // true FP64 on the FP64 pipe
            k_dense5_fma<double><<<grid, 128, 0, st>>>((double2 *)a, n, g, (const double2 *)U64);
        else
            k_dense5_df<<<grid, 128, 0, st>>>((double2 *)a, n, g, (const double2 *)U64);
        return counted(cudaGetLastError(), 1);
    }
    if (precision == 0) {   // split-TF32 on the tensor cores
        static bool attr = false;
        const size_t smem = sizeof(TcSmem);
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_dense5_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const int64_t tiles = (ncol + kTcCols - 1) / kTcCols;
        // two CTAs per SM: 2 x 64 TMEM columns, 2 x ~97 KB shared memory
        int grid = (int)std::min<int64_t>(tiles, (int64_t)device_sm_count() * 2);
        k_dense5_tc<<<grid, kTcCols, smem, st>>>((float2 *)a, n, g, (const double2 *)U64, status, kWaitLimit, 0);
        return counted(cudaGetLastError(), 1);
    }
    int grid = (int)std::min<int64_t>((ncol + 127) / 128, (int64_t)device_sm_count() * 8);
    k_dense5_fma<float><<<grid, 128, 0, st>>>((float2 *)a, n, g, (const double2 *)U64);
    return counted(cudaGetLastError(), 1);
}

// Self-test of the bounded wait: the tensor-core kernel on qubits 0..4 of a
// complex64 state with its MMA issue suppressed and wait_limit polls per
// wait, so every wait runs out; *status becomes 1 and the state is untouched.
cudaError_t launch_dense5_wait_selftest(void *a, int n, const void *U64, int *status, uint32_t wait_limit,
                                        cudaStream_t st)
{
    if (n < 5) return cudaErrorInvalidValue;
    const int q[5] = {0, 1, 2, 3, 4};
    const Dense5Args g = d5_args(q);
    static bool attr = false;
    const size_t smem = sizeof(TcSmem);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_dense5_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_dense5_tc<<<1, kTcCols, smem, st>>>((float2 *)a, n, g, (const double2 *)U64, status, wait_limit, 1);
    return counted(cudaGetLastError(), 1);
}

}  // namespace svs
