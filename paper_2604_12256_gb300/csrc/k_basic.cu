// k_basic.cu -- whole-vector kernels: basis-state initialisation, the
// gate-by-gate sweeps of Algorithm 1 (one dense gate, or one diagonal gate
// touching only the amplitudes it changes), the tensor-product merge of the
// merge booster (Algorithm 7 / Algorithm 5 first branch) and the read-out
// reductions (norm, <Z-string>, probabilities, top-k) in FP64 accumulation
// with a fixed reduction order.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <vector>

#include "kernels.h"

namespace svs {

static std::atomic<uint64_t> g_launches{0};

cudaError_t counted(cudaError_t e, int kernels)
{
    if (e == cudaSuccess) g_launches.fetch_add((uint64_t)kernels, std::memory_order_relaxed);
    return e;
}

uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

static int g_sms = 0;
int device_sm_count()
{
    if (g_sms <= 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            g_sms = v;
        else
            g_sms = kNumSMs;
    }
    return g_sms;
}

static inline int grid_for(int64_t work, int threads, int per_sm)
{
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)device_sm_count() * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// ------------------------------------------------------------ basis state
template <typename T2>
__global__ void k_set_one(T2 *a, uint64_t idx)
{
    T2 one;
    one.x = 1;
    one.y = 0;
    a[idx] = one;
}

cudaError_t launch_init_basis(void *a, int n, bool f64, uint64_t basis, cudaStream_t st)
{
    size_t bytes = ((size_t)1 << n) * (f64 ? 16 : 8);
    cudaError_t e = cudaMemsetAsync(a, 0, bytes, st);
    if (e != cudaSuccess) return e;
    if (f64) k_set_one<double2><<<1, 1, 0, st>>>((double2 *)a, basis);
    else k_set_one<float2><<<1, 1, 0, st>>>((float2 *)a, basis);
    return counted(cudaGetLastError(), 1);
}

// ------------------------------------------------------------ dense gate
struct DenseArgs {
    int sq[6];          // the gate's qubits, ascending (zero-insertion order)
    uint64_t off[64];   // global offset of local index c: sum_i c_i << q[i]
};

template <typename R, int K>
__global__ void __launch_bounds__(256) k_gate_dense(typename Cx<R>::T *__restrict__ a, int n, DenseArgs g,
                                                    const typename Cx<R>::T *__restrict__ M)
{
    using T2 = typename Cx<R>::T;
    constexpr int D = 1 << K;
    const int64_t nb = (int64_t)1 << (n - K);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += stride) {
        uint64_t base = (uint64_t)b;
#pragma unroll
        for (int i = 0; i < K; i++) {
            uint64_t low = base & ((1ull << g.sq[i]) - 1);
            base = ((base >> g.sq[i]) << (g.sq[i] + 1)) | low;
        }
        T2 v[D];
#pragma unroll
        for (int c = 0; c < D; c++) v[c] = a[base | g.off[c]];
#pragma unroll
        for (int r = 0; r < D; r++) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < D; c++) {
                T2 m = __ldg(&M[r * D + c]);
                re = fma(m.x, v[c].x, re);
                re = fma(-m.y, v[c].y, re);
                im = fma(m.x, v[c].y, im);
                im = fma(m.y, v[c].x, im);
            }
            T2 w;
            w.x = re;
            w.y = im;
            a[base | g.off[r]] = w;
        }
    }
}

template <typename R>
static cudaError_t gate_dense_t(void *a, int n, int k, const int *q, const void *dmat, cudaStream_t st)
{
    using T2 = typename Cx<R>::T;
    DenseArgs g;
    int sq[6];
    for (int i = 0; i < k; i++) sq[i] = q[i];
    for (int i = 1; i < k; i++)
        for (int j = i; j > 0 && sq[j - 1] > sq[j]; j--) { int t = sq[j]; sq[j] = sq[j - 1]; sq[j - 1] = t; }
    for (int i = 0; i < 6; i++) g.sq[i] = i < k ? sq[i] : 0;
    for (int c = 0; c < 64; c++) {
        uint64_t o = 0;
        if (c < (1 << k))
            for (int i = 0; i < k; i++) if ((c >> i) & 1) o |= 1ull << q[i];
        g.off[c] = o;
    }
    int64_t groups = (int64_t)1 << (n - k);
    int grid = grid_for(groups, 256, 8);
    T2 *A = (T2 *)a;
    const T2 *M = (const T2 *)dmat;
    switch (k) {
    case 1: k_gate_dense<R, 1><<<grid, 256, 0, st>>>(A, n, g, M); break;
    case 2: k_gate_dense<R, 2><<<grid, 256, 0, st>>>(A, n, g, M); break;
    case 3: k_gate_dense<R, 3><<<grid, 256, 0, st>>>(A, n, g, M); break;
    case 4: k_gate_dense<R, 4><<<grid, 256, 0, st>>>(A, n, g, M); break;
    case 5: k_gate_dense<R, 5><<<grid, 256, 0, st>>>(A, n, g, M); break;
    case 6: k_gate_dense<R, 6><<<grid, 256, 0, st>>>(A, n, g, M); break;
    default: return cudaErrorInvalidValue;
    }
    return counted(cudaGetLastError(), 1);
}

cudaError_t launch_gate_dense(void *a, int n, bool f64, int k, const int *q, const void *dmat, cudaStream_t st)
{
    if (k < 1 || k > 6 || k > n) return cudaErrorInvalidValue;
    return f64 ? gate_dense_t<double>(a, n, k, q, dmat, st) : gate_dense_t<float>(a, n, k, q, dmat, st);
}

// ------------------------------------------------------------ diagonal gate
struct DiagArgs {
    int k, nz;
    int sq[6];
    uint64_t off[64];   // global offsets of the nz local indices to touch
};

template <typename R>
__global__ void __launch_bounds__(256) k_gate_diag(typename Cx<R>::T *__restrict__ a, int n, DiagArgs g,
                                                   const typename Cx<R>::T *__restrict__ d)
{
    using T2 = typename Cx<R>::T;
    const int64_t nb = (int64_t)1 << (n - g.k);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += stride) {
        uint64_t base = (uint64_t)b;
        for (int i = 0; i < g.k; i++) {
            uint64_t low = base & ((1ull << g.sq[i]) - 1);
            base = ((base >> g.sq[i]) << (g.sq[i] + 1)) | low;
        }
        for (int c = 0; c < g.nz; c++) {
            T2 f = __ldg(&d[c]);
            T2 v = a[base | g.off[c]];
            T2 w;
            w.x = v.x * f.x - v.y * f.y;
            w.y = v.x * f.y + v.y * f.x;
            a[base | g.off[c]] = w;
        }
    }
}

cudaError_t launch_gate_diag(void *a, int n, bool f64, int k, const int *q, int nz, const int *cidx,
                             const void *dvals, cudaStream_t st)
{
    if (k < 1 || k > 6 || k > n || nz < 0 || nz > 64) return cudaErrorInvalidValue;
    if (nz == 0) return cudaSuccess;
    DiagArgs g;
    g.k = k;
    g.nz = nz;
    int sq[6];
    for (int i = 0; i < k; i++) sq[i] = q[i];
    for (int i = 1; i < k; i++)
        for (int j = i; j > 0 && sq[j - 1] > sq[j]; j--) { int t = sq[j]; sq[j] = sq[j - 1]; sq[j - 1] = t; }
    for (int i = 0; i < 6; i++) g.sq[i] = i < k ? sq[i] : 0;
    for (int c = 0; c < 64; c++) {
        uint64_t o = 0;
        if (c < nz)
            for (int i = 0; i < k; i++) if ((cidx[c] >> i) & 1) o |= 1ull << q[i];
        g.off[c] = o;
    }
    int64_t groups = (int64_t)1 << (n - k);
    int grid = grid_for(groups, 256, 8);
    if (f64) k_gate_diag<double><<<grid, 256, 0, st>>>((double2 *)a, n, g, (const double2 *)dvals);
    else k_gate_diag<float><<<grid, 256, 0, st>>>((float2 *)a, n, g, (const float2 *)dvals);
    return counted(cudaGetLastError(), 1);
}

// ------------------------------------------------------------ small phase sweep
template <typename R>
__global__ void __launch_bounds__(256) k_phase_small(typename Cx<R>::T *__restrict__ a, int64_t N,
                                                     const uint64_t *__restrict__ terms, int nt)
{
    using T2 = typename Cx<R>::T;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride) {
        uint64_t w = 0;
        for (int t = 0; t < nt; t++) {
            uint64_t m = __ldg(&terms[2 * t]);
            if (((uint64_t)x & m) == m) w += __ldg(&terms[2 * t + 1]);
        }
        double s, c;
        sincospi((double)(int64_t)w * 1.0842021724855044340e-19, &s, &c);
        T2 v = a[x], r;
        r.x = (R)(v.x * c - v.y * s);
        r.y = (R)(v.x * s + v.y * c);
        a[x] = r;
    }
}

cudaError_t launch_phase_small(void *a, int n, bool f64, const uint64_t *terms, int nt, cudaStream_t st)
{
    int64_t N = (int64_t)1 << n;
    int grid = grid_for(N, 256, 8);
    if (f64) k_phase_small<double><<<grid, 256, 0, st>>>((double2 *)a, N, terms, nt);
    else k_phase_small<float><<<grid, 256, 0, st>>>((float2 *)a, N, terms, nt);
    return counted(cudaGetLastError(), 1);
}

// ------------------------------------------------------------ tensor product
template <typename R>
__global__ void __launch_bounds__(256) k_tensor(typename Cx<R>::T *__restrict__ out,
                                                const typename Cx<R>::T *__restrict__ hi,
                                                const typename Cx<R>::T *__restrict__ lo, int n_lo,
                                                int64_t total)
{
    using T2 = typename Cx<R>::T;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t lmask = (1ull << n_lo) - 1;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
        T2 h = __ldg(&hi[(uint64_t)x >> n_lo]);
        T2 l = __ldg(&lo[(uint64_t)x & lmask]);
        T2 w;
        w.x = h.x * l.x - h.y * l.y;
        w.y = h.x * l.y + h.y * l.x;
        out[x] = w;
    }
}

cudaError_t launch_tensor(void *out, const void *hi, int n_hi, const void *lo, int n_lo, bool f64, cudaStream_t st)
{
    int64_t total = (int64_t)1 << (n_hi + n_lo);
    int grid = grid_for(total, 256, 8);
    if (f64) k_tensor<double><<<grid, 256, 0, st>>>((double2 *)out, (const double2 *)hi, (const double2 *)lo, n_lo, total);
    else k_tensor<float><<<grid, 256, 0, st>>>((float2 *)out, (const float2 *)hi, (const float2 *)lo, n_lo, total);
    return counted(cudaGetLastError(), 1);
}

// ------------------------------------------------------------ reductions
// A fixed grid (kRedBlocks x kRedThreads) makes every sum's order independent
// of the device, so results are bit-reproducible run to run.
constexpr int kRedBlocks = kReduceBlocks;   // norm
constexpr int kExpBlocks = 512;              // <Z> strings
static_assert(kExpBlocks <= kReduceBlocks, "partials buffer");
constexpr int kRedThreads = 256;
int reduce_partials() { return kRedBlocks; }

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += sh[i];
    return s;   // valid in thread 0
}

// |a|^2 of one amplitude: exact squares in FP64, one rounding in the sum.
__device__ __forceinline__ double prob_of(float2 v) { return fma((double)v.x, (double)v.x, (double)v.y * (double)v.y); }
// (no contraction: each square rounded, then the sum -- the plain definition)
__device__ __forceinline__ double prob_of(double2 v) { return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)); }
__device__ __forceinline__ float probf(float2 v) { return fmaf(v.x, v.x, v.y * v.y); }

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_norm_part(const typename Cx<R>::T *__restrict__ a, int64_t N,
                                                            double *part)
{
    __shared__ double sh[32];
    double acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (sizeof(R) == 4) {
        // complex64: FP32 sums over runs of 32 amplitudes (four independent
        // chains), FP64 across runs, as the <Z> partials
        for (int64_t i = i0; i < N; i += 32 * stride) {
            float f[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int b = 0; b < 32; b++) {
                const int64_t j = i + b * stride;
                if (j < N) f[b & 3] += probf(a[j]);
            }
            acc += (double)((f[0] + f[1]) + (f[2] + f[3]));
        }
    } else {
        for (int64_t i = i0; i < N; i += stride) acc += prob_of(a[i]);
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double *part, int np, int nt, double *out)
{
    // one block per term; fixed-order tree over np partials
    __shared__ double sh[32];
    const double *p = part + (size_t)blockIdx.x * np;
    double acc = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += p[i];
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
    (void)nt;
}

cudaError_t launch_norm(const void *a, int n, bool f64, double *part, double *out, cudaStream_t st)
{
    int64_t N = (int64_t)1 << n;
    if (f64) k_norm_part<double><<<kRedBlocks, kRedThreads, 0, st>>>((const double2 *)a, N, part);
    else k_norm_part<float><<<kRedBlocks, kRedThreads, 0, st>>>((const float2 *)a, N, part);
    k_sum_parts<<<1, 256, 0, st>>>(part, kRedBlocks, 1, out);
    return counted(cudaGetLastError(), 2);
}

template <typename R, int NT>
__global__ void __launch_bounds__(kRedThreads) k_expect_part(const typename Cx<R>::T *__restrict__ a, int64_t N,
                                                              const uint64_t *__restrict__ masks, int nt,
                                                              double *part)
{
    __shared__ double sh[32];
    __shared__ uint64_t m[NT];
    if (threadIdx.x < NT) m[threadIdx.x] = threadIdx.x < nt ? masks[threadIdx.x] : 0;
    __syncthreads();
    double acc[NT];
#pragma unroll
    for (int t = 0; t < NT; t++) acc[t] = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (sizeof(R) == 4) {
        // complex64: FP32 sums over groups of 8 runs of 32 amplitudes, FP64
        // across groups (the FP64 rate of this part is 1/64 of its FP32
        // rate: one conversion and add per term per run would cost as much
        // as the HBM read).  The
        // grid's stride S = 2^sb is a power of two, so a thread visits
        // i = tid + k S, k = 0 .. K-1, and in a run k = k0 + b (b < 32, k0 a
        // multiple of 32) the sign of mask m is (-1)^(P0 + popc(b & u)) with
        // u = (m >> sb) & 31 and P0 the parity of the run's other bits.  So
        // the run's signed sum for m is (-1)^P0 W[u], W the Walsh-Hadamard
        // transform of its 32 probabilities: one 5-level butterfly per run
        // gives every mask's sum (kept in this thread's shared-memory column
        // and read back at the masks' u).
        __shared__ float wsh[32 * kRedThreads];
        const int sb = 63 - __clzll((unsigned long long)stride);     // log2 S
        const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t K = N >> sb;                                     // amplitudes per thread
        uint32_t u[NT];
        uint32_t Pt = 0;   // parities of tid & m_t
#pragma unroll
        for (int t = 0; t < NT; t++) {
            u[t] = sb < 64 ? (uint32_t)((m[t] >> sb) & 31) : 0;
            Pt |= (uint32_t)(__popcll((uint64_t)tid & m[t]) & 1) << t;
        }
        if (K < 32) {   // short rows (N < 32 S): amplitude by amplitude
            const int64_t kn = K > 0 ? K : (tid < N ? 1 : 0);
            for (int64_t k = 0; k < kn; k++) {
                const int64_t i = tid + (k << sb);
                const double p = (double)probf(a[i]);
#pragma unroll
                for (int t = 0; t < NT; t++) acc[t] += (__popcll((uint64_t)i & m[t]) & 1) ? -p : p;
            }
        } else {
            float *col = wsh + threadIdx.x;
            float acc32[NT];
#pragma unroll
            for (int t = 0; t < NT; t++) acc32[t] = 0.f;
            for (int64_t k0 = 0; k0 < K; k0 += 32) {
                float w[32];
#pragma unroll
                for (int b = 0; b < 32; b++) w[b] = probf(a[tid + ((k0 + b) << sb)]);
#pragma unroll
                for (int h = 1; h < 32; h <<= 1)
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        if (!(j & h)) {
                            const float x = w[j], y = w[j | h];
                            w[j] = x + y;
                            w[j | h] = x - y;
                        }
#pragma unroll
                for (int b = 0; b < 32; b++) col[b * kRedThreads] = w[b];
                const uint64_t hi = (uint64_t)k0 << sb;   // the run's index bits above sb + 4
#pragma unroll
                for (int t = 0; t < NT; t++) {
                    const float c = col[u[t] * kRedThreads];
                    const uint32_t neg = ((Pt >> t) ^ (uint32_t)__popcll(hi & m[t])) & 1u;
                    acc32[t] += __uint_as_float(__float_as_uint(c) ^ (neg << 31));
                }
                if ((k0 & 255) == 224 || k0 + 32 >= K) {   // every 8th run, and the last
#pragma unroll
                    for (int t = 0; t < NT; t++) {
                        acc[t] += (double)acc32[t];
                        acc32[t] = 0.f;
                    }
                }
            }
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
            const double p = prob_of(a[i]);
#pragma unroll
            for (int t = 0; t < NT; t++) acc[t] += (__popcll((uint64_t)i & m[t]) & 1) ? -p : p;
        }
    }
#pragma unroll
    for (int t = 0; t < NT; t++) {
        if (t >= nt) break;
        double s = block_sum(acc[t], sh);
        if (threadIdx.x == 0) part[(size_t)t * gridDim.x + blockIdx.x] = s;
    }
}

cudaError_t launch_expect_z(const void *a, int n, bool f64, const uint64_t *masks, int nt, double *part,
                            double *out, cudaStream_t st)
{
    if (nt < 1 || nt > 16) return cudaErrorInvalidValue;
    int64_t N = (int64_t)1 << n;
    if (f64) k_expect_part<double, 16><<<kExpBlocks, kRedThreads, 0, st>>>((const double2 *)a, N, masks, nt, part);
    else k_expect_part<float, 16><<<kExpBlocks, kRedThreads, 0, st>>>((const float2 *)a, N, masks, nt, part);
    k_sum_parts<<<nt, 256, 0, st>>>(part, kExpBlocks, nt, out);
    return counted(cudaGetLastError(), 2);
}

template <typename R>
__global__ void __launch_bounds__(256) k_probs(const typename Cx<R>::T *__restrict__ a, int64_t N, double *out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) out[i] = prob_of(a[i]);
}

cudaError_t launch_probs(const void *a, int n, bool f64, double *out, cudaStream_t st)
{
    int64_t N = (int64_t)1 << n;
    int grid = grid_for(N, 256, 8);
    if (f64) k_probs<double><<<grid, 256, 0, st>>>((const double2 *)a, N, out);
    else k_probs<float><<<grid, 256, 0, st>>>((const float2 *)a, N, out);
    return counted(cudaGetLastError(), 1);
}

// ------------------------------------------------------------ top-k
// Each block keeps the best k (probability descending, index ascending) of
// its slice in shared memory: candidates better than the current k-th best
// are appended, and the buffer is bitonic-sorted and cut back to k whenever
// it holds more than k.  A second single-block pass merges the block lists.
// The order (p desc, index asc) is total, so the result is unique.
struct KI {
    double p;
    uint64_t i;
};
constexpr int kTopThreads = 256;
constexpr int kTopTile = kTopThreads * 4;
constexpr int kTopCap = 2048;   // >= 1024 kept + one tile
constexpr int kTopBlocksPerSM = 2;   // blocks per SM (more lists make the single-block merge slower)
static int topk_blocks(int64_t N)
{
    int64_t g = (N + kTopTile - 1) / kTopTile;
    int64_t cap = kTopBlocksPerSM * (int64_t)device_sm_count();
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}
// per-block lists (at most kTopBlocksPerSM x SMs of k entries) + the final k
size_t topk_scratch_bytes(int k)
{
    const int sms = device_sm_count() > kNumSMs ? device_sm_count() : kNumSMs;
    return ((size_t)kTopBlocksPerSM * sms + 1) * (size_t)k * sizeof(KI) + 4096;
}

// (p desc, index asc).  Probabilities are >= +0 and the empty entry has p =
// -1, so the order of p is the order of its bits read as a signed 64-bit
// integer: the comparison runs on the integer pipe, not the slow FP64 one.
__device__ __forceinline__ bool better(const KI &a, const KI &b)
{
    const long long pa = __double_as_longlong(a.p), pb = __double_as_longlong(b.p);
    return pa > pb || (pa == pb && a.i < b.i);
}

__device__ void bitonic_desc(KI *buf, int cap)
{
    for (int size = 2; size <= cap; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int t = threadIdx.x; t < cap / 2; t += blockDim.x) {
                int lo = 2 * t - (t & (stride - 1));
                int hi = lo + stride;
                bool desc = ((lo & size) == 0);
                KI x = buf[lo], y = buf[hi];
                bool sw = desc ? better(y, x) : better(x, y);
                if (sw) { buf[lo] = y; buf[hi] = x; }
            }
        }
    }
    __syncthreads();
}

template <typename R, bool FROM_STATE>
__global__ void __launch_bounds__(kTopThreads) k_topk(const typename Cx<R>::T *__restrict__ a, const KI *__restrict__ cand,
                                                      int64_t N, int k, KI *out)
{
    __shared__ KI buf[kTopCap];
    __shared__ int cnt;
    __shared__ KI thr;
    // complex64: a float pre-filter threshold (the FP64 k-th best rounded
    // down by a margin far above the float rounding error), set with thr so
    // that the hot loop does no FP64 work and reads one shared word per tile
    __shared__ float thr_f;
    const KI worst = {-1.0, ~0ull};
    if (threadIdx.x == 0) { cnt = 0; thr = worst; thr_f = -1.0f; }
    __syncthreads();
    int64_t per = (N + gridDim.x - 1) / gridDim.x;
    int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < N ? lo + per : N;
    // the next batch of NB tiles is loaded while this batch is filtered and
    // (now and then) sorted: complex64 keeps 16 amplitudes per thread in
    // flight (enough bytes per SM to cover the HBM latency)
    using T2 = typename Cx<R>::T;
    constexpr int NB = (FROM_STATE && sizeof(R) == 4) ? 4 : 1;
    T2 nz[4 * NB];
    auto load_batch = [&](int64_t t0) {
        if constexpr (FROM_STATE) {
#pragma unroll
            for (int e = 0; e < 4 * NB; e++) {
                const int64_t i = t0 + e * kTopThreads + threadIdx.x;
                if (i < hi) nz[e] = a[i];
            }
        }
    };
    if (lo < hi) load_batch(lo);
    for (int64_t t00 = lo; t00 < hi; t00 += (int64_t)kTopTile * NB) {
        T2 cb[4 * NB];
#pragma unroll
        for (int e = 0; e < 4 * NB; e++) cb[e] = nz[e];
        if (t00 + (int64_t)kTopTile * NB < hi) load_batch(t00 + (int64_t)kTopTile * NB);
#pragma unroll
        for (int sbt = 0; sbt < NB; sbt++) {
        const int64_t t0 = t00 + (int64_t)sbt * kTopTile;
        if (t0 >= hi) break;
        T2 cz[4];
#pragma unroll
        for (int e = 0; e < 4; e++) cz[e] = cb[4 * sbt + e];
        const float thf = thr_f;
        int ins = 0;   // candidates this thread appended
#pragma unroll
        for (int e = 0; e < 4; e++) {
            int64_t i = t0 + e * kTopThreads + threadIdx.x;
            if (i < hi) {
                KI v;
                if constexpr (FROM_STATE) {
                    const auto z = cz[e];
                    if constexpr (sizeof(R) == 4) {
                        if (fmaf(z.x, z.x, z.y * z.y) < thf) continue;
                    }
                    v.p = prob_of(z);
                    v.i = (uint64_t)i;
                } else {
                    v = cand[i];
                }
                if (better(v, thr)) { int pos = atomicAdd(&cnt, 1); buf[pos] = v; ins++; }
            }
        }
        // one barrier when no thread appended anything (the common case once
        // the threshold has risen); otherwise every thread reads the count
        // before a second barrier (so all take the same branch), and the
        // buffer is sorted and cut back to k when another tile might not fit
        if (__syncthreads_or(ins)) {
            const int c = cnt;
            __syncthreads();
            if (c > kTopCap - kTopTile) {
                for (int j = c + threadIdx.x; j < kTopCap; j += blockDim.x) buf[j] = worst;
                bitonic_desc(buf, kTopCap);
                if (threadIdx.x == 0) {
                    cnt = k;
                    thr = buf[k - 1];
                    thr_f = thr.p > 0 ? __double2float_rd(thr.p * (1.0 - 1e-5)) : -1.0f;
                }
                __syncthreads();
            }
        }
        }
    }
    // final: sort what is kept and write exactly k entries (padded with worst)
    for (int j = cnt + threadIdx.x; j < kTopCap; j += blockDim.x) buf[j] = worst;
    bitonic_desc(buf, kTopCap);
    for (int j = threadIdx.x; j < k; j += blockDim.x) out[(size_t)blockIdx.x * k + j] = buf[j];
}

// ---- complex64, k <= 128: warps that never wait for each other.  Each warp
// streams its own contiguous slice of the state, kTwStep amplitudes per step
// in 16-byte loads (two amplitudes per load, eight per lane), with the next
// step's loads in flight.  A float pre-filter against the warp's threshold
// marks the lanes' candidates; one vote skips the rest of the step when
// there are none (the common case once the threshold has risen).  Otherwise
// the candidates are tested in the exact (p, index) order and placed by
// ballot and prefix count into the warp's shared-memory buffer of CAP
// entries, FPC x 32 at a time; when the buffer could overflow the warp sorts
// it (bitonic, warp-synchronous) and cuts it to its best kw.  The block then
// merges its warps' lists into its best k, and the single-block pass merges
// the blocks'.
//
// A warp that keeps its best kw = k is exact.  Keeping fewer (kw = 16, a
// 64-entry buffer) cuts the sorts, which bound this kernel, about tenfold: a
// warp inserts about kw ln(slice / kw) candidates.  It is exact unless a
// warp dropped an element of the true top k, and that needs all kw of the
// warp's kept entries to be in the top k too (each beats the dropped one);
// the caller checks that on the result and reruns with kw = k if so.
constexpr int kTwWarps = 16;    // warps per block
constexpr int kTwStep = 256;    // amplitudes per warp step (8 per lane in 4 16-byte loads)
constexpr int kTwBlocksPerSM = 2;   // 32 warps per SM, 2 KB of loads in flight each
constexpr int kTwMaxK = 128;
constexpr int kTwCap = 256;     // exact mode: >= 128 kept + 128 placed between checks (FPC = 4)
constexpr int kTwCapKeep = 64;  // reduced mode: >= 32 kept + 32 placed between checks (FPC = 1)
static_assert(kTwStep % 64 == 0 && kTwCap >= kTwMaxK + 4 * 32 && kTwCapKeep >= 32 + 32, "buffer sizes");
static_assert(kTwWarps * kTopWarpKeep >= kTwMaxK && kTopWarpKeep <= 32, "a block's warps keep at least k");

// (stage loops kept rolled: the sort is inlined at every overflow check of
// the unrolled placement loop)
__device__ __forceinline__ void warp_bitonic_desc(KI *buf, int cap, int lane)
{
#pragma unroll 1
    for (int size = 2; size <= cap; size <<= 1) {
#pragma unroll 1
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncwarp();
            for (int t = lane; t < cap / 2; t += 32) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool desc = (lo & size) == 0;
                const KI x = buf[lo], y = buf[hi];
                if (desc ? better(y, x) : better(x, y)) { buf[lo] = y; buf[hi] = x; }
            }
        }
    }
    __syncwarp();
}

template <int CAP, int FPC>
__global__ void __launch_bounds__(32 * kTwWarps, kTwBlocksPerSM) k_topk_warp(const float2 *__restrict__ a, int64_t N, int k,
                                                                 int kw, KI *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char tw_raw[];
    KI *wbuf = (KI *)tw_raw;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    KI *buf = wbuf + (size_t)wid * CAP;
    const KI worst = {-1.0, ~0ull};
    const int64_t W = (int64_t)gridDim.x * kTwWarps, gw = (int64_t)blockIdx.x * kTwWarps + wid;
    const int64_t per = (((N + W - 1) / W) + kTwStep - 1) & ~(int64_t)(kTwStep - 1);   // whole steps
    const int64_t lo = gw * per < N ? gw * per : N, hi = lo + per < N ? lo + per : N;
    int cnt = 0;
    KI thr = worst;
    float thf = -1.0f;
    // lo, hi and every step start are multiples of kTwStep (N is a power of
    // two >= kTwStep * kTwWarps), so a step never straddles hi and each
    // 16-byte load holds amplitudes 2j, 2j + 1 of the slice
    const float4 *a4 = (const float4 *)a;
    constexpr int kL = kTwStep / 64;   // 16-byte loads per lane per step
    float4 nz[kL];
    auto load = [&](int64_t t0) {
#pragma unroll
        for (int e = 0; e < kL; e++) nz[e] = a4[(t0 >> 1) + e * 32 + lane];
    };
    if (lo < hi) load(lo);
    for (int64_t t0 = lo; t0 < hi; t0 += kTwStep) {
        float2 cz[2 * kL];
#pragma unroll
        for (int e = 0; e < kL; e++) {
            cz[2 * e] = make_float2(nz[e].x, nz[e].y);
            cz[2 * e + 1] = make_float2(nz[e].z, nz[e].w);
        }
        if (t0 + kTwStep < hi) load(t0 + kTwStep);
        // element f of this lane is amplitude t0 + 64 (f / 2) + 2 lane + (f & 1)
        unsigned pass = 0;
#pragma unroll
        for (int f = 0; f < 2 * kL; f++)
            if (fmaf(cz[f].x, cz[f].x, cz[f].y * cz[f].y) >= thf) pass |= 1u << f;
        if (!__any_sync(~0u, pass != 0)) continue;
#pragma unroll
        for (int f = 0; f < 2 * kL; f++) {
            KI v;
            bool c = false;
            if ((pass >> f) & 1) {
                v.p = prob_of(cz[f]);
                v.i = (uint64_t)(t0 + 64 * (f >> 1) + 2 * lane + (f & 1));
                c = better(v, thr);
            }
            const unsigned m = __ballot_sync(~0u, c);
            if (c) buf[cnt + __popc(m & ((1u << lane) - 1))] = v;
            cnt += __popc(m);
            if ((f + 1) % FPC == 0 && cnt > CAP - 32 * FPC) {   // sort and cut back to kw
                __syncwarp();
                for (int j = cnt + lane; j < CAP; j += 32) buf[j] = worst;
                warp_bitonic_desc(buf, CAP, lane);
                cnt = kw;
                thr = buf[kw - 1];
                thf = thr.p > 0 ? __double2float_rd(thr.p * (1.0 - 1e-5)) : -1.0f;
            }
        }
    }
    __syncwarp();
    for (int j = cnt + lane; j < CAP; j += 32) buf[j] = worst;
    warp_bitonic_desc(buf, CAP, lane);
    // block merge: the warps' best kw, gathered (through registers: the
    // regions overlap) into the first 16 kw entries, sorted; the block's best k
    __syncthreads();
    const int M = kTwWarps * kw;
    int P = 1;
    while (P < M) P <<= 1;
    KI tmp[(kTwWarps * kTwMaxK) / (32 * kTwWarps)];   // <= 4 per thread
    int nt = 0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) tmp[nt++] = wbuf[(size_t)(j / kw) * CAP + j % kw];
    __syncthreads();
    nt = 0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) wbuf[j] = tmp[nt++];
    for (int j = M + threadIdx.x; j < P; j += blockDim.x) wbuf[j] = worst;
    bitonic_desc(wbuf, P);
    for (int j = threadIdx.x; j < k; j += blockDim.x) out[(size_t)blockIdx.x * k + j] = wbuf[j];
}

bool topk_warp_suspect(const uint64_t *idx, int k, int64_t slice, int keep)
{
    if (slice <= 0 || keep <= 0 || k < keep) return false;
    std::vector<uint64_t> w(idx, idx + k);
    for (uint64_t &x : w) x /= (uint64_t)slice;
    std::sort(w.begin(), w.end());
    for (int i = 0; i + keep <= k; i++)
        if (w[i] == w[i + keep - 1]) return true;
    return false;
}

__global__ void k_topk_split(const KI *in, int k, uint64_t *idx, double *p)
{
    for (int j = threadIdx.x; j < k; j += blockDim.x) { idx[j] = in[j].i; p[j] = in[j].p; }
}

cudaError_t launch_topk(const void *a, int n, bool f64, int k, void *scratch, uint64_t *idx, double *p,
                        cudaStream_t st, int warp_keep, int64_t *warp_slice)
{
    if (k < 1 || k > 1024) return cudaErrorInvalidValue;
    if (warp_slice) *warp_slice = 0;
    int64_t N = (int64_t)1 << n;
    int G = topk_blocks(N);
    KI *lists = (KI *)scratch;
    KI *final_;
    if (!f64 && k <= kTwMaxK && N >= (int64_t)kTwStep * kTwWarps && ((uintptr_t)a & 15) == 0) {
        // blocks of independent warps, kTwBlocksPerSM per SM
        const int64_t steps = (N + kTwStep - 1) / kTwStep;   // at most one warp per step
        const int64_t gmax = (steps + kTwWarps - 1) / kTwWarps;
        G = (int)((int64_t)kTwBlocksPerSM * device_sm_count() < gmax ? (int64_t)kTwBlocksPerSM * device_sm_count()
                                                                          : gmax);
        final_ = lists + (size_t)G * k;
        const bool keep = warp_keep == kTopWarpKeep && warp_keep < k;
        static bool attr[2] = {false, false};
        const size_t smem = (size_t)kTwWarps * (keep ? kTwCapKeep : kTwCap) * sizeof(KI);
        auto kern = keep ? k_topk_warp<kTwCapKeep, 1> : k_topk_warp<kTwCap, 4>;
        if (!attr[keep]) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr[keep] = true;
        }
        kern<<<G, 32 * kTwWarps, smem, st>>>((const float2 *)a, N, k, keep ? warp_keep : k, lists);
        if (keep && warp_slice) {   // the warps' slice length, as the kernel computes it
            const int64_t W = (int64_t)G * kTwWarps;
            *warp_slice = (((N + W - 1) / W) + kTwStep - 1) & ~(int64_t)(kTwStep - 1);
        }
    } else {
        final_ = lists + (size_t)G * k;
        if (f64) k_topk<double, true><<<G, kTopThreads, 0, st>>>((const double2 *)a, nullptr, N, k, lists);
        else k_topk<float, true><<<G, kTopThreads, 0, st>>>((const float2 *)a, nullptr, N, k, lists);
    }
    k_topk<float, false><<<1, kTopThreads, 0, st>>>(nullptr, lists, (int64_t)G * k, k, final_);
    k_topk_split<<<1, 256, 0, st>>>(final_, k, idx, p);
    return counted(cudaGetLastError(), 3);
}

}  // namespace svs
