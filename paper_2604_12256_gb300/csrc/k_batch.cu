// k_batch.cu -- small circuits packed into one launch (the serving loop's
// batch path): CTA b runs request b's whole circuit on a state held in its
// shared memory (2^n amplitudes, n <= 13 complex64 / 12 complex128), then
// computes the request's read-out (<Z-string> values and top-k
// probabilities) in the same launch.  The state never touches HBM.
//
// Request ops (32-bit words, see batch.h): dense k-qubit gates (k <= 3) and
// phase polynomials (diagonal gates, fused by the diagonal detector).
#include <cstdint>

#include "batch.h"
#include "kernels.h"

namespace svs {

template <typename R> struct BT;
template <> struct BT<float> { using T2 = float2; };
template <> struct BT<double> { using T2 = double2; };

__device__ __forceinline__ float2 bcis(uint64_t w, float)
{
    float s, c;
    __sincosf((float)(int32_t)(uint32_t)((w + (1ull << 31)) >> 32) * 1.46291807926715968e-09f, &s, &c);
    const float f = fmaf(-0.5f, fmaf(c, c, s * s), 1.5f);
    return make_float2(c * f, s * f);
}
__device__ __forceinline__ double2 bcis(uint64_t w, double)
{
    double s, c;
    sincospi((double)(int64_t)w * 1.0842021724855044340e-19, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ double bprob(float2 v) { return fma((double)v.x, (double)v.x, (double)v.y * (double)v.y); }
__device__ __forceinline__ double bprob(double2 v) { return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)); }

__device__ __forceinline__ uint64_t bld64(const uint32_t *p) { return (uint64_t)p[0] | ((uint64_t)p[1] << 32); }

// block-wide sum of one double per thread (fixed order)
__device__ double bsum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += sh[i];
    return s;
}

template <typename R>
__global__ void __launch_bounds__(kBatchThreads) k_batch(const BatchReq *__restrict__ reqs,
                                                         const uint32_t *__restrict__ blob, double *__restrict__ outs)
{
    using T2 = typename BT<R>::T2;
    extern __shared__ __align__(16) unsigned char smraw[];
    const BatchReq rq = reqs[blockIdx.x];
    const int n = rq.n;
    const int N = 1 << n;
    T2 *st = (T2 *)smraw;
    double *pr = (double *)(st + N);              // probabilities (top-k)
    __shared__ double sh[kBatchThreads / 32];
    __shared__ double best_p[kBatchThreads / 32];
    __shared__ int best_i[kBatchThreads / 32];
    const int tid = threadIdx.x;

    for (int i = tid; i < N; i += kBatchThreads) {
        T2 z;
        z.x = (i == (int)rq.basis) ? (R)1 : (R)0;
        z.y = 0;
        st[i] = z;
    }
    __syncthreads();
    const uint32_t *op = blob + rq.ops_off;
    for (int o = 0; o < rq.nops; o++) {
        const uint32_t hdr = op[0];
        const int type = hdr & 0xff;
        if (type == BOP_DENSE) {
            const int k = (hdr >> 8) & 0xff;
            int q[3], sq[3];
            for (int i = 0; i < k; i++) q[i] = sq[i] = (int)op[1 + i];
            for (int i = 1; i < k; i++)
                for (int j = i; j > 0 && sq[j - 1] > sq[j]; j--) { int t = sq[j]; sq[j] = sq[j - 1]; sq[j - 1] = t; }
            const R *M = (const R *)(op + 4);
            const int D = 1 << k;
            for (int gi = tid; gi < (N >> k); gi += kBatchThreads) {
                int b = gi;
                for (int i = 0; i < k; i++) b = ((b >> sq[i]) << (sq[i] + 1)) | (b & ((1 << sq[i]) - 1));
                T2 x[8];
                int idx[8];
                for (int c = 0; c < D; c++) {
                    int off = 0;
                    for (int i = 0; i < k; i++) if ((c >> i) & 1) off |= 1 << q[i];
                    idx[c] = b | off;
                    x[c] = st[idx[c]];
                }
                for (int r = 0; r < D; r++) {
                    R re = 0, im = 0;
                    for (int c = 0; c < D; c++) {
                        const R mr = M[2 * (r * D + c)], mi = M[2 * (r * D + c) + 1];
                        re = fma(mr, x[c].x, fma(-mi, x[c].y, re));
                        im = fma(mr, x[c].y, fma(mi, x[c].x, im));
                    }
                    T2 y;
                    y.x = re;
                    y.y = im;
                    st[idx[r]] = y;
                }
            }
        } else {   // BOP_PHASE: exp(2 pi i sum_t w_t [x & mask_t == mask_t])
            const int nt = (int)op[1];
            const uint32_t *t = op + 2;
            for (int i = tid; i < N; i += kBatchThreads) {
                uint64_t w = 0;
                for (int j = 0; j < nt; j++) {
                    const uint64_t m = bld64(t + 4 * j);
                    if (((uint64_t)i & m) == m) w += bld64(t + 4 * j + 2);
                }
                const T2 f = bcis(w, (R)0);
                const T2 v = st[i];
                T2 y;
                y.x = v.x * f.x - v.y * f.y;
                y.y = v.x * f.y + v.y * f.x;
                st[i] = y;
            }
        }
        op += op[0] >> 16;   // op length in words (hdr bits 16..31)
        __syncthreads();
    }
    // ---- read-out: <Z-string> values, then top-k probabilities
    double *out = outs + rq.out_off;
    const uint64_t *masks = (const uint64_t *)(blob + rq.masks_off);
    for (int m = 0; m < rq.nmask; m++) {
        const uint64_t mk = masks[m];
        double acc = 0;
        for (int i = tid; i < N; i += kBatchThreads) {
            const double p = bprob(st[i]);
            acc += (__popcll((uint64_t)i & mk) & 1) ? -p : p;
        }
        const double s = bsum(acc, sh);
        if (tid == 0) out[m] = s;
    }
    if (rq.top_k <= 0) return;
    for (int i = tid; i < N; i += kBatchThreads) pr[i] = bprob(st[i]);
    __syncthreads();
    const int k = rq.top_k < N ? rq.top_k : N;
    double *op_p = out + rq.nmask;
    double *op_i = op_p + rq.top_k;
    for (int r = 0; r < k; r++) {
        // block-wide argmax, ties to the lower index
        double bp = -1.0;
        int bi = 0x7fffffff;
        for (int i = tid; i < N; i += kBatchThreads) {
            const double p = pr[i];
            if (p > bp || (p == bp && i < bi)) { bp = p; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double p2 = __shfl_down_sync(0xffffffffu, bp, o);
            const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
            if (p2 > bp || (p2 == bp && i2 < bi)) { bp = p2; bi = i2; }
        }
        if ((tid & 31) == 0) { best_p[tid >> 5] = bp; best_i[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            double p = best_p[0];
            int ii = best_i[0];
            for (int w = 1; w < kBatchThreads / 32; w++)
                if (best_p[w] > p || (best_p[w] == p && best_i[w] < ii)) { p = best_p[w]; ii = best_i[w]; }
            op_p[r] = p;
            op_i[r] = (double)ii;   // exact for indices < 2^53
            pr[ii] = -2.0;          // excluded from later rounds
        }
        __syncthreads();
    }
    for (int r = k + tid; r < rq.top_k; r += kBatchThreads) { op_p[r] = -1.0; op_i[r] = -1.0; }
}

size_t batch_smem_bytes(int n, bool f64) { return ((size_t)1 << n) * ((f64 ? 16 : 8) + 8); }

cudaError_t launch_batch(const BatchReq *reqs_dev, int nreq, int max_n, const uint32_t *blob_dev, double *outs_dev,
                         bool f64, cudaStream_t st)
{
    if (nreq <= 0) return cudaSuccess;
    const size_t smem = batch_smem_bytes(max_n, f64);
    static bool attr32 = false, attr64 = false;
    if (!f64 && !attr32) {
        cudaError_t e = cudaFuncSetAttribute(k_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)batch_smem_bytes(kBatchMaxN64, false));
        if (e != cudaSuccess) return e;
        attr32 = true;
    }
    if (f64 && !attr64) {
        cudaError_t e = cudaFuncSetAttribute(k_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)batch_smem_bytes(kBatchMaxN128, true));
        if (e != cudaSuccess) return e;
        attr64 = true;
    }
    if (f64) k_batch<double><<<nreq, kBatchThreads, smem, st>>>(reqs_dev, blob_dev, outs_dev);
    else k_batch<float><<<nreq, kBatchThreads, smem, st>>>(reqs_dev, blob_dev, outs_dev);
    return counted(cudaGetLastError(), 1);
}

}  // namespace svs
