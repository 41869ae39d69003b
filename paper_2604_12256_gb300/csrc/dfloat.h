// dfloat.h -- double-float arithmetic on the FP32 pipe: a real as hi + lo
// (two floats, about 48 significant bits), complex128 amplitudes as four
// floats.  The FP64 rate of this GPU is 1/64 of its FP32 rate, so the
// complex128 paths of the sweep kernels compute in these pairs and convert
// to and from complex128 once per load and store.  Error-free transforms:
// Knuth's two-sum and the FMA two-product.
#pragma once

#if !defined(__CUDACC_RTC__)
#include <cstdint>
#include <cuda_runtime.h>
#endif

namespace svs {

// complex128 amplitude in registers and shared memory
struct __align__(16) dfc {
    float rh, rl, ih, il;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float v = s - a;
    e = (a - (s - v)) + (b - v);
}
// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ void quick_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}
// acc (s + e) += a * b for double-float reals a = ah + al, b = bh + bl
__device__ __forceinline__ void df_fma_acc(float ah, float al, float bh, float bl, float &s, float &e)
{
    const float p = ah * bh;
    float pe = fmaf(ah, bh, -p);
    pe = fmaf(ah, bl, pe);
    pe = fmaf(al, bh, pe);
    float t;
    two_sum(s, p, s, t);
    e += t + pe;
}
// sum_k a_k b_k of double-float reals, accumulated in double-float: each
// product p + its FMA error, the p's summed by two-sum, the low parts and
// cross terms added to the error word
template <int N>
__device__ __forceinline__ void df_dot(const float (&ah)[N], const float (&al)[N], const float (&bh)[N],
                                       const float (&bl)[N], float &rh, float &rl)
{
    float s = 0.f, e = 0.f;
#pragma unroll
    for (int k = 0; k < N; k++) df_fma_acc(ah[k], al[k], bh[k], bl[k], s, e);
    quick_two_sum(s, e, rh, rl);
}
// a * b for double-float complex
__device__ __forceinline__ dfc cmul(dfc a, dfc b)
{
    dfc r;
    {
        const float ah[2] = {a.rh, -a.ih}, al[2] = {a.rl, -a.il}, bh[2] = {b.rh, b.ih}, bl[2] = {b.rl, b.il};
        df_dot<2>(ah, al, bh, bl, r.rh, r.rl);
    }
    {
        const float ah[2] = {a.rh, a.ih}, al[2] = {a.rl, a.il}, bh[2] = {b.ih, b.rh}, bl[2] = {b.il, b.rl};
        df_dot<2>(ah, al, bh, bl, r.ih, r.il);
    }
    return r;
}
// the complex number 1 in the type of x
__device__ __forceinline__ float2 cone(float2) { return make_float2(1.f, 0.f); }
__device__ __forceinline__ dfc cone(dfc)
{
    dfc r;
    r.rh = 1.f;
    r.rl = r.ih = r.il = 0.f;
    return r;
}
// complex128 <-> double-float complex, in bit operations plus one FP64 add
// per real (the conversions would otherwise take the FP64 pipe too).  A
// double is truncated to float's 24-bit significand; magnitudes below 2^-126
// become 0 (amplitudes that small are far below every tolerance).
__device__ __forceinline__ float trunc_to_float(double d)
{
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    if (e < 1023 - 126) return __uint_as_float(sign);
    return __uint_as_float(sign | ((uint32_t)(e - 1023 + 127) << 23) | (uint32_t)((b >> 29) & 0x7FFFFF));
}
__device__ __forceinline__ double widen(float f)   // exact; float subnormals become 0
{
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xFF;
    if (e == 0) return __longlong_as_double((long long)sign);
    return __longlong_as_double((long long)(sign | ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)(u & 0x7FFFFF) << 29)));
}
__device__ __forceinline__ void split_df(double d, float &h, float &l)
{
    h = trunc_to_float(d);
    l = trunc_to_float(d - widen(h));   // d - h is exact
}
__device__ __forceinline__ dfc to_reg(double2 d)
{
    dfc r;
    split_df(d.x, r.rh, r.rl);
    split_df(d.y, r.ih, r.il);
    return r;
}

__device__ __forceinline__ double2 to_glob(dfc v)
{
    return make_double2(widen(v.rh) + widen(v.rl), widen(v.ih) + widen(v.il));
}

}  // namespace svs
