// chunk_dev.cuh -- device code of the cache-blocked chunk sweep (K4) and the
// fused diagonal sweep (K3): program access, dense ops, phase segments, the
// per-chunk phase sums and the sweep itself.  Compiled by nvcc into the
// library's interpreter kernels (k_chunk.cu) and, as text, by the run-time
// compiler into kernels specialised to one program (jit.cpp): it uses no
// host headers.
#pragma once

#include "program.h"   // first: the fixed-width integer types under run-time compilation
#include "dfloat.h"

namespace svs {

using namespace prog;

template <typename R> struct CT;
template <> struct CT<float> {
    using T2 = float2;    // registers / shared memory
    using G2 = float2;    // HBM
    using W = uint32_t;
    static constexpr int SWZ = swizzle_bits(4);
};
template <> struct CT<double> {
    using T2 = dfc;
    using G2 = double2;
    using W = uint64_t;
    static constexpr int SWZ = swizzle_bits(8);
};

__device__ __forceinline__ float2 to_reg(float2 v) { return v; }
__device__ __forceinline__ float2 to_glob(float2 v) { return v; }

// Program words are read from the CTA's shared-memory copy of the program.
__device__ __forceinline__ uint32_t ldw(const uint32_t *p) { return *p; }
__device__ __forceinline__ uint64_t ld64(const uint32_t *p) { return (uint64_t)p[0] | ((uint64_t)p[1] << 32); }
// 128-bit read of 4 program words (the encoder aligns what is read this way)
__device__ __forceinline__ uint4 ld4(const uint32_t *p) { return *(const uint4 *)p; }

using namespace prog;

template <typename R> __device__ __forceinline__ typename CT<R>::W ldwt(const uint32_t *p);
template <> __device__ __forceinline__ uint32_t ldwt<float>(const uint32_t *p) { return *p; }
template <> __device__ __forceinline__ uint64_t ldwt<double>(const uint32_t *p) { return ld64(p); }

// complex element i of a dense op body or a complex table in the program:
// complex64 as (re, im) floats, complex128 as double-float (rh, rl, ih, il)
__device__ __forceinline__ float2 ldm(const float *b, int i) { return make_float2(b[2 * i], b[2 * i + 1]); }
__device__ __forceinline__ dfc ldm(const double *b, int i)
{
    const float4 q = ((const float4 *)b)[i];
    dfc r;
    r.rh = q.x;
    r.rl = q.y;
    r.ih = q.z;
    r.il = q.w;
    return r;
}
// element i of a 16-byte-aligned complex table: complex64 entries are read
// two per 128-bit load (the loads of i and i ^ 1 are the same word)
__device__ __forceinline__ float2 ldm_a(const float *b, int i)
{
    const float4 q = ((const float4 *)b)[i >> 1];
    return (i & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
}
__device__ __forceinline__ dfc ldm_a(const double *b, int i) { return ldm(b, i); }

// stage the program (H_WORDS words, 16-byte aligned in both spaces) in shared memory
template <int T>
__device__ __forceinline__ void stage_program(const uint32_t *__restrict__ g, uint32_t *s, int tid)
{
    const int nw = (int)__ldg(g + H_WORDS);
    const uint4 *g4 = (const uint4 *)g;
    uint4 *s4 = (uint4 *)s;
    for (int i = tid; i < (nw >> 2); i += T) s4[i] = __ldg(g4 + i);
    for (int i = (nw & ~3) + tid; i < nw; i += T) s[i] = __ldg(g + i);
}

// exp(2 pi i w / 2^bits) for the weight type
__device__ __forceinline__ float2 cis_turns(uint32_t w)
{
    float s, c;
    __sincosf((float)(int32_t)w * 1.46291807926715968e-09f, &s, &c);   // 2 pi / 2^32
    // one Newton step towards |c + i s| = 1 so that phases do not bias the norm
    const float f = fmaf(-0.5f, fmaf(c, c, s * s), 1.5f);
    return make_float2(c * f, s * f);
}
// complex128: cis(2 pi w / 2^64) = T0[w >> 56] T1[(w >> 48) & 255]
// T2[(w >> 40) & 255] cis(e), e = 2 pi (w mod 2^40) / 2^64 < 2 pi 2^-24, with
// cis(e) = (1 - e^2/2, e (1 - e^2/6)) (the next terms are below 1e-27).
// Tk[b] = cis(2 pi b / 2^(8k + 8)) as double-float, split from long-double
// values on the host (set_cis64_tables); the products run in double-float.
__device__ dfc g_cis64[3 * 256];   // double-float (rh, rl, ih, il)

__device__ __forceinline__ dfc cis_turns(uint64_t w)
{
    const dfc t0 = g_cis64[w >> 56];
    const dfc t1 = g_cis64[256 + ((w >> 48) & 255)];
    const dfc t2 = g_cis64[512 + ((w >> 40) & 255)];
    // e = 2 pi r / 2^64, r < 2^40 exact as a double-float (two 20-bit halves)
    const uint64_t r = w & ((1ull << 40) - 1);
    const float rh = (float)(uint32_t)(r >> 20) * 1048576.f, rl = (float)(uint32_t)(r & 0xFFFFF);
    constexpr float kh = 0x1.921fb6p-62f;    // 2 pi 2^-64 = kh + kl to 1e-15
    constexpr float kl = -0x1.777a5cp-87f;
    float eh, el;
    {
        const float ah[2] = {rh, rl}, al[2] = {0.f, 0.f}, bh[2] = {kh, kh}, bl[2] = {kl, kl};
        df_dot<2>(ah, al, bh, bl, eh, el);
    }
    const float e2 = eh * eh;   // < 1.4e-13: its float rounding is far below 1e-16 of 1
    dfc te;
    two_sum(1.f, -0.5f * e2, te.rh, te.rl);
    te.ih = eh;
    te.il = fmaf(-eh * (1.f / 6.f), e2, el);
    return cmul(cmul(cmul(t0, t1), t2), te);
}

// packed f32x2 arithmetic (sm_100+): a 64-bit register pair holds (re, im)
using u64 = unsigned long long;
__device__ __forceinline__ u64 pk2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ u64 pk(float2 v) { return pk2(v.x, v.y); }
__device__ __forceinline__ float2 upk(u64 r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 fmul2(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// complex64: one rounding order written out (a product, then a fused
// multiply-add), so that every kernel compiled from these templates -- by
// nvcc or at run time -- rounds alike whatever the compiler's contraction
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(__fmaf_rn(a.x, b.x, __fmul_rn(-a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

// Amplitude times a phase factor in packed f32x2 form (the specialised
// kernels' phase segments): v f = (v.x, v.y) * (f.x, f.x) + (v.y, v.x) *
// (-f.y, f.y), a packed product and a packed multiply-add per amplitude
// instead of four scalar operations.  The rounding differs from cmul's (the
// products v.x f.x and v.y f.x are rounded, not v.y f.y and v.y f.x), by at
// most an ulp of each component.  cmul_pk takes the factor already as its
// two packed operands (R = (re, re), I = (-im, im)), as a specialised
// kernel's parameter block holds its constant factors.
__device__ __forceinline__ float2 cmul_pk(float2 v, u64 R, u64 I)
{
    return upk(ffma2(pk2(v.y, v.x), I, fmul2(pk(v), R)));
}
__device__ __forceinline__ float2 cmul_f(float2 v, float2 f) { return cmul_pk(v, pk2(f.x, f.x), pk2(-f.y, f.y)); }

// shared-memory swizzle: phys(y) = y ^ fold_SWZ(y >> SWZ); linear over GF(2)
template <int SWZ, int C> __device__ __forceinline__ uint32_t swz(uint32_t y)
{
    uint32_t r = y;
#pragma unroll
    for (int s = SWZ; s < C; s += SWZ) r ^= (y >> s) & ((1u << SWZ) - 1);
    return r;
}

// ------------------------------------------------------------ dense ops
// complex64 2x2 on register bit P from its entries (re, im) m[0..7], row
// major: m x = (mr, mr) * x + (-mi, mi) * (x.im, x.re), packed f32x2
template <int NR, int P>
__device__ __forceinline__ void dense1_general_f(float2 (&v)[NR], const float (&m)[8])
{
    u64 Mr[4], Mi[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        Mr[i] = pk2(m[2 * i], m[2 * i]);
        Mi[i] = pk2(-m[2 * i + 1], m[2 * i + 1]);
    }
#pragma unroll
    for (int g = 0; g < NR; g++) {
        if (g & (1 << P)) continue;
        const float2 y0 = v[g], y1 = v[g | (1 << P)];
        const u64 x0 = pk(y0), x1 = pk(y1), s0 = pk2(y0.y, y0.x), s1 = pk2(y1.y, y1.x);
        v[g] = upk(ffma2(s0, Mi[0], ffma2(x0, Mr[0], ffma2(s1, Mi[1], fmul2(x1, Mr[1])))));
        v[g | (1 << P)] = upk(ffma2(s0, Mi[2], ffma2(x0, Mr[2], ffma2(s1, Mi[3], fmul2(x1, Mr[3])))));
    }
}
// complex64 special 2x2 forms from their real numbers a, b, c, d:
// DS_REAL [[a, b], [c, d]] (H, RY); DS_RX [[a, i b], [i c, d]] (RX)
template <int NR, int P, int SUB>
__device__ __forceinline__ void dense1_special_f(float2 (&v)[NR], float a, float b, float c, float d)
{
    if constexpr (SUB == DS_REAL) {
        const u64 A = pk2(a, a), B = pk2(b, b), Cc = pk2(c, c), D = pk2(d, d);
#pragma unroll
        for (int g = 0; g < NR; g++) {
            if (g & (1 << P)) continue;
            const u64 x0 = pk(v[g]), x1 = pk(v[g | (1 << P)]);
            v[g] = upk(ffma2(x0, A, fmul2(x1, B)));
            v[g | (1 << P)] = upk(ffma2(x0, Cc, fmul2(x1, D)));
        }
    } else {   // a x0 + i b x1, i c x0 + d x1
        const u64 A = pk2(a, a), D = pk2(d, d), B = pk2(-b, b), Cc = pk2(-c, c);
#pragma unroll
        for (int g = 0; g < NR; g++) {
            if (g & (1 << P)) continue;
            const float2 y0 = v[g], y1 = v[g | (1 << P)];
            const u64 x0 = pk(y0), x1 = pk(y1);
            const u64 s0 = pk2(y0.y, y0.x), s1 = pk2(y1.y, y1.x);   // i x = (-im, re) via the signs
            v[g] = upk(ffma2(x0, A, fmul2(s1, B)));
            v[g | (1 << P)] = upk(ffma2(x1, D, fmul2(s0, Cc)));
        }
    }
}

// Scaled one-qubit forms (specialised kernels): the op is s * N with N
// below and the sweep's product of the scalars s applied once elsewhere, so
// each output amplitude costs one packed f32x2 instruction.
__device__ __forceinline__ u64 fadd2(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fsub2(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// N = [[1, +-1], [+-1, +-1]] (H-like): row r is x0 + x1 (0), x0 - x1 (1) or x1 - x0 (2)
template <int NR, int P, int R0, int R1>
__device__ __forceinline__ void dense1_pm(float2 (&v)[NR])
{
#pragma unroll
    for (int g = 0; g < NR; g++) {
        if (g & (1 << P)) continue;
        const u64 x0 = pk(v[g]), x1 = pk(v[g | (1 << P)]);
        v[g] = upk(R0 == 0 ? fadd2(x0, x1) : R0 == 1 ? fsub2(x0, x1) : fsub2(x1, x0));
        v[g | (1 << P)] = upk(R1 == 0 ? fadd2(x0, x1) : R1 == 1 ? fsub2(x0, x1) : fsub2(x1, x0));
    }
}
// N = [[1, t0], [t1, 1]] real (RY-like)
template <int NR, int P>
__device__ __forceinline__ void dense1_rot(float2 (&v)[NR], float t0, float t1)
{
    const u64 A = pk2(t0, t0), B = pk2(t1, t1);
#pragma unroll
    for (int g = 0; g < NR; g++) {
        if (g & (1 << P)) continue;
        const u64 x0 = pk(v[g]), x1 = pk(v[g | (1 << P)]);
        v[g] = upk(ffma2(x1, A, x0));
        v[g | (1 << P)] = upk(ffma2(x0, B, x1));
    }
}
// N = [[1, i u0], [i u1, 1]] (RX-like): x0 + i u0 x1 = x0 + (-u0, u0) * (x1.im, x1.re)
template <int NR, int P>
__device__ __forceinline__ void dense1_rxn(float2 (&v)[NR], float u0, float u1)
{
    const u64 A = pk2(-u0, u0), B = pk2(-u1, u1);
#pragma unroll
    for (int g = 0; g < NR; g++) {
        if (g & (1 << P)) continue;
        const float2 y0 = v[g], y1 = v[g | (1 << P)];
        v[g] = upk(ffma2(pk2(y1.y, y1.x), A, pk(y0)));
        v[g | (1 << P)] = upk(ffma2(pk2(y0.y, y0.x), B, pk(y1)));
    }
}
// complex64 4x4 on register bits P0 < P1 from its entries (re, im) m[0..31],
// row major (specialised kernels: compile-time entries become immediate
// operands; the same multiply-add order as dense_apply's)
template <int NR, int P0, int P1>
__device__ __forceinline__ void dense2_f(float2 (&v)[NR], const float (&m)[32])
{
    constexpr int gm = (1 << P0) | (1 << P1);
#pragma unroll
    for (int g = 0; g < NR; g++) {
        if (g & gm) continue;
        float2 in[4];
#pragma unroll
        for (int c = 0; c < 4; c++) in[c] = v[g | ((c & 1) << P0) | (((c >> 1) & 1) << P1)];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            float re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float mr = m[8 * r + 2 * c], mi = m[8 * r + 2 * c + 1];
                re = fmaf(mr, in[c].x, re);
                re = fmaf(-mi, in[c].y, re);
                im = fmaf(mr, in[c].y, im);
                im = fmaf(mi, in[c].x, im);
            }
            v[g | ((r & 1) << P0) | (((r >> 1) & 1) << P1)] = make_float2(re, im);
        }
    }
}

template <int NR>
__device__ __forceinline__ void scale_all(float2 (&v)[NR], float s)
{
    const u64 S = pk2(s, s);
#pragma unroll
    for (int m = 0; m < NR; m++) v[m] = upk(fmul2(pk(v[m]), S));
}

template <typename R, int NR, int K, int P0, int P1>
__device__ __forceinline__ void dense_apply(typename CT<R>::T2 (&v)[NR], const uint32_t *body)
{
    using T2 = typename CT<R>::T2;
    constexpr int D = 1 << K;
    constexpr int gm = (1 << P0) | (K > 1 ? (1 << P1) : 0);
    const R *mb = (const R *)body;
    if constexpr (sizeof(R) == 8) {
        // complex128 in double-float: each output component is one
        // double-float dot product over the 2D real products
#pragma unroll
        for (int g = 0; g < NR; g++) {
            if (g & gm) continue;
            dfc in[D];
#pragma unroll
            for (int c = 0; c < D; c++) {
                const int off = ((c & 1) << P0) | (K > 1 ? (((c >> 1) & 1) << P1) : 0);
                in[c] = v[g | off];
            }
#pragma unroll
            for (int r = 0; r < D; r++) {
                float ah[2 * D], al[2 * D], bh[2 * D], bl[2 * D];
                float ch[2 * D], cl[2 * D], dh[2 * D], dl[2 * D];
#pragma unroll
                for (int c = 0; c < D; c++) {
                    const dfc m = ldm(mb, r * D + c);
                    // re: mr xr - mi xi      im: mr xi + mi xr
                    ah[2 * c] = m.rh, al[2 * c] = m.rl, bh[2 * c] = in[c].rh, bl[2 * c] = in[c].rl;
                    ah[2 * c + 1] = -m.ih, al[2 * c + 1] = -m.il, bh[2 * c + 1] = in[c].ih, bl[2 * c + 1] = in[c].il;
                    ch[2 * c] = m.rh, cl[2 * c] = m.rl, dh[2 * c] = in[c].ih, dl[2 * c] = in[c].il;
                    ch[2 * c + 1] = m.ih, cl[2 * c + 1] = m.il, dh[2 * c + 1] = in[c].rh, dl[2 * c + 1] = in[c].rl;
                }
                dfc o;
                df_dot<2 * D>(ah, al, bh, bl, o.rh, o.rl);
                df_dot<2 * D>(ch, cl, dh, dl, o.ih, o.il);
                const int off = ((r & 1) << P0) | (K > 1 ? (((r >> 1) & 1) << P1) : 0);
                v[g | off] = o;
            }
        }
        return;
    } else if constexpr (K == 1) {
        // complex64 2x2 (two 128-bit loads of the body)
        const float4 q0 = ((const float4 *)mb)[0], q1 = ((const float4 *)mb)[1];
        const float m[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        dense1_general_f<NR, P0>(v, m);
        return;
    } else {
        // complex64, K = 2: the 16 entries are re-read from shared memory for
        // every group to keep register pressure down
        T2 M1[K == 1 ? 4 : 1];
        if constexpr (K == 1) {
#pragma unroll
            for (int i = 0; i < 4; i++) M1[i] = ldm(mb, i);
        }
        auto M = [&](int i) -> T2 {
            if constexpr (K == 1) return M1[i];
            else return ldm(mb, i);
        };
#pragma unroll
        for (int g = 0; g < NR; g++) {
            if (g & gm) continue;
            T2 in[D];
#pragma unroll
            for (int c = 0; c < D; c++) {
                int off = ((c & 1) << P0) | (K > 1 ? (((c >> 1) & 1) << P1) : 0);
                in[c] = v[g | off];
            }
#pragma unroll
            for (int r = 0; r < D; r++) {
                R re = 0, im = 0;
#pragma unroll
                for (int c = 0; c < D; c++) {
                    const T2 mrc = M(r * D + c);
                    re = fma(mrc.x, in[c].x, re);
                    re = fma(-mrc.y, in[c].y, re);
                    im = fma(mrc.x, in[c].y, im);
                    im = fma(mrc.y, in[c].x, im);
                }
                int off = ((r & 1) << P0) | (K > 1 ? (((r >> 1) & 1) << P1) : 0);
                v[g | off].x = re;
                v[g | off].y = im;
            }
        }
    }
}

// 2x2 matrices with all-real entries (H, RY): 4 flops per amplitude;
// real diagonal and imaginary off-diagonal (RX): likewise
template <typename R, int NR, int P, int SUB>
__device__ __forceinline__ void dense1_special(typename CT<R>::T2 (&v)[NR], const uint32_t *body)
{
    if constexpr (sizeof(R) == 8) {
        // complex128 in double-float; a, b, c, d are the real numbers of the
        // special form (entry i of the body: floats 4i .. 4i + 3 = rh rl ih il)
        const float4 *f4 = (const float4 *)body;
        const float4 qa = f4[0], qb = f4[1], qc = f4[2], qd = f4[3];
        const float ah = qa.x, al = qa.y, dh = qd.x, dl = qd.y;
        const float bh = SUB == DS_REAL ? qb.x : qb.z, bl = SUB == DS_REAL ? qb.y : qb.w;
        const float ch = SUB == DS_REAL ? qc.x : qc.z, cl = SUB == DS_REAL ? qc.y : qc.w;
#pragma unroll
        for (int g = 0; g < NR; g++) {
            if (g & (1 << P)) continue;
            const dfc x0 = v[g], x1 = v[g | (1 << P)];
            dfc y0, y1;
            if constexpr (SUB == DS_REAL) {   // [[a, b], [c, d]] real
                const float p[2] = {ah, bh}, pl[2] = {al, bl}, q[2] = {ch, dh}, ql[2] = {cl, dl};
                { const float xh[2] = {x0.rh, x1.rh}, xl[2] = {x0.rl, x1.rl}; df_dot<2>(p, pl, xh, xl, y0.rh, y0.rl);
                  df_dot<2>(q, ql, xh, xl, y1.rh, y1.rl); }
                { const float xh[2] = {x0.ih, x1.ih}, xl[2] = {x0.il, x1.il}; df_dot<2>(p, pl, xh, xl, y0.ih, y0.il);
                  df_dot<2>(q, ql, xh, xl, y1.ih, y1.il); }
            } else {   // [[a, i b], [i c, d]]: a x0 + i b x1, i c x0 + d x1
                { const float p[2] = {ah, -bh}, pl[2] = {al, -bl}, xh[2] = {x0.rh, x1.ih}, xl[2] = {x0.rl, x1.il};
                  df_dot<2>(p, pl, xh, xl, y0.rh, y0.rl); }
                { const float p[2] = {ah, bh}, pl[2] = {al, bl}, xh[2] = {x0.ih, x1.rh}, xl[2] = {x0.il, x1.rl};
                  df_dot<2>(p, pl, xh, xl, y0.ih, y0.il); }
                { const float p[2] = {-ch, dh}, pl[2] = {-cl, dl}, xh[2] = {x0.ih, x1.rh}, xl[2] = {x0.il, x1.rl};
                  df_dot<2>(p, pl, xh, xl, y1.rh, y1.rl); }
                { const float p[2] = {ch, dh}, pl[2] = {cl, dl}, xh[2] = {x0.rh, x1.ih}, xl[2] = {x0.rl, x1.il};
                  df_dot<2>(p, pl, xh, xl, y1.ih, y1.il); }
            }
            v[g] = y0;
            v[g | (1 << P)] = y1;
        }
        return;
    } else {
        // complex64: one packed f32x2 op updates (re, im) together; entry i of
        // the row-major 2x2 matrix is (mb[2i], mb[2i+1]) (the op body is in the
        // shared-memory copy of the program: plain loads)
        const float4 m0 = ((const float4 *)body)[0], m1 = ((const float4 *)body)[1];
        dense1_special_f<NR, P, SUB>(v, m0.x, SUB == DS_REAL ? m0.z : m0.w, SUB == DS_REAL ? m1.x : m1.y, m1.z);
    }
}

// walk the (P0 < P1 < RB) combinations at compile time
template <typename R, int NR, int RB, int K, int P0, int P1>
struct DenseDispatch {
    static __device__ __forceinline__ void run(int code, int sub, typename CT<R>::T2 (&v)[NR], const uint32_t *body)
    {
        constexpr int mycode = K == 1 ? P0 : (P0 | (P1 << 3));
        if (code == mycode) {
            if constexpr (K == 1) {
                if (sub == DS_REAL) dense1_special<R, NR, P0, DS_REAL>(v, body);
                else if (sub == DS_RX) dense1_special<R, NR, P0, DS_RX>(v, body);
                else dense_apply<R, NR, K, P0, P1>(v, body);
            } else {
                dense_apply<R, NR, K, P0, P1>(v, body);
            }
            return;
        }
        if constexpr (K == 1) {
            if constexpr (P0 + 1 < RB) DenseDispatch<R, NR, RB, K, P0 + 1, 0>::run(code, sub, v, body);
        } else {
            if constexpr (P1 + 1 < RB) DenseDispatch<R, NR, RB, K, P0, P1 + 1>::run(code, sub, v, body);
            else if constexpr (P0 + 2 < RB) DenseDispatch<R, NR, RB, K, P0 + 1, P0 + 2>::run(code, sub, v, body);
        }
    }
};

// index of the lowest set bit; folds to a constant for unrolled loop indices
__host__ __device__ __forceinline__ constexpr int low_bit(int k)
{
    int j = 0;
    while (j < 31 && !((k >> j) & 1)) j++;
    return j;
}

// log2 of a power of two
__host__ __device__ __forceinline__ constexpr int log2_of(int x) { return low_bit(x); }

// ------------------------------------------------------------ phase segment
// Shared sums of a launch: cta_ph[d * SCP + s] (per chunk; SCP = 1 + RB + TB
// slots padded to 16 bytes; slots 1 + RB + i are coefficients of thread bit
// i) and thr_ph[(d * S + s) * T + tid] (per thread, segments d < nhoist),
// S = 1 + RB.
// MODE selects the paths compiled: 0 all of them, chosen per segment at run
// time (the interpreter); 1 factored without a register-only table; 2
// factored with it; 3 terms on several register bits and other bits (a
// specialised kernel knows its segments' shapes and compiles one path each).
template <typename R, int RB, int T, int MODE = 0>
__device__ __forceinline__ void dseg_apply(typename CT<R>::T2 (&v)[1 << RB], uint64_t x0, const uint32_t *body,
                                           const typename CT<R>::W *cta_ph, const typename CT<R>::W *thr_ph,
                                           int nhoist, int tid)
{
    using W = typename CT<R>::W;
    constexpr int NR = 1 << RB;
    constexpr int S = 1 + RB;
    constexpr int TB = log2_of(T);
    constexpr int SCP = (int)cta_stride(RB, TB, sizeof(W));
    const uint4 hd = ld4(body);   // D_INDEX, D_FLAGS, D_NBASE, D_NMULTI
    const int d = (int)hd.x;
    const bool hoisted = d < nhoist;
    const int nb = (int)hd.z;
    const int nm = (int)hd.w;
    uint32_t nlin[(RB + 3) & ~3];
#pragma unroll
    for (int k = 0; k < (RB + 3) / 4; k++) {
        const uint4 q = ld4(body + D_NLIN + 4 * k);
        nlin[4 * k] = q.x, nlin[4 * k + 1] = q.y, nlin[4 * k + 2] = q.z, nlin[4 * k + 3] = q.w;
    }
    const uint32_t *t = body + D_TERMS;
    // this chunk's sums of the segment: 128-bit loads of its padded slots
    W cv[SCP];
#pragma unroll
    for (int k = 0; k < SCP * (int)sizeof(W) / 16; k++) {
        const uint4 q = ((const uint4 *)(cta_ph + d * SCP))[k];
        if constexpr (sizeof(W) == 4) {
            cv[4 * k] = q.x, cv[4 * k + 1] = q.y, cv[4 * k + 2] = q.z, cv[4 * k + 3] = q.w;
        } else {
            cv[2 * k] = (W)q.x | ((W)q.y << 32), cv[2 * k + 1] = (W)q.z | ((W)q.w << 32);
        }
    }
    W base = cv[0];
#pragma unroll
    for (int i = 0; i < TB; i++)
        if ((tid >> i) & 1) base += cv[1 + RB + i];
    if (hoisted) base += thr_ph[(d * S) * T + tid];
    for (int i = 0; i < nb; i++, t += kTermWords) {
        uint64_t m = ld64(t);
        if ((x0 & m) == m) base += ldwt<R>(t + 2);
    }
    W lin[RB];
#pragma unroll
    for (int j = 0; j < RB; j++) {
        lin[j] = cv[1 + j];
        if (hoisted) lin[j] += thr_ph[(d * S + 1 + j) * T + tid];
        const int cnt = (int)nlin[j];
        for (int i = 0; i < cnt; i++, t += kTermWords) {
            uint64_t m = ld64(t);
            if ((x0 & m) == m) lin[j] += ldwt<R>(t + 2);
        }
    }
    const uint32_t *tab = t;
    const R *ctab = (const R *)(t + 2 * NR);   // cis of the register table
    const uint32_t *mt = t + 2 * NR + ctab_words(RB, sizeof(R));
    // (the pivot bit of the segment header is not used here: applying
    // cis(0) = 1 to the amplitudes it would skip is exact)
    const bool tabnz = (hd.y & 1) != 0;
    (void)tabnz;
    (void)mt;
    if constexpr (MODE != 3) {
    if (MODE != 0 || nm == 0) {
        // the phase of register index m is base + sum_j m_j lin[j], so its
        // factor is f[low bits of m] * g[high bits of m], both built from the
        // 1 + RB values cis(base), cis(lin[j]): 1 + RB sin/cos and about two
        // complex products per amplitude
        constexpr int LB = RB / 2, HB = RB - LB;
        typename CT<R>::T2 f[1 << LB], g[1 << HB];
        f[0] = cis_turns(base);
#pragma unroll
        for (int j = 0; j < LB; j++) {
            const auto cj = cis_turns(lin[j]);
#pragma unroll
            for (int m = 0; m < (1 << j); m++) f[m | (1 << j)] = cmul(f[m], cj);
        }
        g[0] = cone(f[0]);
#pragma unroll
        for (int j = 0; j < HB; j++) {
            const auto cj = cis_turns(lin[LB + j]);
            g[1 << j] = cj;
#pragma unroll
            for (int m = 1; m < (1 << j); m++) g[m | (1 << j)] = cmul(g[m], cj);
        }
        if constexpr (MODE == 0 || MODE == 2) {
            if (MODE == 2 || tabnz) {
#pragma unroll
                for (int m = 0; m < NR; m++) {
                    const int lo = m & ((1 << LB) - 1), hi = m >> LB;
                    const auto fg = hi == 0 ? f[lo] : cmul(f[lo], g[hi]);
                    v[m] = cmul(v[m], cmul(fg, ldm_a(ctab, m)));
                }
                return;
            }
        }
        if constexpr (MODE == 0 || MODE == 1) {
#pragma unroll
            for (int m = 0; m < NR; m++) {
                const int lo = m & ((1 << LB) - 1), hi = m >> LB;
                v[m] = cmul(v[m], hi == 0 ? f[lo] : cmul(f[lo], g[hi]));
            }
        }
        return;
    }
    }
    if constexpr (MODE == 0 || MODE == 3) {
    W ph = base;
#pragma unroll
    for (int k = 0; k < NR; k++) {
        const int m = k ^ (k >> 1);
        if (k > 0) {
            const int j = low_bit(k);
            if ((m >> j) & 1) ph += lin[j];
            else ph -= lin[j];
        }
        W p = ph + ldwt<R>(tab + 2 * m);
        for (int i = 0; i < nm; i++) {
            const uint32_t *q = mt + i * kMultiWords;
            uint64_t mm = ld64(q);
            uint32_t rm = ldw(q + 2);
            if ((x0 & mm) == mm && ((uint32_t)m & rm) == rm) p += ldwt<R>(q + 4);
        }
        v[m] = cmul(v[m], cis_turns(p));
    }
    }
}

// Per-thread sums of the thread table (once per launch; each thread owns its
// column, so no synchronisation is needed before its own use).
template <typename R, int T>
__device__ __forceinline__ void thread_sums(const uint32_t *prog, typename CT<R>::W *thr_ph, int nslots, int tid)
{
    using W = typename CT<R>::W;
    for (int i = 0; i < nslots; i++) thr_ph[i * T + tid] = 0;
    const uint32_t *tt = prog + ldw(prog + H_THR_OFF);
    const int nt = (int)ldw(prog + H_NTHR);
    for (int i = 0; i < nt; i++, tt += kThrWords) {
        const uint32_t tm = ldw(tt + 1);
        if (((uint32_t)tid & tm) == tm) thr_ph[ldw(tt) * T + tid] += ldwt<R>(tt + 2);
    }
}

__device__ __forceinline__ void add_atomic(uint32_t *p, uint32_t v) { atomicAdd((unsigned int *)p, (unsigned int)v); }
__device__ __forceinline__ void add_atomic(uint64_t *p, uint64_t v)
{
    atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

// Per-chunk sums of the CTA table, in one of kCtaBuffers buffers of
// `nslots` slots: cta_zero clears a buffer, cta_accum adds the entries whose
// mask chunk base `base` meets (block-wide; integer adds are exact, so the
// atomics' order does not matter).  The caller puts a barrier between the
// two and another before the sums are read.
template <typename R, int T>
__device__ __forceinline__ void cta_zero(typename CT<R>::W *buf, int nslots, int tid)
{
    for (int i = tid; i < nslots; i += T) buf[i] = 0;
}
template <typename R, int T>
__device__ __forceinline__ void cta_accum(const uint32_t *prog, typename CT<R>::W *cta_ph, uint64_t base, int tid)
{
    const uint32_t *ct = prog + ldw(prog + H_CTA_OFF);
    const int nc = (int)ldw(prog + H_NCTA);
    for (int i = tid; i < nc; i += T) {
        const uint32_t *e = ct + i * kCtaWords;
        const uint64_t m = ld64(e + 2);
        if ((base & m) == m) add_atomic(&cta_ph[ldw(e)], ldwt<R>(e + 4));
    }
}

// Sweep input from a fused merge-booster product (TensorSrc in kernels.h):
// amplitude x = hi[x >> n_lo] * lo[x & (2^n_lo - 1)], with the arithmetic of
// k_tensor.  hi == nullptr: the sweep reads the state itself.
template <typename T2> struct TSrc {
    const T2 *hi;
    const T2 *lo;
    int n_lo;
};
template <typename T2> __device__ __forceinline__ T2 tensor_amp(const TSrc<T2> &s, uint64_t x)
{
    const T2 h = __ldg(&s.hi[x >> s.n_lo]);
    const T2 l = __ldg(&s.lo[x & ((1ull << s.n_lo) - 1)]);
    return cmul(h, l);
}

// The sweep's helper lambdas are always inlined (their arrays must stay in
// registers), also when a kernel is compiled with reduced optimisation.
#define SVS_INLINE_LAMBDA __attribute__((always_inline))

// A compile-time stage index: kernels specialised to a program run each
// register stage as its own instantiation (Ops::run_s<..., S>), so the
// compiler never sees one stage's ops inlined into another's.
template <int S> struct StageIdx {
    static constexpr int value = S;
};
__device__ __forceinline__ constexpr int stage_of(int s) { return s; }
template <int S> __device__ __forceinline__ constexpr int stage_of(StageIdx<S>) { return S; }
template <int S, int N, typename F> __device__ __forceinline__ void for_stages(F &f)
{
    if constexpr (S < N) {
        f(StageIdx<S>{});
        for_stages<S + 1, N>(f);
    }
}

// ------------------------------------------------------------ K4 chunk sweep
// The sweep over all chunks; `Ops` supplies the register stages' op
// sequence: InterpOps walks the program in shared memory, a run-time
// specialised kernel (jit.cpp) supplies straight-line code for one program
// (kStages > 0: the stage count and stage layouts are compile-time).
template <typename R, int C, int RB, typename Ops>
__device__ __forceinline__ void chunk_sweep(typename CT<R>::G2 *__restrict__ a, const uint32_t *__restrict__ gprog,
                                            int n, TSrc<typename CT<R>::G2> src, const typename Ops::Params &P)
{
    using T2 = typename CT<R>::T2;
    using G2 = typename CT<R>::G2;
    using W = typename CT<R>::W;
    constexpr int TB = C - RB;
    constexpr int T = 1 << TB;
    constexpr int NR = 1 << RB;
    constexpr int SW = CT<R>::SWZ;
    constexpr int S = 1 + RB;
    constexpr int SCP = (int)cta_stride(RB, TB, sizeof(typename CT<R>::W));
    extern __shared__ __align__(16) unsigned char smraw[];
    T2 *sv = (T2 *)smraw;   // the chunk: interleaved (re, im), swizzled
    uint32_t *prog = (uint32_t *)(sv + (1 << C));
    const int tid = threadIdx.x;
    stage_program<T>(gprog, prog, tid);
    __syncthreads();
    const int nd = (int)ldw(prog + H_NDSEG);
    const int nhoist = (int)ldw(prog + H_NHOIST);
    W *cta_buf = (W *)(prog + ((ldw(prog + H_WORDS) + 3) & ~3u));
    const int cbw = (int)(cta_buffer_bytes(nd, RB, TB, sizeof(W)) / sizeof(W));   // words of one buffer
    W *thr_ph = cta_buf + kCtaBuffers * cbw;
    __shared__ uint64_t s_git[NR / 2];    // global offset of load iteration `it`
    __shared__ uint32_t s_sit[NR / 2];    // swizzled smem position of `it` on the store
    __shared__ uint64_t s_dep[768];       // chunk number byte k -> its free-qubit bits

    int qin[C];
#pragma unroll
    for (int i = 0; i < C; i++) qin[i] = (int)ldw(prog + H_QIN + i);
    int sperm[C];
#pragma unroll
    for (int i = 0; i < C; i++) sperm[i] = (int)ldw(prog + H_SPERM + i);
    const uint64_t freem = ld64(prog + H_FREE_LO);
    const int nst = (int)ldw(prog + H_NSTAGE);

    // element pair e = it * T + tid covers chunk indices y = 2e, 2e + 1:
    // y bit 0 = pair member, bits 1..TB = tid, bits TB+1.. = it
    uint64_t g_tid = 0;
    uint32_t st_tid = 0;   // store: chunk position of output index 2*tid
#pragma unroll
    for (int i = 0; i < TB; i++)
        if ((tid >> i) & 1) { g_tid |= 1ull << qin[i + 1]; st_tid |= 1u << sperm[i + 1]; }
    const uint32_t st_one = 1u << sperm[0];
    if (tid < NR / 2) {
        uint64_t g = 0;
        uint32_t sp = 0;
#pragma unroll
        for (int b = 0; b < RB - 1; b++)
            if ((tid >> b) & 1) { g |= 1ull << qin[TB + 1 + b]; sp |= 1u << sperm[TB + 1 + b]; }
        s_git[tid] = g;
        s_sit[tid] = swz<SW, C>(sp);
    }
    thread_sums<R, T>(prog, thr_ph, nhoist * S, tid);
    // deposit tables: entry 256 k + i = the chunk-number bits i << 8k spread
    // over the free qubits (n - C <= 22 < 24 bits)
    for (int e = tid; e < 768; e += T) {
        const int k = e >> 8;
        uint64_t b = 0, fm = freem, cv = (uint64_t)(e & 255) << (8 * k);
        while (fm) {
            uint64_t low = fm & (~fm + 1);
            if (cv & 1) b |= low;
            cv >>= 1;
            fm ^= low;
        }
        s_dep[e] = b;
    }
    // this thread's part of every stage's layout (the same for all chunks)
    uint64_t *s_x0 = (uint64_t *)((unsigned char *)thr_ph + (((size_t)nhoist * S * T * sizeof(W) + 15) & ~(size_t)15));
    uint32_t *s_pb = (uint32_t *)(s_x0 + (size_t)nst * T);
    for (int s = 0; s < nst; s++) {
        const uint32_t *sp = prog + ldw(prog + H_STAGE_OFF + s);
        uint32_t ybase = 0;
        uint64_t x0t = 0;
        for (int i = 0; i < TB; i++) {
            if ((tid >> i) & 1) {
                ybase |= 1u << ldw(sp + S_THR + i);
                x0t |= 1ull << ldw(sp + S_GTHR + i);
            }
        }
        s_x0[s * T + tid] = x0t;
        s_pb[s * T + tid] = swz<SW, C>(ybase);
    }
    cta_zero<R, T>(cta_buf, 2 * cbw, tid);
    __syncthreads();
    const uint32_t pst_tid = swz<SW, C>(st_tid);
    const uint32_t pst_one = swz<SW, C>(st_one);
    const uint32_t pld_tid = swz<SW, C>((uint32_t)tid << 1);

    const int64_t nchunks = (int64_t)1 << (n - C);
    // chunk base: spread the chunk number over the free (non-chunk) qubits
    // (deposit is linear over disjoint input bytes: three 256-entry tables)
    auto chunk_base = [&](int64_t chn) SVS_INLINE_LAMBDA {
        const uint64_t c = (uint64_t)chn;
        return s_dep[c & 255] | s_dep[256 + ((c >> 8) & 255)] | s_dep[512 + ((c >> 16) & 255)];
    };
    if (blockIdx.x < nchunks) cta_accum<R, T>(prog, cta_buf, chunk_base(blockIdx.x), tid);
    __syncthreads();
    // Ops::kFed: 1 the sweep's input is a merge-booster product (src.hi set),
    // 0 it is the state, -1 decided by src.hi at run time (the interpreter)
    const bool fed = Ops::kFed < 0 ? src.hi != nullptr : Ops::kFed > 0;
    // coalesced loads of one chunk's amplitude pairs into registers
    auto load_regs = [&](T2 (&dst)[NR], uint64_t b) SVS_INLINE_LAMBDA {
        if (fed) {
#pragma unroll
            for (int it = 0; it < NR / 2; it++) {
                const uint64_t g = b | g_tid | s_git[it];
                dst[2 * it] = to_reg(tensor_amp(src, g));
                dst[2 * it + 1] = to_reg(tensor_amp(src, g + 1));
            }
            return;
        }
#pragma unroll
        for (int it = 0; it < NR / 2; it++) {
            const uint64_t g = b | g_tid | s_git[it];
            if constexpr (sizeof(R) == 4) {
                float4 q = __ldcs((const float4 *)(a + g));
                dst[2 * it] = make_float2(q.x, q.y);
                dst[2 * it + 1] = make_float2(q.z, q.w);
            } else {
                dst[2 * it] = to_reg(__ldcs(a + g));
                dst[2 * it + 1] = to_reg(__ldcs(a + g + 1));
            }
        }
    };
    // a direct stage (program.h: specialised kernels only) moves its own
    // amplitudes between HBM and registers: register index m of the thread
    // whose stage-s thread bits are at xb is amplitude xb | Ops::roff(s, m)
    auto load_direct = [&](T2 (&dst)[NR], uint64_t xb, int s) SVS_INLINE_LAMBDA {
#pragma unroll
        for (int m = 0; m < NR; m++) {
            const uint64_t g = xb | Ops::roff(s, m);
            if (fed) {
                dst[m] = to_reg(tensor_amp(src, g));
            } else if constexpr (sizeof(R) == 4) {
                if (Ops::paired(s)) {   // m, m + 1 adjacent: one 16-byte load
                    if (m & 1) continue;
                    const float4 q = __ldcs((const float4 *)(a + g));
                    dst[m] = make_float2(q.x, q.y);
                    dst[m + 1] = make_float2(q.z, q.w);
                } else {
                    dst[m] = __ldcs(a + g);
                }
            } else {
                dst[m] = to_reg(__ldcs(a + g));
            }
        }
    };
    auto store_direct = [&](const T2 (&val)[NR], uint64_t xb, int s) SVS_INLINE_LAMBDA {
#pragma unroll
        for (int m = 0; m < NR; m++) {
            const uint64_t g = xb | Ops::roff(s, m);
            if constexpr (sizeof(R) == 4) {
                if (Ops::paired(s)) {
                    if (m & 1) continue;
                    __stcs((float4 *)(a + g), make_float4(val[m].x, val[m].y, val[m + 1].x, val[m + 1].y));
                } else {
                    __stcs(a + g, val[m]);
                }
            } else {
                __stcs(a + g, to_glob(val[m]));
            }
        }
    };
    constexpr bool kDF = Ops::kDirectFirst, kDL = Ops::kDirectLast;
    // Loads ahead (Ops::kPrefetch, the specialised kernels): the next chunk's
    // amplitudes are loaded into registers (nx) as soon as this chunk's first
    // stage has taken its own, so a whole chunk of loads stays in flight
    // through the register stages and the store (64 registers more per
    // thread: two CTAs per SM).  A sweep fed by a merge-booster product runs a
    // kernel of its own (Ops::kFed = 1) that computes the next chunk's
    // products ahead the same way.  The interpreter has no register double
    // buffer: it fits in 80 registers and three CTAs per SM, whose loads
    // overlap each other's stages.
    constexpr bool kPF = Ops::kPrefetch;
    const bool pf_on = kPF;
    T2 nx[kPF ? NR : 1];
    int64_t ch = blockIdx.x;
    uint64_t base = chunk_base(ch);
    if constexpr (kPF) {
        if (pf_on && ch < nchunks) {
            if constexpr (kDF) load_direct(nx, base | s_x0[tid], 0);
            else load_regs(nx, base);
        }
    }
    int cb = 0;   // CTA-table buffer of this chunk
    for (; ch < nchunks; ch += gridDim.x) {
        const W *cta_ph = cta_buf + cb * cbw;
        W *cta_next = cta_buf + (cb == 2 ? 0 : cb + 1) * cbw;
        const int64_t nch = ch + gridDim.x;
        const uint64_t nbase = nch < nchunks ? chunk_base(nch) : 0;
        T2 v0[NR];   // stage 0's amplitudes when it loads them itself
        if constexpr (kDF) {
            if (kPF && pf_on) {
#pragma unroll
                for (int m = 0; m < NR; m++) v0[m] = nx[kPF ? m : 0];
            } else {
                load_direct(v0, base | s_x0[tid], 0);
            }
        } else {
            T2 pf[NR];
            if (kPF && pf_on) {
#pragma unroll
                for (int m = 0; m < NR; m++) pf[m] = nx[kPF ? m : 0];
            } else {
                load_regs(pf, base);
            }
            // ---- the chunk -> shared
#pragma unroll
            for (int it = 0; it < NR / 2; it++) {
                const uint32_t p = pld_tid ^ swz<SW, C>((uint32_t)it << (TB + 1));
                sv[p] = pf[2 * it];
                sv[p ^ 1] = pf[2 * it + 1];
            }
        }
        if constexpr (kPF) {
            // the next chunk's loads, in flight through this chunk's stages
            if (pf_on && nch < nchunks) {
                if constexpr (kDF) load_direct(nx, nbase | s_x0[tid], 0);
                else load_regs(nx, nbase);
            }
        }
        // buffer (cb + 2) mod 3: last read by the previous chunk
        cta_zero<R, T>(cta_buf + (cb == 0 ? 2 : cb - 1) * cbw, nd * SCP, tid);
        // (the chunk in shared memory; with a direct first stage nothing
        // before the first stage's own store needs a barrier: the CTA
        // buffers it reads were completed before the last chunk's barriers)
        if constexpr (!kDF) __syncthreads();
        // the next chunk's sums (its buffer was cleared during the previous chunk)
        if (nch < nchunks) cta_accum<R, T>(prog, cta_next, nbase, tid);
        // ---- register stages
        auto stage = [&](auto si) SVS_INLINE_LAMBDA {
            const int s = stage_of(si);
            const uint32_t *sp = prog + Ops::stage_off(prog, s);
            uint32_t pv[(RB + 3) & ~3];
            Ops::template stage_pv<RB>(sp, s, pv);
            const uint64_t x0 = base | s_x0[s * T + tid];
            const uint32_t pb = s_pb[s * T + tid];
            T2 v[NR];
            if (kDF && s == 0) {
#pragma unroll
                for (int m = 0; m < NR; m++) v[m] = v0[m];
            } else {
#pragma unroll
                for (int m = 0; m < NR; m++) {
                    uint32_t pm = pb;
#pragma unroll
                    for (int j = 0; j < RB; j++)
                        if ((m >> j) & 1) pm ^= pv[j];
                    v[m] = sv[pm];
                }
            }
            if constexpr (Ops::kStages > 0)
                Ops::template run_s<R, RB, T, decltype(si)::value>(v, x0, prog, sp, cta_ph, thr_ph, nhoist, tid, P);
            else
                Ops::template run<R, RB, T>(s, v, x0, prog, sp, cta_ph, thr_ph, nhoist, tid, P);
            if (kDL && s == Ops::kStages - 1) {
                store_direct(v, x0, s);
                return;
            }
            // make the compiler rebuild the 2^RB addresses here instead of
            // keeping them live across the ops (register pressure); the
            // specialised kernels' offsets are constants
            uint32_t pbw = pb;
            if constexpr (Ops::kStages == 0) {
                asm volatile("" : "+r"(pbw));
#pragma unroll
                for (int j = 0; j < RB; j++) asm volatile("" : "+r"(pv[j]));
            }
#pragma unroll
            for (int m = 0; m < NR; m++) {
                uint32_t pm = pbw;
#pragma unroll
                for (int j = 0; j < RB; j++)
                    if ((m >> j) & 1) pm ^= pv[j];
                sv[pm] = v[m];
            }
            __syncthreads();
        };
        if constexpr (Ops::kStages > 0) {
            for_stages<0, Ops::kStages>(stage);
        } else {
            for (int s = 0; s < nst; s++) stage(s);
        }
        // ---- store: shared -> HBM, output bit i' takes chunk bit sperm[i']
#pragma unroll
        for (int it = 0; it < (kDL ? 0 : NR / 2); it++) {
            const uint64_t g = base | g_tid | s_git[it];
            const uint32_t p0 = pst_tid ^ s_sit[it];
            const uint32_t p1 = p0 ^ pst_one;
            if constexpr (sizeof(R) == 4) {
                const T2 u0 = sv[p0], u1 = sv[p1];
                float4 q = make_float4(u0.x, u0.y, u1.x, u1.y);
                __stcs((float4 *)(a + g), q);
            } else {
                __stcs(a + g, to_glob(sv[p0]));
                __stcs(a + g + 1, to_glob(sv[p1]));
            }
        }
        __syncthreads();
        base = nbase;
        cb = cb == 2 ? 0 : cb + 1;
    }
}


// The numbers a kernel specialised to one program reads from its parameter
// block (jit.cpp); the interpreters read everything from the program.
struct NoParams {};

// The interpreter: the ops of stage s, as the program in shared memory lists them.
struct InterpOps {
    using Params = NoParams;
    static constexpr int kStages = 0;
    static constexpr bool kPrefetch = false;
    static constexpr int kFed = -1;   // fed by a product or not: decided at run time
    static constexpr bool kDirectFirst = false, kDirectLast = false;
    static __device__ __forceinline__ uint64_t roff(int, int) { return 0; }
    static __device__ __forceinline__ bool paired(int) { return false; }
    static __device__ __forceinline__ uint32_t stage_off(const uint32_t *prog, int s)
    {
        return ldw(prog + H_STAGE_OFF + s);
    }
    template <int RB>
    static __device__ __forceinline__ void stage_pv(const uint32_t *sp, int, uint32_t (&pv)[(RB + 3) & ~3])
    {
#pragma unroll
        for (int k = 0; k < (RB + 3) / 4; k++) {
            const uint4 q = ld4(sp + S_PV + 4 * k);
            pv[4 * k] = q.x, pv[4 * k + 1] = q.y, pv[4 * k + 2] = q.z, pv[4 * k + 3] = q.w;
        }
    }
    template <typename R, int RB, int T>
    static __device__ __forceinline__ void run(int, typename CT<R>::T2 (&v)[1 << RB], uint64_t x0,
                                               const uint32_t *, const uint32_t *sp, const typename CT<R>::W *cta_ph,
                                               const typename CT<R>::W *thr_ph, int nhoist, int tid, const Params &)
    {
        constexpr int NR = 1 << RB;
        const int nops = (int)ldw(sp + S_NOPS);
        const uint32_t *op = sp + S_SIZE;
        for (int k = 0; k < nops; k++) {
            const uint32_t hdr = ldw(op + O_HDR);
            const int type = hdr & 0xff;
            if (type == OP_DENSE) {
                const int kq = (hdr >> 8) & 0xf;
                const int sub = (hdr >> 12) & 0xf;
                const int code = (int)(hdr >> 16);
                if (kq == 1) DenseDispatch<R, NR, RB, 1, 0, 0>::run(code, sub, v, op + O_BODY);
                else DenseDispatch<R, NR, RB, 2, 0, 1>::run(code, sub, v, op + O_BODY);
            } else {
                dseg_apply<R, RB, T>(v, x0, op + O_BODY, cta_ph, thr_ph, nhoist, tid);
            }
            op += ldw(op + O_WORDS);
        }
    }
};

// ------------------------------------------------------------ K3 diagonal sweep
// tile of 2^C consecutive amplitudes, C = 7 + RB: thread t holds amplitudes
// tile + t + m * 128 (register bits on top -> each warp load is contiguous)
// `Ops::seg` applies the sweep's one phase segment to a thread's amplitudes:
// DiagInterp decodes it from the program, a kernel specialised to the
// program (jit.cpp) is generated from it.
template <typename R, int RB, typename Ops>
__device__ __forceinline__ void diag_sweep(typename CT<R>::G2 *__restrict__ a, const uint32_t *__restrict__ gprog,
                                           int n, TSrc<typename CT<R>::G2> src, const typename Ops::Params &P)
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
        Ops::template seg<R, RB, 128>(v, x0, prog, op, cta_ph, thr_ph, nhoist, tid, P);
#pragma unroll
        for (int m = 0; m < NR; m++) __stcs(a + x0 + ((uint64_t)m << 7), to_glob(v[m]));
        __syncthreads();
        cb = cb == 2 ? 0 : cb + 1;
    }
}

struct DiagInterp {
    using Params = NoParams;
    template <typename R, int RB, int T>
    static __device__ __forceinline__ void seg(typename CT<R>::T2 (&v)[1 << RB], uint64_t x0, const uint32_t *,
                                               const uint32_t *op, const typename CT<R>::W *cta_ph,
                                               const typename CT<R>::W *thr_ph, int nhoist, int tid, const Params &)
    {
        dseg_apply<R, RB, T>(v, x0, op, cta_ph, thr_ph, nhoist, tid);
    }
};

}  // namespace svs
