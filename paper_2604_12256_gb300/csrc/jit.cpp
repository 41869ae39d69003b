// jit.cpp -- sweep kernels specialised to one program at run time.
//
// The interpreter kernels (k_chunk.cu) decode every op of every stage from
// the program in shared memory for every chunk: a branch tree over the op's
// register positions and subtype, loads of its header and matrix, loops over
// phase terms.  For a program that is swept many times this work is the same
// each time, so the specialised kernel does it once, on the host.  Its source
// instantiates the same sweep templates (chunk_dev.cuh: chunk_sweep,
// diag_sweep) with:
// - the stage layouts and the ops as straight-line calls, register positions
//   compile-time, exact identity ops dropped;
// - phase segments generated from the program's CTA and thread tables (sums
//   without entries folded away, only the per-chunk sums needed read, a
//   product table over the register bits that carry a phase);
// - H-, RY- and RX-like one-qubit ops without their scalar (one packed f32x2
//   instruction per output amplitude), the sweep's product of scalars
//   applied once;
// - direct first and last stages where the program's layouts allow them.
// The source holds structure only.  Every number -- matrix entries, the
// scaled forms' ratios, phase weights of body terms, constant phase sums and
// factors (folded on the host in long double), the sweep's scale -- is a
// slot of the kernel's parameter block, a __grid_constant__ kernel argument
// (constant bank) filled per launch.  Programs that differ only in their
// numbers (a circuit with fresh angles) therefore share one compiled kernel.
// The arithmetic is the interpreter's up to the rounding order of those
// rewrites; the results agree to a few float ulps.
//
// Compilation uses NVRTC (loaded with dlopen, so the library loads without
// it) to a sm_103a cubin, loaded with cudaLibraryLoadData.  Kernels are
// cached by their source, at most jit_set_cache_limit() of them (least
// recently used first out; an evicted kernel's library is unloaded once no
// launch can still use it); a second map remembers each recent program's
// source and parameter values, so a repeated program costs no generation.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <chrono>
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <list>
#include <map>
#include <unordered_map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "program.h"

namespace svs {

// the device headers the generated source includes (jit_headers.cpp, written
// by the build from the csrc files)
extern const int kJitHeaderCount;
extern const char *const kJitHeaderNames[];
extern const char *const kJitHeaderSources[];

namespace {

struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    std::string err;
};

const Nvrtc &nvrtc()
{
    static Nvrtc n = [] {
        Nvrtc r;
        std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
        const char *homes[] = {getenv("CUDA_HOME"), "/usr/local/cuda"};
        for (const char *home : homes)
            if (home) names.push_back(std::string(home) + "/lib64/libnvrtc.so.13");
        void *h = nullptr;
        for (const std::string &nm : names)
            if ((h = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            r.err = "NVRTC (libnvrtc.so.13) not found: specialised sweep kernels need it";
            return r;
        }
        r.create = (decltype(r.create))dlsym(h, "nvrtcCreateProgram");
        r.compile = (decltype(r.compile))dlsym(h, "nvrtcCompileProgram");
        r.cubin_size = (decltype(r.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        r.cubin = (decltype(r.cubin))dlsym(h, "nvrtcGetCUBIN");
        r.log_size = (decltype(r.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        r.log = (decltype(r.log))dlsym(h, "nvrtcGetProgramLog");
        r.destroy = (decltype(r.destroy))dlsym(h, "nvrtcDestroyProgram");
        if (!r.create || !r.compile || !r.cubin_size || !r.cubin || !r.log_size || !r.log || !r.destroy)
            r.err = "NVRTC: missing entry points";
        return r;
    }();
    return n;
}

// Values of a generated kernel: the parameter block's words, in the order
// the generator reads them.  The source refers to slot k as P.w[k].
struct PBlock {
    std::vector<uint32_t> w;
    std::string u(uint32_t v)
    {
        w.push_back(v);
        return "P.w[" + std::to_string(w.size() - 1) + "]";
    }
    std::string f(float v)
    {
        uint32_t b;
        std::memcpy(&b, &v, 4);
        return "__uint_as_float(" + u(b) + ")";
    }
    std::string fbits(uint32_t bits) { return "__uint_as_float(" + u(bits) + ")"; }
    // a constant factor as the two packed operands (re, re), (-im, im) of the
    // f32x2 complex product, 8-byte aligned in the block
    std::string pk(float re, float im)
    {
        if (w.size() & 1) w.push_back(0);
        const size_t k = w.size();
        const float q[4] = {re, re, -im, im};
        for (float x : q) {
            uint32_t b;
            std::memcpy(&b, &x, 4);
            w.push_back(b);
        }
        return "*(const u64 *)&P.w[" + std::to_string(k) + "], *(const u64 *)&P.w[" + std::to_string(k + 2) + "]";
    }
};

constexpr const char *kKernelName = "svs_chunk_jit";
constexpr const char *kDiagKernelName = "svs_diag_jit";
// parameter-block words a launch may pass (kernel arguments are limited to
// 32764 bytes; the other arguments take 40)
constexpr size_t kMaxParamWords = 8000;

// ---- phase segments
// Where each sum of a segment comes from, read off the program's tables: a
// slot is "dynamic" when an entry depends on the chunk (a CTA entry with a
// mask), on the thread (a thread-table entry) or on the amplitude block (a
// term in the body); otherwise it is the constant sum of its always-met CTA
// entries (a parameter), and absent when it has none.
struct SlotSrc {
    bool cta_dyn = false;   // CTA entries with a mask: read the per-chunk sum
    int ncst = 0;           // always-met CTA entries
    uint32_t cst = 0;       // their sum
    bool thr = false;       // thread-table entries (hoisted segment)
};

// A complex factor while the code is generated: exactly one (no entries),
// a constant known on the host (folded in long double, passed as two
// parameter slots) or a run-time value in a variable.
struct Fac {
    enum Kind { ONE, CONST, VAR } kind = ONE;
    long double re = 1, im = 0;
    std::string var;
};

std::string fac_expr(PBlock &P, const Fac &f)
{
    if (f.kind == Fac::VAR) return f.var;
    const std::string re = P.f((float)f.re);
    return "make_float2(" + re + ", " + P.f((float)f.im) + ")";
}

Fac cis_const(const SlotSrc &ss)
{
    Fac f;
    if (ss.ncst == 0) return f;   // no entries: exactly one
    const long double th = 6.283185307179586476925286766559L * (long double)ss.cst * 0x1p-32L;
    f.kind = Fac::CONST;
    f.re = cosl(th);
    f.im = sinl(th);
    return f;
}

// a * b, emitting a run-time product into `o` (variable `name`) when needed
Fac fac_mul(std::ostringstream &o, PBlock &P, const Fac &a, const Fac &b, const std::string &name)
{
    if (a.kind == Fac::ONE) return b;
    if (b.kind == Fac::ONE) return a;
    Fac r;
    if (a.kind == Fac::CONST && b.kind == Fac::CONST) {
        r.kind = Fac::CONST;
        r.re = a.re * b.re - a.im * b.im;
        r.im = a.re * b.im + a.im * b.re;
        return r;
    }
    r.kind = Fac::VAR;
    r.var = name;
    const std::string ea = fac_expr(P, a);
    o << "                const float2 " << name << " = cmul(" << ea << ", " << fac_expr(P, b) << ");\n";
    return r;
}

// Straight-line code of one factored phase segment (no terms on several
// register bits and other bits) of a complex64 program: the sums it needs,
// one sin/cos per run-time factor, the product table over the register bits
// that carry a phase, and one complex product per amplitude whose factor is
// not exactly one (packed f32x2: cmul_f, or cmul_pk for a constant).  `scaled`: the sweep's product of scalars (`scale`)
// multiplies this segment's base factor.
void gen_segment(std::ostringstream &o, PBlock &P, const std::vector<uint32_t> &w, size_t body,
                 const std::vector<SlotSrc> &slots, int RB, int TB, int T, int SCP, bool scaled, long double scale)
{
    using namespace prog;
    const uint32_t *b = &w[body];
    const int d = (int)b[D_INDEX], nb = (int)b[D_NBASE];
    const int NR = 1 << RB, S = 1 + RB;
    const uint32_t tabmask = RB <= 5 ? b[D_TABMASK] : 0xffffffffu;
    o << "            {   // phase segment " << d << "\n";
    // which 128-bit words of the segment's CTA slots are read
    std::vector<char> need_q((size_t)SCP / 4, 0);
    auto slot_dyn = [&](int k) { return slots[(size_t)d * SCP + k].cta_dyn; };
    for (int k = 0; k < 1 + RB + TB; k++)
        if (slot_dyn(k)) need_q[k / 4] = 1;
    for (int q = 0; q < SCP / 4; q++)
        if (need_q[q])
            o << "                const uint4 cq" << q << " = ((const uint4 *)(cta_ph + " << d * SCP << "))[" << q
              << "];\n";
    const char *comp = "xyzw";
    auto cta_val = [&](int k) { return "cq" + std::to_string(k / 4) + "." + comp[k % 4]; };
    const uint32_t *t = b + D_TERMS;
    // sum of slot s (0 = base, 1 + j = register bit j): body terms follow
    // the interpreter's order (base terms, then each register bit's)
    auto emit_sum = [&](int s, int nterm, const std::string &name) -> bool {
        const SlotSrc &ss = slots[(size_t)d * SCP + s];
        const bool thr = s < S && ss.thr;
        if (!ss.cta_dyn && !thr && nterm == 0) return false;   // constant or absent: folded
        o << "                uint32_t " << name << " = "
          << (ss.cta_dyn ? cta_val(s) : ss.ncst ? P.u(ss.cst) : std::string("0u")) << ";\n";
        if (s == 0)
            for (int i = 0; i < TB; i++)
                if (slot_dyn(1 + RB + i))
                    o << "                if (tid & " << (1 << i) << ") " << name << " += " << cta_val(1 + RB + i) << ";\n";
        if (thr) o << "                " << name << " += thr_ph[" << (d * S + s) * T << " + tid];\n";
        for (int i = 0; i < nterm; i++, t += kTermWords) {
            const uint64_t m = (uint64_t)t[0] | ((uint64_t)t[1] << 32);
            o << "                if ((x0 & 0x" << std::hex << m << "ull) == 0x" << m << std::dec << "ull) " << name
              << " += " << P.u(t[2]) << ";\n";
        }
        return true;
    };
    Fac fb;
    // the base: CTA thread-bit coefficients make it run-time too
    {
        bool coef = false;
        for (int i = 0; i < TB; i++) coef = coef || slot_dyn(1 + RB + i);
        const SlotSrc &s0 = slots[(size_t)d * SCP];
        if (emit_sum(0, nb, "pb") || coef) {
            if (!(s0.cta_dyn || s0.thr || nb)) {
                // only thread-bit coefficients: start from the constant
                o << "                uint32_t pb = " << (s0.ncst ? P.u(s0.cst) : std::string("0u")) << ";\n";
                for (int i = 0; i < TB; i++)
                    if (slot_dyn(1 + RB + i))
                        o << "                if (tid & " << (1 << i) << ") pb += " << cta_val(1 + RB + i) << ";\n";
            }
            o << "                const float2 e0 = cis_turns(pb);\n";
            fb.kind = Fac::VAR;
            fb.var = "e0";
        } else {
            fb = cis_const(s0);
        }
    }
    std::vector<Fac> fl(RB);
    for (int j = 0; j < RB; j++) {
        const std::string nm = "pl" + std::to_string(j);
        if (emit_sum(1 + j, (int)b[D_NLIN + j], nm)) {
            o << "                const float2 e" << 1 + j << " = cis_turns(" << nm << ");\n";
            fl[j].kind = Fac::VAR;
            fl[j].var = "e" + std::to_string(1 + j);
        } else {
            fl[j] = cis_const(slots[(size_t)d * SCP + 1 + j]);
        }
    }
    // product table over the register bits with a phase: tb[idx], idx the
    // bits of m at those positions
    std::vector<int> K;
    for (int j = 0; j < RB; j++)
        if (fl[j].kind != Fac::ONE) K.push_back(j);
    if (scaled) {   // the sweep's deferred scale of its scaled one-qubit ops
        Fac sc;
        sc.kind = Fac::CONST;
        sc.re = scale;
        sc.im = 0;
        fb = fac_mul(o, P, fb, sc, "e0s");
    }
    std::vector<Fac> tb(1);
    tb[0] = fb;
    for (size_t k = 0; k < K.size(); k++) {
        const size_t h = tb.size();
        tb.resize(2 * h);
        for (size_t i = 0; i < h; i++)
            tb[h + i] = fac_mul(o, P, tb[i], fl[K[k]], "f" + std::to_string(h + i));
    }
    const float *ctab = (const float *)(t + 2 * NR);   // after the register-only phases
    for (int m = 0; m < NR; m++) {
        size_t idx = 0;
        for (size_t k = 0; k < K.size(); k++)
            if ((m >> K[k]) & 1) idx |= (size_t)1 << k;
        Fac f = tb[idx];
        if ((tabmask >> m) & 1) {
            Fac c;
            c.kind = Fac::CONST;
            c.re = ctab[2 * m];   // the program's float factor, as the interpreter multiplies
            c.im = ctab[2 * m + 1];
            if (f.kind == Fac::VAR) {
                // two packed products (the constant's, then the table entry's,
                // which other amplitudes share) instead of a scalar product of
                // the two factors that would then be packed for this one use
                o << "                v[" << m << "] = cmul_pk(v[" << m << "], " << P.pk((float)c.re, (float)c.im)
                  << ");\n";
                o << "                v[" << m << "] = cmul_f(v[" << m << "], " << f.var << ");\n";
                continue;
            }
            f = fac_mul(o, P, f, c, "g" + std::to_string(m));
        }
        // the amplitude's product in packed form (cmul_f, cmul_pk): a
        // constant factor comes as its two packed operands
        if (f.kind == Fac::CONST)
            o << "                v[" << m << "] = cmul_pk(v[" << m << "], " << P.pk((float)f.re, (float)f.im) << ");\n";
        else if (f.kind == Fac::VAR)
            o << "                v[" << m << "] = cmul_f(v[" << m << "], " << f.var << ");\n";
    }
    o << "            }\n";
}

// A one-qubit op as s * N with one packed instruction per output amplitude
// (dense1_pm / dense1_rot / dense1_rxn), or none of those forms.
struct Scaled {
    int form = 0;            // 0 none, 1 +-1 entries, 2 real [[1, t0], [t1, 1]], 3 [[1, i u0], [i u1, 1]]
    long double s = 1;       // the scalar
    float t0 = 0, t1 = 0;    // form 2, 3
    int r0 = 0, r1 = 0;      // form 1: rows (0 x0 + x1, 1 x0 - x1, 2 x1 - x0)
};

// The form follows the op's structure (its subtype and which entries are
// equal), not its angle: RX(t) and the real rotations of the Euler split
// keep form 3 / 2 for every t except the measure-zero set where the pivot
// is (nearly) zero, so circuits with fresh angles reuse their kernels.
Scaled scaled_form(const uint32_t *b, int sub)
{
    using namespace prog;
    auto f = [&](int i) {
        float x;
        std::memcpy(&x, &b[i], 4);
        return (long double)x;
    };
    Scaled r;
    const long double a = f(0), d = f(6);
    if (!(fabsl(a) >= 0x1p-24L)) return r;   // the pivot divides: keep it away from zero
    if (sub == DS_REAL) {
        const long double bb = f(2), cc = f(4);
        if (fabsl(bb) == fabsl(a) && fabsl(cc) == fabsl(a) && fabsl(d) == fabsl(a)) {
            // rows (1, b/a), (c/a, d/a) of +-1: x0 + x1, x0 - x1, x1 - x0
            const int sb = bb / a > 0 ? 1 : -1, sc = cc / a > 0 ? 1 : -1, sd = d / a > 0 ? 1 : -1;
            if (sc < 0 && sd < 0) return r;
            r.form = 1;
            r.s = a;
            r.r0 = sb > 0 ? 0 : 1;
            r.r1 = sc > 0 ? (sd > 0 ? 0 : 1) : 2;
            return r;
        }
        if (d == a) {
            r.form = 2;
            r.s = a;
            r.t0 = (float)(bb / a);
            r.t1 = (float)(cc / a);
        }
        return r;
    }
    if (sub == DS_RX && d == a) {
        r.form = 3;
        r.s = a;
        r.t0 = (float)(f(3) / a);
        r.t1 = (float)(f(5) / a);
    }
    return r;
}

// the phase slots of every segment of program w
std::vector<SlotSrc> read_slots(const std::vector<uint32_t> &w, int RB, int SCP)
{
    using namespace prog;
    const int S = 1 + RB;
    std::vector<SlotSrc> slots((size_t)w[H_NDSEG] * SCP);
    for (uint32_t i = 0; i < w[H_NCTA]; i++) {
        const uint32_t *e = &w[w[H_CTA_OFF] + (size_t)i * kCtaWords];
        SlotSrc &ss = slots[e[0]];
        if (e[2] | e[3]) {
            ss.cta_dyn = true;
        } else {
            ss.ncst++;
            ss.cst += e[4];
        }
    }
    for (uint32_t i = 0; i < w[H_NTHR]; i++) {
        const uint32_t *e = &w[w[H_THR_OFF] + (size_t)i * kThrWords];
        slots[(size_t)(e[0] / S) * SCP + e[0] % S].thr = true;
    }
    return slots;
}

const char *kParamStruct = "struct __align__(8) JP { uint32_t w[";

}  // namespace

bool jit_supported(bool f64, int C, int RB) { return !f64 && ((C == 12 && (RB == 4 || RB == 5)) || (C == 13 && RB == 5)); }
bool jit_supported_diag(bool f64, int RB) { return !f64 && RB == 4; }

// CUDA source of the fused diagonal sweep (K3) specialised to program `w`:
// its one phase segment as generated code, the sweep as in the interpreter.
static bool jit_source_diag(const std::vector<uint32_t> &w, std::string &src, std::vector<uint32_t> &vals,
                            std::string &err)
{
    using namespace prog;
    const int C = (int)w[H_C], RB = (int)w[H_RB];
    if (w[H_WBYTES] != 4 || !jit_supported_diag(false, RB) || C != 7 + RB || w[H_NSTAGE] != 1) {
        err = "specialised kernels: complex64 diagonal sweeps with RB = 4 only";
        return false;
    }
    const int TB = 7, SCP = (int)cta_stride(RB, TB, 4);
    const std::vector<SlotSrc> slots = read_slots(w, RB, SCP);
    const size_t body = w[H_STAGE_OFF] + S_SIZE + O_BODY;
    PBlock P;
    std::ostringstream g;
    if (w[body + D_NMULTI])
        g << "            dseg_apply<R, RB, T, 3>(v, x0, prog + " << body << ", cta_ph, thr_ph, nhoist, tid);\n";
    else
        gen_segment(g, P, w, body, slots, RB, TB, 128, SCP, false, 1.0L);
    if (P.w.empty()) P.w.push_back(0);
    if (P.w.size() & 1) P.w.push_back(0);   // the block is 8-byte aligned: whole 8-byte units
    std::ostringstream o;
    o << "#include \"chunk_dev.cuh\"\nnamespace svs {\n" << kParamStruct << P.w.size() << "]; };\n"
      << "struct JDiag {\n    using Params = JP;\n"
         "    template <typename R, int RB, int T>\n"
         "    static __device__ __forceinline__ void seg(typename CT<R>::T2 (&v)[1 << RB], uint64_t x0,\n"
         "        const uint32_t *prog, const uint32_t *, const typename CT<R>::W *cta_ph,\n"
         "        const typename CT<R>::W *thr_ph, int nhoist, int tid, const JP &P)\n    {\n"
      << g.str() << "    }\n};\n}  // namespace svs\n";
    o << "extern \"C\" __global__ void __launch_bounds__(128) " << kDiagKernelName
      << "(svs::CT<float>::G2 *__restrict__ a, const uint32_t *__restrict__ gprog, int n, "
         "svs::TSrc<svs::CT<float>::G2> src, const __grid_constant__ svs::JP P)\n{\n    svs::diag_sweep<float, "
      << RB << ", svs::JDiag>(a, gprog, n, src, P);\n}\n";
    src = o.str();
    vals.swap(P.w);
    return true;
}

// CUDA source of the kernel specialised to program `w` (complex64, C = 12,
// RB = 4 or 5) and the values of its parameter block.  Ops are walked as the
// interpreter walks them.
bool jit_source(const std::vector<uint32_t> &w, int kind, std::string &src, std::vector<uint32_t> &vals,
                std::string &err)
{
    using namespace prog;
    if (kind == JIT_DIAG) return jit_source_diag(w, src, vals, err);
    const int C = (int)w[H_C], RB = (int)w[H_RB], ns = (int)w[H_NSTAGE];
    if (w[H_WBYTES] != 4 || !jit_supported(false, C, RB)) {
        err = "specialised kernels: complex64 chunk programs with C = 12, RB = 4 or 5, or C = 13, RB = 5 only";
        return false;
    }
    const int T = 1 << (C - RB), NR = 1 << RB, TB = C - RB;
    const int SCP = (int)cta_stride(RB, TB, 4);
    // where every phase sum comes from (per segment and slot)
    const std::vector<SlotSrc> slots = read_slots(w, RB, SCP);
    PBlock P;
    std::ostringstream o;
    o << "    static constexpr int kStages = " << ns << ";\n";
    o << "    static constexpr bool kPrefetch = true;\n";
    // fed by a merge-booster product or not, fixed per kernel
    o << "    static constexpr int kFed = " << (kind == JIT_CHUNK_FED ? 1 : 0) << ";\n";
    // direct boundary stages: their register offsets in HBM
    const uint32_t direct = w[H_DIRECT];
    o << "    static constexpr bool kDirectFirst = " << ((direct & DIRECT_FIRST) ? "true" : "false")
      << ", kDirectLast = " << ((direct & DIRECT_LAST) ? "true" : "false") << ";\n";
    o << "    static __device__ __forceinline__ bool paired(int s)\n    {\n";
    for (int s = 0; s < ns; s++)
        o << "        if (s == " << s << ") return " << (w[w[H_STAGE_OFF + s] + S_REG] == 0 ? "true" : "false") << ";\n";
    o << "        return false;\n    }\n";
    o << "    static __device__ __forceinline__ uint64_t roff(int s, int m)\n    {\n";
    for (int s = 0; s < ns; s++) {
        if (!((s == 0 && (direct & DIRECT_FIRST)) || (s == ns - 1 && (direct & DIRECT_LAST)))) continue;
        const size_t so = w[H_STAGE_OFF + s];
        for (int m = 0; m < NR; m++) {
            uint64_t off = 0;
            for (int j = 0; j < RB; j++)
                if ((m >> j) & 1) off |= 1ull << w[H_QIN + w[so + S_REG + j]];
            o << "        if (s == " << s << " && m == " << m << ") return " << off << "ull;\n";
        }
    }
    o << "        return 0;\n    }\n";
    o << "    static __device__ __forceinline__ uint32_t stage_off(const uint32_t *, int s)\n    {\n";
    for (int s = 0; s < ns; s++) o << "        if (s == " << s << ") return " << w[H_STAGE_OFF + s] << "u;\n";
    o << "        return 0u;\n    }\n";
    o << "    template <int RB>\n    static __device__ __forceinline__ void stage_pv(const uint32_t *, int s, "
         "uint32_t (&pv)[(RB + 3) & ~3])\n    {\n";
    for (int s = 0; s < ns; s++) {
        const size_t so = w[H_STAGE_OFF + s];
        o << "        if (s == " << s << ") {";
        for (int j = 0; j < ((RB + 3) & ~3); j++) o << " pv[" << j << "] = " << (j < RB ? w[so + S_PV + j] : 0) << "u;";
        o << " }\n";
    }
    o << "    }\n";
    // one instantiation per stage (S compile-time): each holds its own ops only
    o << "    template <typename R, int RB, int T, int S>\n"
         "    static __device__ __forceinline__ void run_s(typename CT<R>::T2 (&v)[1 << RB], uint64_t x0,\n"
         "        const uint32_t *prog, const uint32_t *, const typename CT<R>::W *cta_ph,\n"
         "        const typename CT<R>::W *thr_ph, int nhoist, int tid, const JP &P)\n    {\n";
    // pass 1: the scaled forms of one-qubit ops (their form follows the op's
    // structure) and where their scalars are applied.  The product of the
    // scalars since the last factored phase segment is folded into the next
    // one (its base factor, free) or, after the last, multiplies the
    // amplitudes at the end of the last stage: each product is applied right
    // after the growth it undoes (no amplitude is scaled down before it has
    // grown).  A group's product is kept above 2^-60, so that magnitudes stay
    // below 2^60 times their own: an op whose scalar would push it lower
    // (angles within about 2^-30 of the rotation's zero, in practice never)
    // keeps its unscaled form.
    std::map<size_t, Scaled> scaled;
    std::map<size_t, long double> fold;   // factored segment body -> product folded into it
    long double grp = 1;
    bool grp_open = false;
    for (int s = 0; s < ns; s++) {
        size_t op = w[H_STAGE_OFF + s] + S_SIZE;
        for (uint32_t k = 0; k < w[w[H_STAGE_OFF + s] + S_NOPS]; k++) {
            const uint32_t hdr = w[op];
            const size_t body = op + O_BODY;
            if ((hdr & 0xff) == OP_DENSE && ((hdr >> 8) & 0xf) == 1) {
                const Scaled sf = scaled_form(&w[body], (hdr >> 12) & 0xf);
                if (sf.form && fabsl(grp * sf.s) >= 0x1p-60L) {
                    scaled[body] = sf;
                    grp *= sf.s;
                    grp_open = true;
                }
            } else if ((hdr & 0xff) == OP_DSEG && !w[body + D_NMULTI] && grp_open) {
                fold[body] = grp;
                grp = 1;
                grp_open = false;
            }
            op += w[op + O_WORDS];
        }
    }
    for (int s = 0; s < ns; s++) {
        const size_t so = w[H_STAGE_OFF + s];
        o << "        " << (s ? "else " : "") << "if constexpr (S == " << s << ") {\n";
        size_t op = so + S_SIZE;
        for (uint32_t k = 0; k < w[so + S_NOPS]; k++) {
            const uint32_t hdr = w[op], len = w[op + O_WORDS];
            const size_t body = op + O_BODY;
            if ((hdr & 0xff) == OP_DENSE) {
                const int kq = (hdr >> 8) & 0xf, sub = (hdr >> 12) & 0xf, code = (int)(hdr >> 16);
                const auto sc = scaled.find(body);
                if (kq == 1 && sub == DS_REAL && w[body] == 0x3f800000u && w[body + 2] == 0 && w[body + 4] == 0 &&
                    w[body + 6] == 0x3f800000u) {
                    // exactly the identity in complex64 (e.g. H H): nothing to do
                } else if (sc != scaled.end()) {
                    const Scaled &f = sc->second;
                    if (f.form == 1) {
                        o << "            dense1_pm<" << NR << ", " << code << ", " << f.r0 << ", " << f.r1 << ">(v);\n";
                    } else {
                        const std::string t0 = P.f(f.t0);
                        o << "            dense1_" << (f.form == 2 ? "rot<" : "rxn<") << NR << ", " << code << ">(v, "
                          << t0 << ", " << P.f(f.t1) << ");\n";
                    }
                } else if (kq == 1 && sub != DS_GENERAL) {
                    const bool re = sub == DS_REAL;
                    const std::string pa = P.fbits(w[body]), pb = P.fbits(w[body + (re ? 2 : 3)]);
                    const std::string pc = P.fbits(w[body + (re ? 4 : 5)]), pd = P.fbits(w[body + 6]);
                    o << "            dense1_special_f<" << NR << ", " << code << ", " << sub << ">(v, " << pa << ", "
                      << pb << ", " << pc << ", " << pd << ");\n";
                } else if (kq == 1) {
                    o << "            { const float m[8] = {";
                    for (int i = 0; i < 8; i++) o << (i ? ", " : "") << P.fbits(w[body + i]);
                    o << "}; dense1_general_f<" << NR << ", " << code << ">(v, m); }\n";
                } else {
                    o << "            { const float m[32] = {";
                    for (int i = 0; i < 32; i++) o << (i ? ", " : "") << P.fbits(w[body + i]);
                    o << "}; dense2_f<" << NR << ", " << (code & 7) << ", " << ((code >> 3) & 7) << ">(v, m); }\n";
                }
            } else if (w[body + D_NMULTI]) {
                // terms on several register bits and other bits: the general path
                o << "            dseg_apply<R, RB, T, 3>(v, x0, prog + " << body << ", cta_ph, thr_ph, nhoist, tid);\n";
            } else {
                const auto fd = fold.find(body);
                gen_segment(o, P, w, body, slots, RB, TB, T, SCP, fd != fold.end(), fd != fold.end() ? fd->second : 1.0L);
            }
            op += len;
        }
        if (s == ns - 1 && grp_open) o << "            scale_all<" << NR << ">(v, " << P.f((float)grp) << ");\n";
        o << "        }\n";
    }
    o << "    }\n};\n}  // namespace svs\n";
    // registers for two CTAs per SM (2^12-amplitude chunks: 128 threads of
    // 32 amplitudes or 256 of 16), or one of 256 threads (2^13 amplitudes)
    o << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << (C == 13 ? 1 : 2) << ") " << kKernelName
      << "(svs::CT<float>::G2 *__restrict__ a, const uint32_t *__restrict__ gprog, int n, "
         "svs::TSrc<svs::CT<float>::G2> src, const __grid_constant__ svs::JP P)\n{\n    svs::chunk_sweep<float, "
      << C << ", " << RB << ", svs::JOps>(a, gprog, n, src, P);\n}\n";
    if (P.w.empty()) P.w.push_back(0);
    std::ostringstream full;
    if (P.w.size() & 1) P.w.push_back(0);   // the block is 8-byte aligned: whole 8-byte units
    full << "#include \"chunk_dev.cuh\"\nnamespace svs {\n" << kParamStruct << P.w.size() << "]; };\n"
         << "struct JOps {\n    using Params = JP;\n" << o.str();
    src = full.str();
    vals.swap(P.w);
    return true;
}

// NVRTC: source -> sm_103a cubin
bool jit_compile(const std::string &src, std::vector<char> &cubin, std::string &err)
{
    const Nvrtc &nv = nvrtc();
    if (!nv.err.empty()) {
        err = nv.err;
        return false;
    }
    nvrtcProgram p = nullptr;
    if (nv.create(&p, src.c_str(), "svs_chunk_jit.cu", kJitHeaderCount, kJitHeaderSources, kJitHeaderNames) !=
        NVRTC_SUCCESS) {
        err = "NVRTC: create failed";
        return false;
    }
    // SVSIM_JIT_FAST_COMPILE = 0 | min | mid | max: NVRTC's --Ofast-compile
    // level (compile time against run time; the sweep's helpers stay inlined)
    static const std::string fast = [] {
        const char *e = getenv("SVSIM_JIT_FAST_COMPILE");
        const std::string v = e ? e : "0";
        return (v == "min" || v == "mid" || v == "max") ? "--Ofast-compile=" + v : std::string();
    }();
    const char *opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-lineinfo", fast.c_str()};
    const nvrtcResult r = nv.compile(p, fast.empty() ? 4 : 5, opts);
    bool ok = r == NVRTC_SUCCESS;
    if (!ok) {
        size_t ls = 0;
        nv.log_size(p, &ls);
        std::string log(ls, '\0');
        nv.log(p, log.data());
        err = "NVRTC: compile failed: " + log.substr(0, 2000);
    } else {
        size_t cs = 0;
        nv.cubin_size(p, &cs);
        cubin.resize(cs);
        nv.cubin(p, cubin.data());
    }
    nv.destroy(&p);
    return ok;
}

struct JitKernel {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    unsigned dev_mask = 0;    // devices it was launched on (dynamic shared-memory limit raised)
    size_t pwords = 0;        // parameter-block words
    int kind = JIT_CHUNK;
    uint64_t stamp = 0;       // last use (LRU)
};

namespace {

std::mutex g_mu;
// kernels by source (structure only), and recent programs by their words
std::unordered_map<std::string, std::shared_ptr<JitKernel>> g_kernels;
struct ProgEntry {
    std::string src;
    std::shared_ptr<const std::vector<uint32_t>> vals;
    uint64_t stamp = 0;
};
std::unordered_map<std::string, ProgEntry> g_progs;
std::vector<std::shared_ptr<JitKernel>> g_retired;   // evicted, unloaded when no launch can use them
size_t g_limit = 256;
uint64_t g_clock = 0;
uint64_t g_compiles = 0;
double g_compile_ms = 0;   // wall time of jit_prepare's compiles

std::string key_of(const std::vector<uint32_t> &w, int kind)
{
    return std::string(1, (char)('0' + kind)) + std::string((const char *)w.data(), w.size() * 4);
}

// Unload evicted kernels no host thread holds any more, after the devices
// they ran on have finished all work (a launch may still be queued).
void unload_retired_locked()
{
    bool any = false;
    for (const auto &k : g_retired) any = any || k.use_count() == 1;
    if (!any) return;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return;
    unsigned synced = 0;
    std::vector<std::shared_ptr<JitKernel>> keep;
    for (auto &k : g_retired) {
        if (k.use_count() != 1) {
            keep.push_back(k);
            continue;
        }
        bool ok = true;
        for (int d = 0; d < 32 && ok; d++)
            if (((k->dev_mask >> d) & 1) && !((synced >> d) & 1)) {
                ok = cudaSetDevice(d) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
                if (ok) synced |= 1u << d;
            }
        if (ok && k->lib) cudaLibraryUnload(k->lib);
        else if (!ok) keep.push_back(k);
    }
    cudaSetDevice(cur);
    g_retired.swap(keep);
}

void evict_locked()
{
    while (g_kernels.size() > g_limit) {
        auto lru = g_kernels.begin();
        for (auto it = g_kernels.begin(); it != g_kernels.end(); ++it)
            if (it->second->stamp < lru->second->stamp) lru = it;
        g_retired.push_back(lru->second);
        g_kernels.erase(lru);
    }
    while (g_progs.size() > 4 * g_limit) {
        auto lru = g_progs.begin();
        for (auto it = g_progs.begin(); it != g_progs.end(); ++it)
            if (it->second.stamp < lru->second.stamp) lru = it;
        g_progs.erase(lru);
    }
    unload_retired_locked();
}

// compile and load one kernel
bool build_one(const std::string &src, int kind, size_t pwords, std::shared_ptr<JitKernel> &out, std::string &err)
{
    std::vector<char> cubin;
    if (!jit_compile(src, cubin, err)) return false;
    auto k = std::make_shared<JitKernel>();
    k->pwords = pwords;
    k->kind = kind;
    cudaError_t e = cudaLibraryLoadData(&k->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&k->kern, k->lib, kind == JIT_DIAG ? kDiagKernelName : kKernelName);
    if (e != cudaSuccess) {
        err = std::string("loading a specialised kernel: ") + cudaGetErrorString(e);
        if (k->lib) cudaLibraryUnload(k->lib);
        return false;
    }
    out = k;
    return true;
}

}  // namespace

bool jit_prepare(const std::vector<JitProg> &progs, std::vector<JitHandle> &out, std::string &err)
{
    out.assign(progs.size(), JitHandle());
    // 1. each program's source and parameter values (remembered per program)
    std::vector<std::string> srcs(progs.size());
    for (size_t i = 0; i < progs.size(); i++) {
        const std::string wk = key_of(*progs[i].w, progs[i].kind);
        {
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_progs.find(wk);
            if (it != g_progs.end()) {
                it->second.stamp = ++g_clock;
                srcs[i] = it->second.src;
                out[i].vals = it->second.vals;
                continue;
            }
        }
        std::string src;
        auto vals = std::make_shared<std::vector<uint32_t>>();
        if (!jit_source(*progs[i].w, progs[i].kind, src, *vals, err)) return false;
        if (vals->size() > kMaxParamWords) {
            srcs[i].clear();   // too many numbers for the argument space: the interpreter runs it
            continue;
        }
        srcs[i] = src;
        out[i].vals = vals;
        std::lock_guard<std::mutex> lk(g_mu);
        ProgEntry &pe = g_progs[wk];
        pe.src = src;
        pe.vals = vals;
        pe.stamp = ++g_clock;
    }
    // 2. kernels: cached ones by source; compile the missing ones in parallel
    std::vector<size_t> todo;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (size_t i = 0; i < progs.size(); i++) {
            if (srcs[i].empty()) continue;
            auto it = g_kernels.find(srcs[i]);
            if (it != g_kernels.end()) {
                it->second->stamp = ++g_clock;
                out[i].k = it->second;
                continue;
            }
            bool dup = false;
            for (size_t j : todo) dup = dup || srcs[j] == srcs[i];
            if (!dup) todo.push_back(i);
        }
    }
    if (!todo.empty()) {
        const auto t0 = std::chrono::steady_clock::now();
        const size_t nt = std::min<size_t>(todo.size(), std::max(1u, std::min(8u, std::thread::hardware_concurrency())));
        std::vector<std::string> errs(todo.size());
        std::vector<std::shared_ptr<JitKernel>> built(todo.size());
        std::vector<std::thread> th;
        for (size_t t = 0; t < nt; t++)
            th.emplace_back([&, t] {
                for (size_t x = t; x < todo.size(); x += nt) {
                    const size_t i = todo[x];
                    build_one(srcs[i], progs[i].kind, out[i].vals->size(), built[x], errs[x]);
                }
            });
        for (auto &x : th) x.join();
        std::lock_guard<std::mutex> lk(g_mu);
        g_compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        for (size_t x = 0; x < todo.size(); x++) {
            if (!built[x]) {
                err = errs[x];
                return false;
            }
            g_compiles++;
            built[x]->stamp = ++g_clock;
            // a concurrent build of the same source keeps the first
            g_kernels.emplace(srcs[todo[x]], built[x]);
        }
        for (size_t i = 0; i < progs.size(); i++)
            if (!srcs[i].empty() && !out[i].k) {
                auto it = g_kernels.find(srcs[i]);
                if (it != g_kernels.end()) out[i].k = it->second;
            }
        evict_locked();
    }
    for (size_t i = 0; i < progs.size(); i++)
        if (!srcs[i].empty() && !out[i].k) {
            err = "specialised kernel missing after its build";
            return false;
        }
    return true;
}

size_t jit_cache_size(double *compile_ms, uint64_t *compiles)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (compile_ms) *compile_ms = g_compile_ms;
    if (compiles) *compiles = g_compiles;
    return g_kernels.size();
}

void jit_set_cache_limit(size_t max_kernels)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_limit = std::max<size_t>(1, max_kernels);
    evict_locked();
}

static cudaError_t launch_jit(const JitHandle &h, void *a, int n, const uint32_t *prog, size_t smem, TensorSrc src,
                              cudaStream_t st, int threads, int C)
{
    if (!h.k || !h.vals || h.vals->size() != h.k->pwords) return cudaErrorInvalidDeviceFunction;   // jit_prepare first
    JitKernel &k = *h.k;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!((k.dev_mask >> dev) & 1)) {
            e = cudaKernelSetAttributeForDevice(k.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024, dev);
            if (e != cudaSuccess) return e;
            k.dev_mask |= 1u << dev;
        }
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)k.kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    const int64_t work = (int64_t)1 << (n - C);
    const int64_t g = (int64_t)device_sm_count() * occ;
    const int grid = (int)(g < work ? g : work);
    struct {
        const void *hi, *lo;
        int n_lo;
    } ts{src.hi, src.lo, src.n_lo};
    void *args[] = {&a, (void *)&prog, &n, &ts, (void *)h.vals->data()};
    e = cudaLaunchKernel((const void *)k.kern, dim3(grid), dim3(threads), args, smem, st);
    return counted(e, 1);
}

// The specialised chunk sweep: persistent grid = resident CTAs x SMs.
cudaError_t launch_chunk_jit(const JitHandle &h, void *a, int n, const std::vector<uint32_t> &w, const uint32_t *prog,
                             size_t smem, TensorSrc src, cudaStream_t st)
{
    const int C = (int)w[prog::H_C], RB = (int)w[prog::H_RB];
    // a kernel built for a fed sweep reads only the product's factors, one
    // built for a plain sweep only the state
    if (h.k && (h.k->kind == JIT_CHUNK_FED) != (src.hi != nullptr)) return cudaErrorInvalidValue;
    if (src.hi && (src.n_lo < 0 || src.n_lo > n || !src.lo)) return cudaErrorInvalidValue;
    return launch_jit(h, a, n, prog, smem, src, st, 1 << (C - RB), C);
}

// The specialised fused diagonal sweep: tiles of 2^(7 + RB) amplitudes, 128
// threads, grid = resident CTAs x SMs (as launch_diag_sweep).
cudaError_t launch_diag_jit(const JitHandle &h, void *a, int n, const std::vector<uint32_t> &w, const uint32_t *prog,
                            size_t smem, TensorSrc src, cudaStream_t st)
{
    if (src.hi && (src.n_lo < 0 || src.n_lo > n || !src.lo)) return cudaErrorInvalidValue;
    return launch_jit(h, a, n, prog, smem, src, st, 128, (int)w[prog::H_C]);
}

}  // namespace svs
