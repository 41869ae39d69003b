// jit.cpp -- chunk-sweep kernels specialised to one program at run time.
//
// The interpreter kernel (k_chunk.cu) decodes every op of every stage from
// the program in shared memory for every chunk: a branch tree over the op's
// register positions and subtype, and loads of its header and matrix.  For a
// program that is swept many times this work is the same each time, so the
// specialised kernel does it once, on the host: its source lists the stage
// layouts and the ops as straight-line calls of the same device templates
// (chunk_dev.cuh), with compile-time register positions and the 2x2 matrices
// of one-qubit ops as literals.  The phase tables, term lists and per-chunk
// sums stay in the staged program, exactly as the interpreter reads them, so
// both kernels compute the same arithmetic in the same order: their results
// are bit-identical.
//
// Compilation uses NVRTC (loaded with dlopen, so the library loads without
// it) to a sm_103a cubin, loaded with cudaLibraryLoadData; kernels are cached
// per program (its words) for the life of the process.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <chrono>
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <map>
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

// exact float literal
std::string flit(uint32_t bits)
{
    float f;
    std::memcpy(&f, &bits, 4);
    char b[48];
    std::snprintf(b, sizeof b, "%af", (double)f);
    return b;
}

constexpr const char *kKernelName = "svs_chunk_jit";

}  // namespace

bool jit_supported(bool f64, int C, int RB) { return !f64 && C == 12 && RB == 4; }

// CUDA source of the kernel specialised to program `w` (complex64, C = 12,
// RB = 4).  Ops are walked as the interpreter walks them.
bool jit_source(const std::vector<uint32_t> &w, std::string &src, std::string &err)
{
    using namespace prog;
    const int C = (int)w[H_C], RB = (int)w[H_RB], ns = (int)w[H_NSTAGE];
    if (w[H_WBYTES] != 4 || !jit_supported(false, C, RB)) {
        err = "specialised kernels: complex64 chunk programs with C = 12, RB = 4 only";
        return false;
    }
    const int T = 1 << (C - RB), NR = 1 << RB;
    std::ostringstream o;
    o << "#include \"chunk_dev.cuh\"\nnamespace svs {\nstruct JOps {\n";
    o << "    static constexpr int kStages = " << ns << ";\n";
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
    o << "    template <typename R, int RB, int T>\n"
         "    static __device__ __forceinline__ void run(int s, typename CT<R>::T2 (&v)[1 << RB], uint64_t x0,\n"
         "        const uint32_t *prog, const uint32_t *, const typename CT<R>::W *cta_ph,\n"
         "        const typename CT<R>::W *thr_ph, int nhoist, int tid)\n    {\n";
    for (int s = 0; s < ns; s++) {
        const size_t so = w[H_STAGE_OFF + s];
        o << "        if (s == " << s << ") {\n";
        size_t op = so + S_SIZE;
        for (uint32_t k = 0; k < w[so + S_NOPS]; k++) {
            const uint32_t hdr = w[op], len = w[op + O_WORDS];
            const size_t body = op + O_BODY;
            if ((hdr & 0xff) == OP_DENSE) {
                const int kq = (hdr >> 8) & 0xf, sub = (hdr >> 12) & 0xf, code = (int)(hdr >> 16);
                if (kq == 1 && sub != DS_GENERAL) {
                    const bool re = sub == DS_REAL;
                    o << "            dense1_special_f<" << NR << ", " << code << ", " << sub << ">(v, " << flit(w[body])
                      << ", " << flit(w[body + (re ? 2 : 3)]) << ", " << flit(w[body + (re ? 4 : 5)]) << ", "
                      << flit(w[body + 6]) << ");\n";
                } else if (kq == 1) {
                    o << "            { const float m[8] = {";
                    for (int i = 0; i < 8; i++) o << (i ? ", " : "") << flit(w[body + i]);
                    o << "}; dense1_general_f<" << NR << ", " << code << ">(v, m); }\n";
                } else {
                    o << "            dense_apply<R, " << NR << ", 2, " << (code & 7) << ", " << ((code >> 3) & 7)
                      << ">(v, prog + " << body << ");\n";
                }
            } else {
                // the segment's path: factored (without / with the register
                // table) or with terms on several register bits
                const uint32_t *b = &w[body];
                const int mode = b[D_NMULTI] ? 3 : (b[D_FLAGS] & 1) ? 2 : 1;
                o << "            dseg_apply<R, RB, T, " << mode << ">(v, x0, prog + " << body
                  << ", cta_ph, thr_ph, nhoist, tid);\n";
            }
            op += len;
        }
        o << "        }\n";
    }
    o << "    }\n};\n}  // namespace svs\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << T << ", 3) " << kKernelName
      << "(svs::CT<float>::G2 *__restrict__ a, const uint32_t *__restrict__ gprog, int n, "
         "svs::TSrc<svs::CT<float>::G2> src)\n{\n    svs::chunk_sweep<float, "
      << C << ", " << RB << ", svs::JOps>(a, gprog, n, src);\n}\n";
    src = o.str();
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
    const char *opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-lineinfo"};
    const nvrtcResult r = nv.compile(p, 4, opts);
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

namespace {

struct JitKernel {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    unsigned dev_mask = 0;    // devices whose dynamic shared-memory limit is raised
};

std::mutex g_mu;
std::map<std::string, std::shared_ptr<JitKernel>> g_cache;
double g_compile_ms = 0;   // wall time of jit_prepare's compiles

std::string key_of(const std::vector<uint32_t> &w) { return std::string((const char *)w.data(), w.size() * 4); }

std::shared_ptr<JitKernel> lookup(const std::string &key)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    return it == g_cache.end() ? nullptr : it->second;
}

// compile and load one program's kernel into the cache
bool build_one(const std::vector<uint32_t> &w, std::string &err)
{
    const std::string key = key_of(w);
    if (lookup(key)) return true;
    std::string src;
    std::vector<char> cubin;
    if (!jit_source(w, src, err) || !jit_compile(src, cubin, err)) return false;
    auto k = std::make_shared<JitKernel>();
    cudaError_t e = cudaLibraryLoadData(&k->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&k->kern, k->lib, kKernelName);
    if (e != cudaSuccess) {
        err = std::string("loading a specialised kernel: ") + cudaGetErrorString(e);
        return false;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache.emplace(key, k);   // a concurrent build of the same program keeps the first
    return true;
}

}  // namespace

bool jit_prepare(const std::vector<const std::vector<uint32_t> *> &progs, std::string &err)
{
    std::vector<const std::vector<uint32_t> *> todo;
    for (const auto *w : progs)
        if (!lookup(key_of(*w))) {
            bool dup = false;
            for (const auto *x : todo) dup = dup || *x == *w;
            if (!dup) todo.push_back(w);
        }
    if (todo.empty()) return true;
    const auto t0 = std::chrono::steady_clock::now();
    // compile in parallel (NVRTC programs are independent)
    const size_t nt = std::min<size_t>(todo.size(), std::max(1u, std::min(8u, std::thread::hardware_concurrency())));
    std::vector<std::string> errs(todo.size());
    std::vector<std::thread> th;
    for (size_t t = 0; t < nt; t++)
        th.emplace_back([&, t] {
            for (size_t i = t; i < todo.size(); i += nt) build_one(*todo[i], errs[i]);
        });
    for (auto &x : th) x.join();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    for (const std::string &e : errs)
        if (!e.empty()) {
            err = e;
            return false;
        }
    return true;
}

size_t jit_cache_size(double *compile_ms)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (compile_ms) *compile_ms = g_compile_ms;
    return g_cache.size();
}

cudaError_t launch_chunk_jit(void *a, int n, const std::vector<uint32_t> &w, const uint32_t *prog, size_t smem,
                             TensorSrc src, cudaStream_t st)
{
    std::shared_ptr<JitKernel> k = lookup(key_of(w));
    if (!k) return cudaErrorInvalidDeviceFunction;   // jit_prepare first
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!((k->dev_mask >> dev) & 1)) {
            e = cudaKernelSetAttributeForDevice(k->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024, dev);
            if (e != cudaSuccess) return e;
            k->dev_mask |= 1u << dev;
        }
    }
    const int C = (int)w[prog::H_C], RB = (int)w[prog::H_RB];
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)k->kern, 1 << (C - RB), smem);
    if (e != cudaSuccess) return e;
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    const int64_t work = (int64_t)1 << (n - C);
    const int64_t g = (int64_t)device_sm_count() * occ;
    const int grid = (int)(g < work ? g : work);
    struct {
        const void *hi, *lo;
        int n_lo;
    } ts{src.hi, src.lo, src.n_lo};
    void *args[] = {&a, (void *)&prog, &n, &ts};
    e = cudaLaunchKernel((const void *)k->kern, dim3(grid), dim3(1 << (C - RB)), args, smem, st);
    return counted(e, 1);
}

}  // namespace svs
