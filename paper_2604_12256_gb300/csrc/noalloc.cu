// noalloc.cu -- an expectation-value entry point that allocates nothing.
//
// sim_expectation() keeps its reduction partials in memory the handle
// allocated with cudaMalloc.  Some callers cannot allocate device memory at
// the point where they need the read-out: code running inside an allocator
// callback or a memory-pool hook, embedded callers whose device memory is
// owned and budgeted by a host framework, and applications that forbid
// allocation after start-up (fixed memory plans).  For them,
// sim_expectation_noalloc() runs the same FP64 reduction kernels with the
// partials in a fixed, file-scope device array instead.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "kernels.h"
#include "svsim.h"

namespace {

// kReduceBlocks partials for each of up to 16 Z strings (the kernels' fixed grid)
constexpr int kMaxTermsPerCall = 16;
constexpr int kScratchDoubles = svs::kReduceBlocks * kMaxTermsPerCall;   // 128 KiB

// One copy per device that loads the library, kept until the process exits.
// Every call on a device shares it; the kernels overwrite every partial they
// read, so nothing needs clearing between calls.
static __device__ __align__(256) double g_expect_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

thread_local char g_msg[256];

int fail(int code, const char *msg, cudaError_t e = cudaSuccess)
{
    if (e != cudaSuccess)
        snprintf(g_msg, sizeof g_msg, "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(g_msg, sizeof g_msg, "%s", msg);
    return code;
}

}  // namespace

extern "C" {

const char *sim_noalloc_error(void) { return g_msg; }

int sim_expectation_noalloc(const void *dev_state, int n_qubits, sim_dtype dtype, const uint64_t *dev_masks,
                            size_t n_terms, double *dev_out, void *cuda_stream)
{
    if (!dev_state || !dev_masks || !dev_out) return fail(SIM_EINVAL, "null pointer argument");
    if (dtype != SIM_C64 && dtype != SIM_C128) return fail(SIM_EINVAL, "dtype must be SIM_C64 or SIM_C128");
    const int nmax = dtype == SIM_C64 ? 34 : 33;
    if (n_qubits < 1 || n_qubits > nmax) return fail(SIM_EUNSUPPORTED, "n_qubits outside 1..34 (c64) / 1..33 (c128)");
    if (n_terms < 1 || n_terms > (size_t)kMaxTermsPerCall)
        return fail(SIM_EINVAL, "n_terms must be 1..16 (the fixed scratch holds 16 terms)");
    if (svs::reduce_partials() * (int)n_terms > kScratchDoubles) return fail(SIM_EUNSUPPORTED, "scratch too small");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SIM_ECUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return fail(SIM_EUNSUPPORTED, "device index above 63");
    double *scratch = nullptr;
    {
        // set-up, once per device, with that device current: the host-side
        // name of the array is not a device address, so ask for the address
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_expect_scratch);
            if (e != cudaSuccess) return fail(SIM_ECUDA, "cudaGetSymbolAddress", e);
            g_scratch_ptr[dev] = (double *)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    e = svs::launch_expect_z(dev_state, n_qubits, dtype == SIM_C128, dev_masks, (int)n_terms, scratch, dev_out,
                             (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(SIM_ECUDA, "expectation kernels", e);
    return SIM_OK;
}

}  // extern "C"
