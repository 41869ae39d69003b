// fault.cpp -- host-side fault injection for tests (no counterpart in the
// paper).  The library's device allocations (dev_malloc) and the executor's
// kernel launches ask here first; a test lets the next `skip` operations of
// a kind through and arms the `count` after them to fail as if the device
// had refused them: the allocation returns
// cudaErrorMemoryAllocation without calling cudaMalloc, the launch is not
// made and reports cudaErrorLaunchOutOfResources.  The failure is made on
// the host before the CUDA call, so no GPU state is touched; the error paths
// above it (SIM_ENOMEM / SIM_ECUDA to the caller, handles and servers that
// stay usable) are what the tests check.
//
// Armed by sim_fault_inject() or, at load, by the environment variable
// SVSIM_FAULT = "alloc:N" or "launch:N".
#include <mutex>
#include <cstdlib>
#include <cstring>

#include <cuda_runtime.h>

#include "internal.h"
#include "svsim.h"

namespace svs {
namespace {

// per kind: operations to let through, then operations to fail
struct Arm {
    int skip = 0, fail = 0;
};
std::mutex g_mu;
Arm g_alloc, g_launch;

bool take(Arm &a)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (a.skip > 0) {
        a.skip--;
        return false;
    }
    if (a.fail > 0) {
        a.fail--;
        return true;
    }
    return false;
}

struct FromEnv {
    FromEnv()
    {
        const char *e = std::getenv("SVSIM_FAULT");
        if (!e) return;
        const char *colon = std::strchr(e, ':');
        const int n = colon ? std::atoi(colon + 1) : 1;
        if (!std::strncmp(e, "alloc", 5)) g_alloc.fail = n;
        else if (!std::strncmp(e, "launch", 6)) g_launch.fail = n;
    }
} g_from_env;

}  // namespace

bool fault_alloc_fails() { return take(g_alloc); }
bool fault_launch_fails() { return take(g_launch); }

cudaError_t dev_malloc(void **p, size_t bytes)
{
    if (fault_alloc_fails()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

}  // namespace svs

extern "C" int sim_fault_inject(int kind, int skip, int count)
{
    if (skip < 0 || count < 0) return SIM_EINVAL;
    svs::Arm *a = kind == SIM_FAULT_ALLOC ? &svs::g_alloc : kind == SIM_FAULT_LAUNCH ? &svs::g_launch : nullptr;
    if (!a) return SIM_EINVAL;
    std::lock_guard<std::mutex> lk(svs::g_mu);
    a->skip = skip;
    a->fail = count;
    return SIM_OK;
}
