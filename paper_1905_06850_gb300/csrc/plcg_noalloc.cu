// plcg_noalloc.cu -- plcg_solve_stencil_noalloc: a stencil solve that
// allocates nothing.
//
// Some callers cannot allocate device memory when they solve: code running
// under a strict memory budget or a pre-reserved pool, real-time loops that
// must not enter the allocator, or plugins that are handed a stream but no
// allocator.  This entry point runs the solve exactly as plcg_solve would
// (the same argument checks, shifts, kernel, launch shape and kernel
// arguments: solve_stencil_fixed in plcg_api.cu builds them with the code
// plcg_solve uses), but the solver's scratch (basis rings, search direction,
// residual, reduction partials, barrier counter, result record) lives in one
// file-scope __device__ array of kScratchBytes.  Every GPU that loads the
// library holds that array until the process exits.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it.  Make that first call before any stream
// capture.  All calls share the one array, and it keeps the last call's
// contents (each call clears the barrier counter and the result record, the
// only parts that must start at zero); calls whose kernels overlap on the GPU
// race with each other.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/plcg.h"
#include "plcg_internal.h"
#include "plcg_kernels.h"

using namespace plcg;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

plcg_status nafail(plcg_status st, const std::string &msg)
{
    set_last_error(msg);   // reported by plcg_last_error()
    return st;
}

}  // namespace

extern "C" plcg_status plcg_solve_stencil_noalloc(const plcg_stencil_desc *d, const double *b,
                                                  double *x, const plcg_params *prm,
                                                  plcg_result *res, void *stream)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nafail(PLCG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nafail(PLCG_ERR_INVALID, "device ordinal too large");
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            // once per device, with that device current: the array's device address
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess)
                return nafail(PLCG_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") +
                                                 cudaGetErrorString(e));
            g_scratch_ptr[dev] = p;
        }
        base = static_cast<char *>(g_scratch_ptr[dev]);
    }
    return solve_stencil_fixed(d, b, x, prm, res, stream, base, kScratchBytes, "plcg_solve_stencil_noalloc");
}
