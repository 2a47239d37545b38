// plcg_noalloc.cu -- plcg_solve_stencil_noalloc: a stencil solve that
// allocates nothing.
//
// Some callers cannot allocate device memory when they solve: code running
// under a strict memory budget or a pre-reserved pool, real-time loops that
// must not enter the allocator, or plugins that are handed a stream but no
// allocator.  This entry point runs the same persistent solver kernels as
// plcg_solve, but their scratch (basis rings, search direction, residual,
// reduction partials, barrier counter, result record) lives in one
// file-scope __device__ array of kScratchBytes.  Every GPU that loads the
// library holds that array until the process exits.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it.  Make that first call before any stream
// capture.  All calls share the one array, and it keeps the last call's
// contents; calls whose kernels overlap on the GPU race with each other.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
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

plcg_status nacuda(cudaError_t e, const char *what)
{
    return nafail(e == cudaErrorMemoryAllocation ? PLCG_ERR_NOMEM : PLCG_ERR_CUDA,
                  std::string(what) + ": " + cudaGetErrorString(e));
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

template <typename T>
plcg_status run(const StencilDesc &st, int64_t n, const double *b, double *x,
                const plcg_params *prm, const double *sigma, cudaStream_t stream,
                char *base, plcg_result *res)
{
    const int l = prm->l;
    const bool cg = prm->method == PLCG_METHOD_CG;
    const bool f32 = sizeof(T) == 4;
    const int want = 16 / (int)sizeof(T);
    const int vec = (st.nx % want == 0) ? want : 1;
    const void *func = kernel_ptr(f32, kOpStencil, vec, cg ? 0 : l, cg);
    if (!func) return nafail(PLCG_ERR_UNIMPL, "no kernel for this configuration");
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, kBlock, 0);
    if (e != cudaSuccess) return nacuda(e, "device query");
    if (per_sm < 1) return nafail(PLCG_ERR_CUDA, "solver kernel cannot be resident");
    const int64_t unit = (int64_t)kBlock * vec;
    int64_t P = (int64_t)per_sm * sms;
    if (prm->grid_ctas > 0) P = std::min<int64_t>(P, prm->grid_ctas);
    P = std::max<int64_t>(1, std::min<int64_t>(P, (n + unit - 1) / unit));

    SolveArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    int nvec = 0;
    if (!cg) {
        for (int k = 0; k <= l; ++k) {
            int d = 3;
            if (k == l) d = std::max(3, l);
            if (k == 0 && prm->dots_2l1) d = std::max(3, l + 1);
            a.depth[k] = d;
            a.ddiv[k] = make_fastdiv((uint32_t)d);
            a.base[k] = nvec;
            nvec += d;
        }
    } else {
        nvec = 3;
    }
    const size_t vbytes = up256((size_t)n * sizeof(T));
    size_t off = 0;
    const size_t o_ring = off; off += vbytes * nvec;
    const size_t o_p = off; off += vbytes;
    const size_t o_rc = off; off += vbytes;
    const size_t o_r = off; off += up256((size_t)n * sizeof(double));
    const int slots = cg ? 2 : (l + 1);
    const size_t o_part = off; off += up256((size_t)slots * P * kMaxDots * sizeof(double));
    const size_t o_npart = off; off += up256((size_t)P * kNormSlots * sizeof(double));
    const size_t o_bar = off; off += 256;
    const size_t o_out = off; off += up256(sizeof(DevResult));
    if (off > kScratchBytes)
        return nafail(PLCG_ERR_INVALID,
                      "plcg_solve_stencil_noalloc: this solve needs " + std::to_string(off) +
                      " bytes of scratch; the fixed no-allocation scratch holds " +
                      std::to_string(kScratchBytes) + " bytes (use plcg_solve)");
    a.n = n;
    a.st = st;
    a.vstride = (int64_t)(vbytes / sizeof(T));
    a.b = b;
    a.x = x;
    a.r = reinterpret_cast<double *>(base + o_r);
    a.zring = reinterpret_cast<T *>(base + o_ring);
    a.p = reinterpret_cast<T *>(base + o_p);
    a.rc = reinterpret_cast<T *>(base + o_rc);
    a.part = reinterpret_cast<double *>(base + o_part);
    a.npart = reinterpret_cast<double *>(base + o_npart);
    a.bar = reinterpret_cast<unsigned *>(base + o_bar);
    a.out = reinterpret_cast<DevResult *>(base + o_out);
    a.method = cg ? 1 : 0;
    a.l = l;
    for (int k = 0; k < l && k < kMaxL; ++k) a.sigma[k] = sigma[k];
    a.rtol = prm->rtol;
    a.maxit = prm->maxit;
    a.dots_2l1 = prm->dots_2l1 ? 1 : 0;
    a.max_restarts = prm->max_restarts;
    a.inner_floor = prm->inner_rtol_floor;
    a.fp32 = f32 ? 1 : 0;
    a.poll_limit = 30000000ull;
    a.force_timeout = 0;

    // the barrier counter and the result record must start at zero
    e = cudaMemsetAsync(base + o_bar, 0, 256, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_out, 0, sizeof(DevResult), stream);
    if (e != cudaSuccess) return nacuda(e, "clearing the scratch");
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(func, dim3((unsigned)P), dim3(kBlock), args, 0, stream);
    if (e != cudaSuccess) return nacuda(e, "launch");
    DevResult o;
    e = cudaMemcpyAsync(&o, a.out, sizeof(DevResult), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return nacuda(e, "reading the result");
    if (res) {
        res->status = o.status;
        res->iters = o.iters;
        res->spmvs = o.spmvs;
        res->restarts = o.restarts;
        res->refinements = o.refinements;
        res->recursive_relres = o.recursive_relres;
        res->true_relres = o.true_relres;
        res->seconds = 0.0;   // this entry point records no CUDA events
        res->latency = 0.0;
    }
    if (o.status != PLCG_OK) return nafail((plcg_status)o.status, "solve ended with a non-OK status");
    return PLCG_OK;
}

}  // namespace

extern "C" plcg_status plcg_solve_stencil_noalloc(const plcg_stencil_desc *d, const double *b,
                                                  double *x, const plcg_params *prm,
                                                  plcg_result *res, void *stream)
{
    if (!d || !b || !x || !prm) return nafail(PLCG_ERR_INVALID, "NULL argument");
    if (!((d->dim == 2 && d->points == 5) || (d->dim == 3 && d->points == 7)))
        return nafail(PLCG_ERR_INVALID, "stencil: need dim 2 with 5 points or dim 3 with 7 points");
    const int64_t nz = (d->dim == 3) ? d->nz : 1;
    if (d->nx < 1 || d->ny < 1 || nz < 1 || d->nx >= (1 << 30) || d->ny >= (1 << 30) || nz >= (1 << 30))
        return nafail(PLCG_ERR_INVALID, "stencil: bad grid sizes");
    const int64_t n = d->nx * d->ny * nz;
    if (n >= (int64_t(1) << 31)) return nafail(PLCG_ERR_INVALID, "stencil: n must be < 2^31");
    if (!std::isfinite(d->center) || !std::isfinite(d->off) || !std::isfinite(d->diag_shift))
        return nafail(PLCG_ERR_INVALID, "stencil: non-finite coefficient");
    if (prm->method != PLCG_METHOD_PLCG && prm->method != PLCG_METHOD_CG)
        return nafail(PLCG_ERR_INVALID, "unknown method");
    if (prm->method == PLCG_METHOD_PLCG && (prm->l < 1 || prm->l > kMaxL))
        return nafail(PLCG_ERR_INVALID, "l must be in 1..8");
    if (!(prm->rtol > 0.0) || !std::isfinite(prm->rtol) || prm->maxit < 0 ||
        prm->maxit > (int64_t(1) << 30) || prm->max_restarts < 0)
        return nafail(PLCG_ERR_INVALID, "bad rtol, maxit or max_restarts");
    if (prm->prec != PLCG_FP64 && prm->prec != PLCG_FP32_FP64DOT)
        return nafail(PLCG_ERR_INVALID, "unknown precision");
    if (prm->prec == PLCG_FP32_FP64DOT && !(prm->inner_rtol_floor > 0.0 && prm->inner_rtol_floor < 1.0))
        return nafail(PLCG_ERR_INVALID, "inner_rtol_floor must be in (0, 1)");
    if (prm->precond != PLCG_PRECOND_NONE && prm->precond != PLCG_PRECOND_JACOBI)
        return nafail(PLCG_ERR_INVALID, "unknown preconditioner");
    if (prm->precond == PLCG_PRECOND_JACOBI && !(d->center + d->diag_shift > 0.0))
        return nafail(PLCG_ERR_INVALID, "Jacobi preconditioner: the stencil center is not positive");
    if ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15)
        return nafail(PLCG_ERR_INVALID, "b and x must be 16-byte aligned");
    double sigma[kMaxL] = {0};
    if (prm->method == PLCG_METHOD_PLCG) {
        if (prm->shifts) {
            for (int k = 0; k < prm->l; ++k) {
                if (!std::isfinite(prm->shifts[k])) return nafail(PLCG_ERR_INVALID, "non-finite shift");
                sigma[k] = prm->shifts[k];
            }
        } else {
            if (!(prm->lmax >= prm->lmin) || !std::isfinite(prm->lmin) || !std::isfinite(prm->lmax))
                return nafail(PLCG_ERR_INVALID, "need lmin <= lmax for the Chebyshev shifts");
            const double pi = 3.14159265358979323846;
            for (int i = 0; i < prm->l; ++i)   // Sec. 2.2, Eq. (chebyshev)
                sigma[i] = 0.5 * (prm->lmax + prm->lmin) +
                           0.5 * (prm->lmax - prm->lmin) * std::cos((2 * i + 1) * pi / (2.0 * prm->l));
        }
        // Jacobi on a constant-coefficient stencil: M = c I, so the shifts of
        // M^{-1} A become shifts of A scaled by c (same iterates)
        if (prm->precond == PLCG_PRECOND_JACOBI)
            for (int k = 0; k < prm->l; ++k) sigma[k] *= d->center + d->diag_shift;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nacuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return nafail(PLCG_ERR_INVALID, "device ordinal too large");
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            // once per device, with that device current: the array's device address
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return nacuda(e, "cudaGetSymbolAddress(no-alloc scratch)");
            g_scratch_ptr[dev] = p;
        }
        base = static_cast<char *>(g_scratch_ptr[dev]);
    }
    StencilDesc st;
    st.dim = d->dim;
    st.nx = (int)d->nx;
    st.ny = (int)d->ny;
    st.nz = (int)nz;
    st.center = d->center + d->diag_shift;
    st.off = d->off;
    st.dnx = make_fastdiv((uint32_t)d->nx);
    st.dny = make_fastdiv((uint32_t)d->ny);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prm->prec == PLCG_FP64) return run<double>(st, n, b, x, prm, sigma, s, base, res);
    return run<float>(st, n, b, x, prm, sigma, s, base, res);
}
