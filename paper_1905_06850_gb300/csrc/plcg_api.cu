// plcg_api.cu -- host side of the C ABI declared in include/plcg.h.
//
// Validates arguments, owns device copies of the operator and the solve
// workspaces, picks a kernel instantiation (precision x operator x l) and
// launches it cooperatively (all CTAs co-resident, which the bounded grid
// barrier of the persistent solver relies on).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/plcg.h"
#include "plcg_internal.h"
#include "plcg_kernels.h"

using namespace plcg;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;
static unsigned long long g_poll_limit = 0;     // 0 = default
static int g_force_timeout = 0;

static plcg_status fail(plcg_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define CUDA_TRY(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? PLCG_ERR_NOMEM : PLCG_ERR_CUDA,   \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                    \
    } while (0)

extern "C" const char *plcg_last_error(void) { return g_last_error.c_str(); }
void plcg::set_last_error(const std::string &msg) { g_last_error = msg; }
extern "C" const char *plcg_version(void) { return "plcg 0.1 (sm_103a)"; }
extern "C" void plcg_debug_set_poll_limit(uint64_t polls) { g_poll_limit = polls; }
extern "C" void plcg_debug_force_barrier_timeout(int on) { g_force_timeout = on ? 1 : 0; }

// Systems of at most this many rows run on the cluster-resident solver
// (p(l >= 2)-CG and classic CG; p(1)-CG up to half of it), 0: never; set by
// plcg_set_cluster_rows.  The default comes from timing both paths on GB300:
// at 4096 rows the cluster is faster for every method (p(1)-CG 6.0 vs 6.8 us
// per iteration), at 10^4 rows for l >= 2 and CG (p(2)-CG 6.5 vs 7.7 us) but
// not for p(1)-CG (8.0 vs 7.1 us: sixteen SMs of FP64 units against twenty),
// and above ~2x10^4 rows the grid wins throughout.
constexpr int64_t kClusterRowsDefault = 12288;
constexpr int64_t kVec1Rows = 16384;
static int64_t g_cluster_rows = kClusterRowsDefault;

extern "C" plcg_status plcg_set_cluster_rows(int64_t max_rows)
{
    if (max_rows < 0) return fail(PLCG_ERR_INVALID, "plcg_set_cluster_rows: max_rows must be >= 0");
    g_cluster_rows = max_rows;
    return PLCG_OK;
}

// The largest cluster (<= want, 16 at most) that the device can place for
// func, or 0: clusters above 8 CTAs need the non-portable-size attribute.
static int cluster_size_for(const void *func, int want)
{
    static std::mutex mu;
    static std::unordered_map<const void *, int> cache;   // func -> largest placeable cluster
    int cmax = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(func);
        if (it != cache.end()) cmax = it->second;
    }
    if (cmax == 0) {
        cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        for (int c : {16, 8, 4, 2, 1}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)c);
            cfg.blockDim = dim3(kBlock);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = (unsigned)c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, func, &cfg) == cudaSuccess && nclusters >= 1) {
                cmax = c;
                break;
            }
        }
        cudaGetLastError();   // a refused size leaves no sticky error
        std::lock_guard<std::mutex> lk(mu);
        cache[func] = cmax > 0 ? cmax : -1;
    }
    return cmax > 0 ? std::min(cmax, std::max(1, want)) : 0;
}

static unsigned long long poll_limit()
{
    // ~2 s at 64 ns per poll (the poll itself adds an L2 round trip)
    return g_poll_limit ? g_poll_limit : 30000000ull;
}

// ------------------------------------------------------------------ matrix
struct Workspace {
    void *mem = nullptr;        // one allocation for everything below
    size_t bytes = 0;
};

static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct plcg_matrix {
    int kind = kOpStencil;
    int64_t n = 0;
    StencilDesc st{};
    int csr_prec = PLCG_FP64;
    int64_t nnz = 0;
    int64_t *rowptr = nullptr;
    int32_t *col = nullptr;
    void *val = nullptr;         // CSR values; structured 27-point: [14][cstride] coefficients
    int64_t cstride = 0;
    void *val_alloc = nullptr;   // structured 27-point: the allocation val points into
    size_t val_bytes = 0;        // ... and its size
    // Jacobi data (CSR): 1 / a_rr in FP64, 1 / a_rr and a_rr in the stored type
    double *jdinv64 = nullptr;
    void *jdinv = nullptr;
    void *jdiag = nullptr;       // CSR: own array; structured 27-point: coef[0] (not owned)
    bool jacobi_ok = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    Workspace ws;
    double *b_dev = nullptr, *x_dev = nullptr;   // plcg_solve_host staging
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    DevResult *host_res = nullptr;              // pinned
    std::mutex mu;
};

extern "C" void plcg_params_default(plcg_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->method = PLCG_METHOD_PLCG;
    p->l = 1;
    p->shifts = nullptr;
    p->lmin = 0.0;
    p->lmax = 8.0;
    p->rtol = 1e-8;
    p->maxit = 100000;
    p->prec = PLCG_FP64;
    p->dots_2l1 = 0;
    p->max_restarts = 8;
    p->inner_rtol_floor = 1e-4;
    p->grid_ctas = 0;
    p->precond = PLCG_PRECOND_NONE;
}

static plcg_status matrix_common_init(plcg_matrix *A, void *stream)
{
    A->stream = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaGetDevice(&A->device));
    CUDA_TRY(cudaDeviceGetAttribute(&A->num_sms, cudaDevAttrMultiProcessorCount, A->device));
    CUDA_TRY(cudaEventCreate(&A->ev0));
    CUDA_TRY(cudaEventCreate(&A->ev1));
    CUDA_TRY(cudaMallocHost(&A->host_res, sizeof(DevResult)));
    return PLCG_OK;
}

// Validates a stencil description and fills the operator fields of *A (kind,
// n, st); no CUDA call.
static plcg_status stencil_from_desc(const plcg_stencil_desc *d, plcg_matrix *A)
{
    if (!((d->dim == 2 && d->points == 5) || (d->dim == 3 && d->points == 7)))
        return fail(PLCG_ERR_INVALID, "stencil: need dim 2 with 5 points or dim 3 with 7 points");
    const int64_t nz = (d->dim == 3) ? d->nz : 1;
    if (d->nx < 1 || d->ny < 1 || nz < 1)
        return fail(PLCG_ERR_INVALID, "stencil: grid sizes must be >= 1");
    if (d->nx >= (1 << 30) || d->ny >= (1 << 30) || nz >= (1 << 30) ||
        d->nx * d->ny * nz >= (int64_t(1) << 31))
        return fail(PLCG_ERR_INVALID, "stencil: n must be < 2^31");
    if (!std::isfinite(d->center) || !std::isfinite(d->off) || !std::isfinite(d->diag_shift))
        return fail(PLCG_ERR_INVALID, "stencil: non-finite coefficient");
    A->kind = kOpStencil;
    A->n = d->nx * d->ny * nz;
    A->st.dim = d->dim;
    A->st.nx = (int)d->nx;
    A->st.ny = (int)d->ny;
    A->st.nz = (int)nz;
    A->st.center = d->center + d->diag_shift;
    A->st.off = d->off;
    A->st.dnx = make_fastdiv((uint32_t)d->nx);
    A->st.dny = make_fastdiv((uint32_t)d->ny);
    return PLCG_OK;
}

extern "C" plcg_status plcg_create_stencil(const plcg_stencil_desc *d, void *stream,
                                           plcg_matrix **out)
{
    if (!d || !out) return fail(PLCG_ERR_INVALID, "plcg_create_stencil: NULL argument");
    *out = nullptr;
    plcg_matrix tmp;
    plcg_status st = stencil_from_desc(d, &tmp);
    if (st != PLCG_OK) return st;
    plcg_matrix *A = new plcg_matrix();
    stencil_from_desc(d, A);
    st = matrix_common_init(A, stream);
    if (st != PLCG_OK) { plcg_destroy(A); return st; }
    *out = A;
    return PLCG_OK;
}

extern "C" plcg_status plcg_create_csr(int64_t n, int64_t nnz, const int64_t *rowptr,
                                       const int32_t *col, const double *val, int on_device,
                                       int prec, void *stream, plcg_matrix **out)
{
    if (!out) return fail(PLCG_ERR_INVALID, "plcg_create_csr: NULL out");
    *out = nullptr;
    if (n <= 0 || n >= (int64_t(1) << 31) || nnz < 0)
        return fail(PLCG_ERR_INVALID, "csr: need 0 < n < 2^31 and nnz >= 0");
    if (!rowptr || (nnz > 0 && (!col || !val)))
        return fail(PLCG_ERR_INVALID, "csr: NULL array");
    if (prec != PLCG_FP64 && prec != PLCG_FP32_FP64DOT)
        return fail(PLCG_ERR_INVALID, "csr: unknown precision %d", prec);
    if (!on_device) {
        if (rowptr[0] != 0 || rowptr[n] != nnz)
            return fail(PLCG_ERR_INVALID, "csr: rowptr[0] must be 0 and rowptr[n] = nnz");
        for (int64_t r = 0; r < n; ++r)
            if (rowptr[r + 1] < rowptr[r])
                return fail(PLCG_ERR_INVALID, "csr: rowptr decreases at row %lld", (long long)r);
        for (int64_t e = 0; e < nnz; ++e)
            if (col[e] < 0 || col[e] >= n)
                return fail(PLCG_ERR_INVALID, "csr: column index out of range at entry %lld",
                            (long long)e);
        for (int64_t e = 0; e < nnz; ++e)
            if (!std::isfinite(val[e]))
                return fail(PLCG_ERR_INVALID, "csr: non-finite value at entry %lld", (long long)e);
    }
    plcg_matrix *A = new plcg_matrix();
    A->kind = kOpCsr;
    A->n = n;
    A->nnz = nnz;
    A->csr_prec = prec;
    plcg_status st = matrix_common_init(A, stream);
    if (st != PLCG_OK) { plcg_destroy(A); return st; }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t vsz = (prec == PLCG_FP64) ? sizeof(double) : sizeof(float);
    // col and val carry 4 zeroed entries of padding: the solver bulk-copies
    // entry ranges rounded out to 16-byte boundaries
    cudaError_t e = cudaMalloc(&A->rowptr, (n + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&A->col, (nnz + 4) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&A->val, (nnz + 4) * vsz);
    if (e == cudaSuccess) e = cudaMemset(A->col, 0, (nnz + 4) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(A->val, 0, (nnz + 4) * vsz);
    if (e == cudaSuccess) e = cudaMemcpy(A->rowptr, rowptr, (n + 1) * sizeof(int64_t), kind);
    if (e == cudaSuccess && nnz) e = cudaMemcpy(A->col, col, nnz * sizeof(int32_t), kind);
    if (e == cudaSuccess && nnz) {
        if (prec == PLCG_FP64) {
            e = cudaMemcpy(A->val, val, nnz * sizeof(double), kind);
        } else {
            // round to FP32 once: on the device when the values already live there
            double *tmp = nullptr;
            const double *src = val;
            if (!on_device) {
                e = cudaMalloc(&tmp, nnz * sizeof(double));
                if (e == cudaSuccess) e = cudaMemcpy(tmp, val, nnz * sizeof(double), kind);
                src = tmp;
            }
            if (e == cudaSuccess) e = launch_round_to_f32(src, static_cast<float *>(A->val), nnz, nullptr);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (tmp) cudaFree(tmp);
        }
    }
    // Jacobi preconditioner data (Sec. 2.2): the diagonal and its inverse
    int *bad = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&A->jdinv64, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&A->jdiag, n * vsz);
    if (e == cudaSuccess) {
        if (prec == PLCG_FP64) A->jdinv = A->jdinv64;
        else e = cudaMalloc(&A->jdinv, n * vsz);
    }
    if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(bad, 0, sizeof(int));
    if (e == cudaSuccess)
        e = launch_jacobi_setup(prec != PLCG_FP64, A->rowptr, A->col, A->val, n, A->jdinv64,
                                A->jdinv, A->jdiag, bad, nullptr);
    int hbad = 1;
    if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (bad) cudaFree(bad);
    A->jacobi_ok = (e == cudaSuccess && hbad == 0);
    if (e != cudaSuccess) {
        plcg_status s2 = fail(e == cudaErrorMemoryAllocation ? PLCG_ERR_NOMEM : PLCG_ERR_CUDA,
                              "csr upload: %s", cudaGetErrorString(e));
        plcg_destroy(A);
        return s2;
    }
    *out = A;
    return PLCG_OK;
}

extern "C" plcg_status plcg_create_var27(int64_t nx, int64_t ny, int64_t nz, const double *coef,
                                         int on_device, int prec, void *stream, plcg_matrix **out)
{
    if (!out) return fail(PLCG_ERR_INVALID, "plcg_create_var27: NULL out");
    *out = nullptr;
    if (!coef) return fail(PLCG_ERR_INVALID, "var27: NULL coefficients");
    if (nx < 1 || ny < 1 || nz < 1 || nx >= (1 << 30) || ny >= (1 << 30) || nz >= (1 << 30))
        return fail(PLCG_ERR_INVALID, "var27: grid sizes must be in [1, 2^30)");
    const int64_t n = nx * ny * nz;
    if (n >= (int64_t(1) << 31)) return fail(PLCG_ERR_INVALID, "var27: n must be < 2^31");
    if (prec != PLCG_FP64 && prec != PLCG_FP32_FP64DOT)
        return fail(PLCG_ERR_INVALID, "var27: unknown precision %d", prec);
    if (!on_device)
        for (int64_t e = 0; e < 14 * n; ++e)
            if (!std::isfinite(coef[e]))
                return fail(PLCG_ERR_INVALID, "var27: non-finite coefficient at entry %lld", (long long)e);
    plcg_matrix *A = new plcg_matrix();
    A->kind = kOpVar27;
    A->n = n;
    A->csr_prec = prec;
    A->st.dim = 3;
    A->st.nx = (int)nx;
    A->st.ny = (int)ny;
    A->st.nz = (int)nz;
    A->st.dnx = make_fastdiv((uint32_t)nx);
    A->st.dny = make_fastdiv((uint32_t)ny);
    plcg_status st = matrix_common_init(A, stream);
    if (st != PLCG_OK) { plcg_destroy(A); return st; }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t vsz = (prec == PLCG_FP64) ? sizeof(double) : sizeof(float);
    const size_t cnt = (size_t)14 * n;
    // the 14 arrays start on 256-byte boundaries, with v27_halo(nx, ny) zero
    // elements before the first and at least as many after each (the stride
    // is n rounded up to 64 elements plus the halo), so the staged sweep's
    // 16-byte-rounded copies of backward coefficients stay inside zeros
    const int64_t halo = v27_halo(nx, ny);
    A->cstride = (n + 63) / 64 * 64 + halo;
    A->val_bytes = ((size_t)halo + (size_t)14 * A->cstride + 64) * vsz;
    cudaError_t e = cudaMalloc(&A->val_alloc, A->val_bytes);
    if (e == cudaSuccess) e = cudaMemset(A->val_alloc, 0, A->val_bytes);
    A->val = static_cast<char *>(A->val_alloc) + halo * vsz;
    if (e == cudaSuccess) {
        if (prec == PLCG_FP64) {
            e = cudaMemcpy2D(A->val, A->cstride * sizeof(double), coef, n * sizeof(double),
                             n * sizeof(double), 14, kind);
        } else {
            double *tmp = nullptr;
            const double *src = coef;
            if (!on_device) {
                e = cudaMalloc(&tmp, cnt * sizeof(double));
                if (e == cudaSuccess) e = cudaMemcpy(tmp, coef, cnt * sizeof(double), kind);
                src = tmp;
            }
            for (int j = 0; j < 14 && e == cudaSuccess; ++j)
                e = launch_round_to_f32(src + (size_t)j * n, static_cast<float *>(A->val) + (size_t)j * A->cstride,
                                        n, nullptr);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (tmp) cudaFree(tmp);
        }
    }
    // entries towards cells outside the grid are ignored: store them as zero,
    // so that the tiled sweep applies every row without boundary tests
    if (e == cudaSuccess) e = launch_var27_zero_outside(prec != PLCG_FP64, A->val, A->cstride, A->st, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    // Jacobi data: the diagonal is coef[0]; its inverse is formed here
    int *bad = nullptr;
    A->jdiag = A->val;
    if (e == cudaSuccess) e = cudaMalloc(&A->jdinv64, n * sizeof(double));
    if (e == cudaSuccess) {
        // padded to 256 bytes: the tiled sweep bulk-copies 16-byte groups
        if (prec == PLCG_FP64) A->jdinv = A->jdinv64;
        else e = cudaMalloc(&A->jdinv, align_up(n * vsz, 256));
    }
    if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(bad, 0, sizeof(int));
    if (e == cudaSuccess)
        e = launch_var27_jacobi_setup(prec != PLCG_FP64, A->val, n, A->jdinv64, A->jdinv, bad, nullptr);
    int hbad = 1;
    if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (bad) cudaFree(bad);
    A->jacobi_ok = (e == cudaSuccess && hbad == 0);
    if (e != cudaSuccess) {
        plcg_status s2 = fail(e == cudaErrorMemoryAllocation ? PLCG_ERR_NOMEM : PLCG_ERR_CUDA,
                              "var27 upload: %s", cudaGetErrorString(e));
        plcg_destroy(A);
        return s2;
    }
    *out = A;
    return PLCG_OK;
}

extern "C" void plcg_destroy(plcg_matrix *A)
{
    if (!A) return;
    if (A->stream) cudaStreamSynchronize(A->stream);
    else cudaDeviceSynchronize();
    cudaFree(A->rowptr);
    cudaFree(A->col);
    if (A->jdiag != A->val) cudaFree(A->jdiag);
    cudaFree(A->val_alloc ? A->val_alloc : A->val);
    if (A->jdinv != A->jdinv64) cudaFree(A->jdinv);
    cudaFree(A->jdinv64);
    cudaFree(A->ws.mem);
    cudaFree(A->b_dev);
    cudaFree(A->x_dev);
    if (A->host_res) cudaFreeHost(A->host_res);
    if (A->ev0) cudaEventDestroy(A->ev0);
    if (A->ev1) cudaEventDestroy(A->ev1);
    delete A;
}

// ------------------------------------------------------------------ solve
static void chebyshev_shifts(int l, double lmin, double lmax, double *sig)
{
    // Sec. 2.2, Eq. (chebyshev): zeros of T_l mapped to [lmin, lmax]
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < l; ++i)
        sig[i] = 0.5 * (lmax + lmin) + 0.5 * (lmax - lmin) * std::cos((2 * i + 1) * pi / (2.0 * l));
}

// The shifts of a p(l)-CG solve: prm->shifts, else Chebyshev shifts on
// [lmin, lmax].  With the Jacobi preconditioner they describe M^{-1} A; for
// a constant-coefficient stencil M = c I, and the solve runs the
// unpreconditioned recurrences on A with the shifts scaled by c -- the same
// iterates and scalars in exact arithmetic, with natural norms that are the
// 2-norms divided by sqrt(c) on both sides of the stop test.
static void resolve_shifts(const plcg_matrix *A, const plcg_params *prm, double lmin, double lmax,
                           double *sigma)
{
    if (prm->shifts) std::memcpy(sigma, prm->shifts, prm->l * sizeof(double));
    else chebyshev_shifts(prm->l, lmin, lmax, sigma);
    if (prm->precond == PLCG_PRECOND_JACOBI && A->kind == kOpStencil)
        for (int k = 0; k < prm->l; ++k) sigma[k] *= A->st.center;
}

static plcg_status ensure_ws(plcg_matrix *A, size_t bytes)
{
    if (A->ws.bytes >= bytes) return PLCG_OK;
    if (A->ws.mem) {
        if (A->stream) cudaStreamSynchronize(A->stream);
        cudaFree(A->ws.mem);
        A->ws.mem = nullptr;
        A->ws.bytes = 0;
    }
    CUDA_TRY(cudaMalloc(&A->ws.mem, bytes));
    A->ws.bytes = bytes;
    return PLCG_OK;
}


// Layout of one solve's workspace and its kernel arguments.  With base ==
// nullptr only the sizes are computed; *bytes is the workspace size and
// *out_off the offset of the result record inside it.
template <typename T>
static plcg_status build_solve(const plcg_matrix *A, const double *b, double *x,
                               const plcg_params *prm, const double *sigma, int max_ctas,
                               char *base, SolveArgs<T> *args, const void **func_out,
                               int64_t *P_out, int *per_sm_out, size_t *bytes, size_t *out_off)
{
    const int64_t n = A->n;
    const int l = prm->l;
    const bool cg = prm->method == PLCG_METHOD_CG;
    const bool jac = prm->precond == PLCG_PRECOND_JACOBI && A->kind != kOpStencil;
    const int op = !jac ? A->kind : (A->kind == kOpCsr) ? (int)kOpCsrJacobi : (int)kOpVar27Jacobi;
    const bool f32 = sizeof(T) == 4;
    // FP64 vectors over FP32 matrix values (the matrix was created with FP32 values)
    const bool c32 = prm->prec == PLCG_FP32_MATRIX;
    if (c32 && f32) return fail(PLCG_ERR_INVALID, "internal: FP32 matrix path with FP32 vectors");
    const unsigned value_bytes = c32 ? 4u : (unsigned)sizeof(T);
    // Stencil rows per thread: 16 bytes of a vector (rows in one x-line),
    // except FP64 systems of at most kVec1Rows rows, which take one row per
    // thread so that their FP64-bound sweep spreads over twice the SMs (or
    // balances better over one cluster's 16): measured on GB300, 2D 100^2
    // p(1)-CG 7.11 -> 6.61 us per iteration, p(2) 6.54 -> 6.06, 2D 64^2 p(1)
    // 5.93 -> 5.16, 3D 20^3 p(1) 7.70 -> 6.78; from ~6*10^4 rows it costs
    // (3D 40^3 p(1) 8.9 -> 10.4 us), and the FP32 sweeps never gain
    int vec = 1;
    if (op == kOpStencil) {
        const int want = 16 / (int)sizeof(T);
        vec = (A->st.nx % want == 0 && !(sizeof(T) == 8 && n <= kVec1Rows)) ? want : 1;
    }
    // FP64 p(l)-CG on 2^19 rows or more: the scaled-basis kernel (one FP64
    // multiply per recurrence and row fewer; below that the longer scalar step
    // costs more) -- l <= 5 on the stencils, l = 1 on the stored operators
    const bool sc = !f32 && !cg && n >= (int64_t(1) << 19) && (l == 1 || (op == kOpStencil && l <= 5));
    const void *func = kernel_ptr(f32, op, vec, cg ? 0 : l, cg, sc, c32);
    if (!func) return fail(PLCG_ERR_UNIMPL, "no kernel for prec=%d op=%d vec=%d l=%d", prm->prec, op, vec, l);
    // CSR kernels stage each unit's entries in dynamic shared memory (FP64
    // classic CG excepted, see cg_body); the FP32 27-point kernels stage
    // coefficient and z tiles (classic CG's SpMV without vector slots)
    unsigned dsmem = (op_is_csr(op) && (!cg || f32)) ? csr_stage_bytes(value_bytes)
                   : (op_is_var27(op) && f32 && !c32)
                       ? (cg ? v27_tile_bytes_cg((unsigned)sizeof(T))
                             : v27_tile_bytes((unsigned)sizeof(T), l, op_is_jacobi(op))) : 0u;
    if (dsmem) {
        CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
        CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    }
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, kBlock, dsmem));
    if (per_sm < 1) return fail(PLCG_ERR_CUDA, "solver kernel cannot be resident");
    const int64_t unit = (int64_t)kBlock * vec;
    const int64_t nunits = (n + unit - 1) / unit;
    int64_t P = (int64_t)per_sm * A->num_sms;
    if (prm->grid_ctas > 0) P = std::min<int64_t>(P, prm->grid_ctas);
    if (max_ctas > 0) P = std::min<int64_t>(P, max_ctas);
    P = std::max<int64_t>(1, std::min<int64_t>(P, nunits));
    // small systems: one thread-block cluster holds the whole solve (its
    // barrier and distributed shared memory replace the grid barrier and the
    // partials in global memory)
    int cluster = 0;
    if (n <= (cg || l >= 2 ? g_cluster_rows : g_cluster_rows / 2) && !c32 &&
        (op == kOpStencil || op == kOpCsr) && (cg || l <= 4) && prm->grid_ctas == 0) {
        const void *cf = f32 ? kptr_cluster_f32(op, vec, cg ? 0 : l, cg) : kptr_cluster_f64(op, vec, cg ? 0 : l, cg);
        const int c = cf ? cluster_size_for(cf, (int)std::min<int64_t>(16, nunits)) : 0;
        if (c > 0 && (max_ctas == 0 || c <= max_ctas)) {
            func = cf;
            cluster = c;
            P = c;
            per_sm = 1;
            dsmem = 0;
        }
    }

    SolveArgs<T> &a = *args;
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
        nvec = 3;   // p ring of two + the FP32 inner iterate
    }
    // ring vectors are packed with stride n (ring() indexes whole vectors);
    // 128-bit access needs n * sizeof(T) to be a multiple of 16
    if (((size_t)n * sizeof(T)) % 16 != 0 && vec > 1)
        return fail(PLCG_ERR_INVALID, "internal: vector length not 16-byte aligned");
    // structured 27-point operators: a zero halo before the first ring vector
    // and at least one after every vector (the stride includes it), zeroed by
    // the kernel at the start of each solve, so that the tiles' z-line copies
    // stay inside the vector and zeros
    const int64_t halo = op_is_var27(op) ? v27_halo(A->st.nx, A->st.ny) : 0;
    const size_t vbytes = align_up((size_t)(n + halo) * sizeof(T), 256);
    size_t off = 0;
    const size_t o_ring = off; off += (size_t)halo * sizeof(T) + vbytes * nvec;
    const size_t o_p = off; off += vbytes;
    const size_t o_rc = off; off += vbytes;
    const size_t o_r = off; off += align_up((size_t)n * sizeof(double), 256);
    const int slots = cg ? 2 : (l + 1);
    const size_t o_part = off; off += align_up((size_t)slots * P * kMaxDots * sizeof(double), 256);
    const size_t o_npart = off; off += align_up((size_t)P * kNormSlots * sizeof(double), 256);
    const size_t o_bar = off; off += 256;
    const size_t o_out = off; off += align_up(sizeof(DevResult), 256);
    *bytes = off;
    *out_off = o_out;
    *func_out = func;
    *P_out = P;
    *per_sm_out = per_sm;
    if (!base) return PLCG_OK;
    a.n = n;
    a.st = A->st;
    a.csr.rowptr = A->rowptr;
    a.csr.col = A->col;
    a.csr.val = A->val;
    a.csr.stride = A->cstride;
    a.vstride = (int64_t)(vbytes / sizeof(T));   // ring vectors 256-byte aligned
    a.ws_lo = base;
    a.ws_hi = base + off;
    if (A->val_alloc) {
        a.cf_lo = static_cast<const char *>(A->val_alloc);
        a.cf_hi = a.cf_lo + A->val_bytes;
    }
    if (jac) {
        // 1 / a_rr in the vector type (FP64 vectors: the FP64 inverse), a_rr
        // in the stored value type
        a.csr.dinv = f32 ? A->jdinv : static_cast<const void *>(A->jdinv64);
        a.csr.diag = A->jdiag;
        a.dinv64 = A->jdinv64;
    }
    a.b = b;
    a.x = x;
    a.r = reinterpret_cast<double *>(base + o_r);
    a.zring = reinterpret_cast<T *>(base + o_ring + (size_t)halo * sizeof(T));
    a.halo = halo;
    a.nring = nvec;
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
    a.poll_limit = poll_limit();
    a.force_timeout = g_force_timeout;
    // l >= 2: compute each iteration's scalars during the previous sweep where
    // that latency is a visible share of an iteration (smaller systems)
    a.lookahead = (!cg && l >= 2 && n < (int64_t(1) << 22)) ? 1 : 0;
    a.dsmem = dsmem;
    a.cluster = cluster;
    // staging a warp's CSR entries pays when rows are long; short rows (the
    // diagonal toy has one entry) read them directly (measured)
    a.stage = (op_is_csr(op) && A->nnz >= 4 * n && !cluster) ? 1 : 0;
    return PLCG_OK;
}

// Launch shape and flags of the calling thread's last single-solve launch
// (plcg_debug_last_launch).
static thread_local plcg_launch_info g_last_launch{};

extern "C" void plcg_debug_last_launch(plcg_launch_info *out)
{
    if (out) *out = g_last_launch;
}

// Clear the barrier counter and result record, then launch the persistent
// solver cooperatively (every CTA resident) on `stream`; returns at once.
template <typename T>
static plcg_status launch_built(const SolveArgs<T> &a0, const void *func, int64_t P,
                                cudaStream_t stream)
{
    SolveArgs<T> a = a0;
    CUDA_TRY(cudaMemsetAsync(a.bar, 0, 256, stream));
    CUDA_TRY(cudaMemsetAsync(a.out, 0, sizeof(DevResult), stream));
    g_last_launch.kernel = (uint64_t)reinterpret_cast<uintptr_t>(func);
    g_last_launch.grid_ctas = (int)P;
    g_last_launch.dyn_smem = a.dsmem;
    g_last_launch.lookahead = a.lookahead;
    g_last_launch.staged = a.stage;
    g_last_launch.poll_limit = a.poll_limit;
    g_last_launch.force_timeout = a.force_timeout;
    g_last_launch.cluster = a.cluster;
    void *args[] = {&a};
    if (a.cluster > 0) {
        // the grid is one cluster: the hardware places all its CTAs together
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)P);
        cfg.blockDim = dim3(kBlock);
        cfg.dynamicSmemBytes = a.dsmem;
        cfg.stream = stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)P;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        CUDA_TRY(cudaLaunchKernelExC(&cfg, func, args));
    } else {
        CUDA_TRY(cudaLaunchCooperativeKernel(func, dim3((unsigned)P), dim3(kBlock), args, a.dsmem, stream));
    }
    return PLCG_OK;
}

static plcg_status result_status(const DevResult &o)
{
    if (o.status == PLCG_ERR_TIMEOUT)
        return fail(PLCG_ERR_TIMEOUT, "a bounded device wait expired (grid barrier)");
    if (o.status != PLCG_OK) {
        const char *why = o.status == PLCG_ERR_BREAKDOWN ? "square-root breakdowns exceeded max_restarts"
                        : o.status == PLCG_ERR_MAXIT ? "iteration budget exhausted"
                        : o.status == PLCG_ERR_NONFINITE ? "non-finite value in the recurrences"
                        : "solve failed";
        return fail((plcg_status)o.status, "%s", why);
    }
    return PLCG_OK;
}

template <typename T>
static plcg_status run_solve(plcg_matrix *A, const double *b, double *x, const plcg_params *prm,
                             const double *sigma, plcg_result *res, double *trace = nullptr,
                             int trace_cap = 0)
{
    SolveArgs<T> a;
    const void *func = nullptr;
    int64_t P = 0;
    int per_sm = 0;
    size_t bytes = 0, o_out = 0;
    plcg_status st = build_solve<T>(A, b, x, prm, sigma, 0, nullptr, &a, &func, &P, &per_sm, &bytes, &o_out);
    if (st != PLCG_OK) return st;
    st = ensure_ws(A, bytes);
    if (st != PLCG_OK) return st;
    st = build_solve<T>(A, b, x, prm, sigma, 0, static_cast<char *>(A->ws.mem), &a, &func, &P,
                        &per_sm, &bytes, &o_out);
    if (st != PLCG_OK) return st;
    a.trace = trace;
    a.trace_cap = trace_cap;
    CUDA_TRY(cudaEventRecord(A->ev0, A->stream));
    st = launch_built<T>(a, func, P, A->stream);
    if (st != PLCG_OK) return st;
    CUDA_TRY(cudaEventRecord(A->ev1, A->stream));
    CUDA_TRY(cudaMemcpyAsync(A->host_res, a.out, sizeof(DevResult), cudaMemcpyDeviceToHost, A->stream));
    CUDA_TRY(cudaStreamSynchronize(A->stream));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, A->ev0, A->ev1));
    const DevResult &o = *A->host_res;
    if (res) {
        res->status = o.status;
        res->iters = o.iters;
        res->spmvs = o.spmvs;
        res->restarts = o.restarts;
        res->refinements = o.refinements;
        res->recursive_relres = o.recursive_relres;
        res->true_relres = o.true_relres;
        res->seconds = ms * 1e-3;
        res->latency = res->seconds;
    }
    return result_status(o);
}

static plcg_status check_params(const plcg_matrix *A, const plcg_params *p)
{
    if (!p) return fail(PLCG_ERR_INVALID, "NULL params");
    if (p->method != PLCG_METHOD_PLCG && p->method != PLCG_METHOD_CG)
        return fail(PLCG_ERR_INVALID, "unknown method %d", p->method);
    if (p->method == PLCG_METHOD_PLCG && (p->l < 1 || p->l > kMaxL))
        return fail(PLCG_ERR_INVALID, "l must be in 1..%d", kMaxL);
    if (!(p->rtol > 0.0) || !std::isfinite(p->rtol))
        return fail(PLCG_ERR_INVALID, "rtol must be a positive finite number");
    if (p->maxit < 0 || p->maxit > (int64_t(1) << 30))
        return fail(PLCG_ERR_INVALID, "maxit must be in [0, 2^30]");
    if (p->max_restarts < 0) return fail(PLCG_ERR_INVALID, "max_restarts must be >= 0");
    if (p->prec != PLCG_FP64 && p->prec != PLCG_FP32_FP64DOT && p->prec != PLCG_FP32_MATRIX)
        return fail(PLCG_ERR_INVALID, "unknown precision %d", p->prec);
    if (p->prec == PLCG_FP32_MATRIX) {
        if (A->kind == kOpStencil)
            return fail(PLCG_ERR_UNIMPL, "PLCG_FP32_MATRIX: a stencil operator stores no matrix values");
        if (A->csr_prec != PLCG_FP32_FP64DOT)
            return fail(PLCG_ERR_INVALID, "PLCG_FP32_MATRIX needs a matrix created with FP32 values "
                                          "(PLCG_FP32_FP64DOT)");
    } else if (A->kind != kOpStencil && p->prec != A->csr_prec) {
        return fail(PLCG_ERR_INVALID, "matrix was created for precision %d", A->csr_prec);
    }
    if (p->prec == PLCG_FP32_FP64DOT && !(p->inner_rtol_floor > 0.0 && p->inner_rtol_floor < 1.0))
        return fail(PLCG_ERR_INVALID, "inner_rtol_floor must be in (0, 1)");
    if (p->precond != PLCG_PRECOND_NONE && p->precond != PLCG_PRECOND_JACOBI)
        return fail(PLCG_ERR_INVALID, "unknown preconditioner %d", p->precond);
    if (p->precond == PLCG_PRECOND_JACOBI) {
        if (A->kind != kOpStencil && !A->jacobi_ok)
            return fail(PLCG_ERR_INVALID, "Jacobi preconditioner: a diagonal entry is not positive");
        if (A->kind == kOpStencil && !(A->st.center > 0.0))
            return fail(PLCG_ERR_INVALID, "Jacobi preconditioner: the stencil center is not positive");
    }
    if (p->method == PLCG_METHOD_PLCG) {
        if (p->shifts) {
            for (int k = 0; k < p->l; ++k)
                if (!std::isfinite(p->shifts[k])) return fail(PLCG_ERR_INVALID, "non-finite shift");
        } else if (!std::isfinite(p->lmin) || !std::isfinite(p->lmax) || p->lmax < p->lmin) {
            return fail(PLCG_ERR_INVALID, "need lmin <= lmax for the Chebyshev shifts");
        }
    }
    return PLCG_OK;
}

extern "C" plcg_status plcg_solve(plcg_matrix *A, const double *b, double *x,
                                  const plcg_params *prm, plcg_result *res)
{
    if (!A || !b || !x) return fail(PLCG_ERR_INVALID, "plcg_solve: NULL argument");
    plcg_status st = check_params(A, prm);
    if (st != PLCG_OK) return st;
    if ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15)
        return fail(PLCG_ERR_INVALID, "b and x must be 16-byte aligned");
    double sigma[kMaxL] = {0};
    if (prm->method == PLCG_METHOD_PLCG) resolve_shifts(A, prm, prm->lmin, prm->lmax, sigma);
    std::lock_guard<std::mutex> lock(A->mu);
    CUDA_TRY(cudaSetDevice(A->device));
    if (prm->prec != PLCG_FP32_FP64DOT) return run_solve<double>(A, b, x, prm, sigma, res);
    return run_solve<float>(A, b, x, prm, sigma, res);
}

// A solve whose workspace is the caller's [base, base + cap): the argument
// checks, shifts, kernel choice, launch shape and kernel arguments of
// plcg_solve (build_solve), with no allocation.  Synchronous; res->seconds = 0.
template <typename T>
static plcg_status run_solve_fixed(const plcg_matrix *A, const double *b, double *x,
                                   const plcg_params *prm, const double *sigma, char *base,
                                   size_t cap, const char *who, plcg_result *res)
{
    SolveArgs<T> a;
    const void *func = nullptr;
    int64_t P = 0;
    int per_sm = 0;
    size_t bytes = 0, o_out = 0;
    plcg_status st = build_solve<T>(A, b, x, prm, sigma, 0, nullptr, &a, &func, &P, &per_sm, &bytes, &o_out);
    if (st != PLCG_OK) return st;
    if (bytes > cap)
        return fail(PLCG_ERR_INVALID,
                    "%s: this solve needs %zu bytes of scratch; the fixed no-allocation scratch holds %zu bytes "
                    "(use plcg_solve)", who, bytes, cap);
    st = build_solve<T>(A, b, x, prm, sigma, 0, base, &a, &func, &P, &per_sm, &bytes, &o_out);
    if (st != PLCG_OK) return st;
    st = launch_built<T>(a, func, P, A->stream);
    if (st != PLCG_OK) return st;
    DevResult o;
    CUDA_TRY(cudaMemcpyAsync(&o, a.out, sizeof(DevResult), cudaMemcpyDeviceToHost, A->stream));
    CUDA_TRY(cudaStreamSynchronize(A->stream));
    if (res) {
        res->status = o.status;
        res->iters = o.iters;
        res->spmvs = o.spmvs;
        res->restarts = o.restarts;
        res->refinements = o.refinements;
        res->recursive_relres = o.recursive_relres;
        res->true_relres = o.true_relres;
        res->seconds = 0.0;   // no CUDA events are recorded on this path
        res->latency = 0.0;
    }
    return result_status(o);
}

plcg_status plcg::solve_stencil_fixed(const plcg_stencil_desc *d, const double *b, double *x,
                                      const plcg_params *prm, plcg_result *res, void *stream,
                                      char *base, size_t cap, const char *who)
{
    if (!d || !b || !x || !prm) return fail(PLCG_ERR_INVALID, "%s: NULL argument", who);
    plcg_matrix A;   // a host-side description only: no device data, no allocation
    plcg_status st = stencil_from_desc(d, &A);
    if (st != PLCG_OK) return st;
    st = check_params(&A, prm);
    if (st != PLCG_OK) return st;
    if ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15)
        return fail(PLCG_ERR_INVALID, "b and x must be 16-byte aligned");
    A.stream = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaGetDevice(&A.device));
    CUDA_TRY(cudaDeviceGetAttribute(&A.num_sms, cudaDevAttrMultiProcessorCount, A.device));
    double sigma[kMaxL] = {0};
    if (prm->method == PLCG_METHOD_PLCG) resolve_shifts(&A, prm, prm->lmin, prm->lmax, sigma);
    if (prm->prec != PLCG_FP32_FP64DOT) return run_solve_fixed<double>(&A, b, x, prm, sigma, base, cap, who, res);
    return run_solve_fixed<float>(&A, b, x, prm, sigma, base, cap, who, res);
}

extern "C" plcg_status plcg_solve_host(plcg_matrix *A, const double *b, double *x,
                                       const plcg_params *prm, plcg_result *res)
{
    if (!A || !b || !x) return fail(PLCG_ERR_INVALID, "plcg_solve_host: NULL argument");
    plcg_status st = check_params(A, prm);
    if (st != PLCG_OK) return st;
    {
        std::lock_guard<std::mutex> lock(A->mu);
        CUDA_TRY(cudaSetDevice(A->device));
        if (!A->b_dev) CUDA_TRY(cudaMalloc(&A->b_dev, A->n * sizeof(double)));
        if (!A->x_dev) CUDA_TRY(cudaMalloc(&A->x_dev, A->n * sizeof(double)));
        CUDA_TRY(cudaMemcpyAsync(A->b_dev, b, A->n * sizeof(double), cudaMemcpyHostToDevice, A->stream));
        CUDA_TRY(cudaMemcpyAsync(A->x_dev, x, A->n * sizeof(double), cudaMemcpyHostToDevice, A->stream));
    }
    st = plcg_solve(A, A->b_dev, A->x_dev, prm, res);
    if (st == PLCG_ERR_INVALID || st == PLCG_ERR_CUDA || st == PLCG_ERR_UNIMPL || st == PLCG_ERR_NOMEM)
        return st;
    std::lock_guard<std::mutex> lock(A->mu);
    CUDA_TRY(cudaMemcpyAsync(x, A->x_dev, A->n * sizeof(double), cudaMemcpyDeviceToHost, A->stream));
    CUDA_TRY(cudaStreamSynchronize(A->stream));
    return st;
}

// ------------------------------------------------------------------ spectrum
// Number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm
// sequence of the LDL^T pivots; Golub & Van Loan, Matrix Computations, 8.4).
static int sturm_count(const std::vector<double> &d, const std::vector<double> &e, double x)
{
    int cnt = 0;
    double q = 1.0;
    for (size_t j = 0; j < d.size(); ++j) {
        q = (d[j] - x) - (j ? e[j - 1] * e[j - 1] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// The k-th smallest eigenvalue (k = 0 .. m-1) by bisection on [lo, hi].
static double tridiag_eig(const std::vector<double> &d, const std::vector<double> &e, int k, double lo,
                          double hi)
{
    for (int it = 0; it < 200 && hi - lo > 1e-13 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(d, e, mid) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

extern "C" plcg_status plcg_estimate_interval(plcg_matrix *A, const plcg_params *prm, int steps,
                                              double *lmin, double *lmax)
{
    if (!A || !prm || !lmin || !lmax) return fail(PLCG_ERR_INVALID, "plcg_estimate_interval: NULL argument");
    if (steps < 2 || steps > 1000) return fail(PLCG_ERR_INVALID, "plcg_estimate_interval: steps must be in [2, 1000]");
    plcg_params p = *prm;
    p.method = PLCG_METHOD_CG;
    p.maxit = steps;
    p.rtol = 1e-300;
    p.max_restarts = 0;
    p.inner_rtol_floor = 1e-300;   // FP32 path: the first inner solve runs all steps
    plcg_status st = check_params(A, &p);
    if (st != PLCG_OK) return st;
    std::lock_guard<std::mutex> lock(A->mu);
    CUDA_TRY(cudaSetDevice(A->device));
    if (!A->b_dev) CUDA_TRY(cudaMalloc(&A->b_dev, A->n * sizeof(double)));
    if (!A->x_dev) CUDA_TRY(cudaMalloc(&A->x_dev, A->n * sizeof(double)));
    double *trace = nullptr;
    CUDA_TRY(cudaMalloc(&trace, 2 * (size_t)steps * sizeof(double)));
    cudaError_t e = launch_fill_random(A->b_dev, A->n, 0x5eed5eedull, A->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(A->x_dev, 0, A->n * sizeof(double), A->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(trace, 0, 2 * (size_t)steps * sizeof(double), A->stream);
    if (e != cudaSuccess) {
        cudaFree(trace);
        return fail(PLCG_ERR_CUDA, "plcg_estimate_interval: %s", cudaGetErrorString(e));
    }
    plcg_result res{};
    const double nosig[kMaxL] = {0};   // classic CG uses no shifts
    st = (p.prec != PLCG_FP32_FP64DOT) ? run_solve<double>(A, A->b_dev, A->x_dev, &p, nosig, &res, trace, steps)
                               : run_solve<float>(A, A->b_dev, A->x_dev, &p, nosig, &res, trace, steps);
    std::vector<double> t(2 * (size_t)steps, 0.0);
    e = cudaMemcpy(t.data(), trace, t.size() * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(trace);
    if (e != cudaSuccess) return fail(PLCG_ERR_CUDA, "plcg_estimate_interval: %s", cudaGetErrorString(e));
    if (st != PLCG_OK && st != PLCG_ERR_MAXIT) return st;
    // Lanczos tridiagonal of the (preconditioned) operator from the CG
    // coefficients (Saad, Iterative Methods, Sec. 6.7.3):
    // T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j
    // the steps the first segment recorded (it ends early only when CG does)
    int k = 0;
    while (k < (int)std::min<int64_t>(res.iters, steps) && t[2 * k] != 0.0) ++k;
    if (k < 1) return fail(PLCG_ERR_INVALID, "plcg_estimate_interval: no CG step completed");
    std::vector<double> d(k), off(k > 1 ? k - 1 : 0);
    for (int j = 0; j < k; ++j) {
        const double al = t[2 * j], be = t[2 * j + 1];
        if (!(al > 0.0) || !std::isfinite(al) || !(be >= 0.0))
            return fail(PLCG_ERR_NONFINITE, "plcg_estimate_interval: invalid CG coefficient");
        d[j] = 1.0 / al + (j ? t[2 * j - 1] / t[2 * j - 2] : 0.0);
        if (j + 1 < k) off[j] = std::sqrt(be) / al;
    }
    double lo = d[0], hi = d[0];   // Gershgorin bracket of T
    for (int j = 0; j < k; ++j) {
        const double r = (j ? std::fabs(off[j - 1]) : 0.0) + (j + 1 < k ? std::fabs(off[j]) : 0.0);
        lo = std::min(lo, d[j] - r);
        hi = std::max(hi, d[j] + r);
    }
    *lmin = tridiag_eig(d, off, 0, lo, hi);
    *lmax = tridiag_eig(d, off, k - 1, lo, hi);
    return PLCG_OK;
}

// ------------------------------------------------------------------ batched
namespace {

// Device buffers of batched solves, per device, grown on demand and kept
// until the process exits.
struct BatchCtx {
    std::mutex mu;
    char *mem = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};
BatchCtx g_batch[64];

}  // namespace

// Batched schedule (set by the autotuner through plcg_set_batched_schedule):
// gang size G, the work threshold (as a multiple of one CTA's fair share)
// above which a system goes to the gangs, and the largest fraction of the
// launch's CTAs that may form gangs.
static int g_batch_G = 8;
static double g_batch_beta = 1.0;
static double g_batch_gang_frac = 0.5;
// Launch shape of FP32 batched solves (0, 0, 0: each method's default).
static int g_batch_ctas_per_sm = 0;
static int g_batch_rows_per_thread = 0;
static int g_batch_vector_width = 0;

extern "C" plcg_status plcg_set_batched_launch(int ctas_per_sm, int rows_per_thread, int vector_width)
{
    if (ctas_per_sm == 0 && rows_per_thread == 0 && vector_width == 0) {
        g_batch_ctas_per_sm = g_batch_rows_per_thread = g_batch_vector_width = 0;
        return PLCG_OK;
    }
    const bool rows = (ctas_per_sm == 3 || ctas_per_sm == 4) && vector_width == 1 &&
                      (rows_per_thread == 1 || rows_per_thread == 2 || rows_per_thread == 4);
    const bool pairs = ctas_per_sm == 4 && rows_per_thread == 1 && vector_width == 2;
    if (!rows && !pairs)
        return fail(PLCG_ERR_INVALID, "batched launch shape: need 3 or 4 CTAs per SM, 1, 2 or 4 row groups "
                                      "per thread and vector width 1, or (4, 1, 2), or (0, 0, 0)");
    g_batch_ctas_per_sm = ctas_per_sm;
    g_batch_rows_per_thread = rows_per_thread;
    g_batch_vector_width = vector_width;
    return PLCG_OK;
}

extern "C" plcg_status plcg_set_batched_schedule(int gang_size, double large_work_factor,
                                                 double max_gang_fraction)
{
    if (gang_size == 0) {
        g_batch_G = 8;
        g_batch_beta = 1.0;
        g_batch_gang_frac = 0.5;
        return PLCG_OK;
    }
    if (gang_size < 1 || gang_size > 64 || !(large_work_factor > 0.0) ||
        !(max_gang_fraction >= 0.0 && max_gang_fraction <= 1.0))
        return fail(PLCG_ERR_INVALID, "bad batched schedule");
    g_batch_G = gang_size;
    g_batch_beta = large_work_factor;
    g_batch_gang_frac = max_gang_fraction;
    return PLCG_OK;
}

// Estimated solve work of a stencil system: n * sqrt(kappa), with kappa from
// the closed-form extreme eigenvalues of the constant-coefficient Dirichlet
// stencil (a Kronecker sum: center + 2 off cos(j pi / (n_d + 1)) per axis).
static double stencil_work(const plcg_matrix *M)
{
    const double pi = 3.14159265358979323846;
    const int dims[3] = {M->st.nx, M->st.ny, M->st.nz};
    double s = 0.0;
    for (int d = 0; d < M->st.dim; ++d) s += 2.0 * std::fabs(M->st.off) * std::cos(pi / (dims[d] + 1.0));
    const double lmin = std::max(M->st.center - s, 1e-300), lmax = M->st.center + s;
    return (double)M->n * std::sqrt(std::max(1.0, lmax / lmin));
}

template <typename T>
static plcg_status run_batched(int count, plcg_matrix *const *A, const double *const *b,
                               double *const *x, const double *lmin, const double *lmax,
                               const plcg_params *prm, plcg_result *results)
{
    const bool f32 = sizeof(T) == 4;
    const bool cg = prm->method == PLCG_METHOD_CG;
    const int l = cg ? 1 : prm->l;
    // the tuned launch shape applies to FP32 solves; FP64 uses the defaults
    const void *func = f32 ? batched_kernel_ptr(f32, l, cg, g_batch_ctas_per_sm, g_batch_rows_per_thread,
                                                g_batch_vector_width)
                           : batched_kernel_ptr(f32, l, cg);
    if (!func) return fail(PLCG_ERR_UNIMPL, "plcg_solve_batched: l must be 1..4");
    cudaStream_t stream = A[0]->stream;
    int dev = A[0]->device;
    if (dev < 0 || dev >= 64) return fail(PLCG_ERR_INVALID, "device ordinal too large");
    BatchCtx &ctx = g_batch[dev];
    std::lock_guard<std::mutex> lock(ctx.mu);

    // host descriptors and work estimates
    std::vector<BatchSys> sys(count);
    std::vector<double> work(count);
    double wsum = 0.0;
    for (int i = 0; i < count; ++i) {
        const plcg_matrix *M = A[i];
        BatchSys &y = sys[i];
        y.dim = M->st.dim;
        y.nx = M->st.nx;
        y.ny = M->st.ny;
        y.nz = M->st.nz;
        y.dnx = M->st.dnx;
        y.dny = M->st.dny;
        y.center = M->st.center;
        y.off = M->st.off;
        y.b = b[i];
        y.x = x[i];
        y.out = nullptr;
        std::memset(y.sigma, 0, sizeof(y.sigma));
        if (!cg) {
            const double lo = lmin ? lmin[i] : prm->lmin, hi = lmax ? lmax[i] : prm->lmax;
            if (!prm->shifts && (!std::isfinite(lo) || !std::isfinite(hi) || hi < lo))
                return fail(PLCG_ERR_INVALID, "system %d: need lmin <= lmax", i);
            resolve_shifts(M, prm, lo, hi, y.sigma);
        }
        work[i] = stencil_work(M);
        wsum += work[i];
    }

    // ring layout (as for a single solve)
    SolveArgs<T> proto;
    std::memset(&proto, 0, sizeof(proto));
    int nvec = 0;
    if (!cg) {
        for (int k = 0; k <= l; ++k) {
            int d = 3;
            if (k == l) d = std::max(3, l);
            if (k == 0 && prm->dots_2l1) d = std::max(3, l + 1);
            proto.depth[k] = d;
            proto.ddiv[k] = make_fastdiv((uint32_t)d);
            proto.base[k] = nvec;
            nvec += d;
        }
    } else {
        nvec = 3;
    }
    proto.method = cg ? 1 : 0;
    proto.l = l;
    proto.rtol = prm->rtol;
    proto.maxit = prm->maxit;
    proto.dots_2l1 = prm->dots_2l1 ? 1 : 0;
    proto.max_restarts = prm->max_restarts;
    proto.inner_floor = prm->inner_rtol_floor;
    proto.fp32 = f32 ? 1 : 0;
    proto.poll_limit = poll_limit();
    proto.lookahead = (!cg && l >= 2) ? 1 : 0;

    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, kBlock, 0));
    if (per_sm < 1) return fail(PLCG_ERR_CUDA, "batched kernel cannot be resident");
    const int Pmax = per_sm * A[0]->num_sms;

    // schedule: systems whose work exceeds beta * (fair share of one CTA of a
    // full launch) go to gangs; the launch then has the gangs' CTAs plus at
    // most one CTA per remaining system
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return work[p] > work[q]; });
    const int G = std::max(1, std::min(g_batch_G, Pmax));
    const double share = wsum / std::min<int64_t>((int64_t)count * G, Pmax);
    std::vector<int> large, small;
    for (int k = 0; k < count; ++k)
        (G > 1 && work[order[k]] > g_batch_beta * share ? large : small).push_back(order[k]);
    int ngangs = std::min<int>((int)large.size(), (int)(g_batch_gang_frac * Pmax) / G);
    if (ngangs == 0) {
        small.insert(small.begin(), large.begin(), large.end());
        large.clear();
    }
    const int P = (int)std::max<int64_t>(1, std::min<int64_t>(Pmax, (int64_t)ngangs * G + (int64_t)small.size()));
    int64_t nmax_s = 1, nmax_l = 1;
    for (int i : small) nmax_s = std::max<int64_t>(nmax_s, A[i]->n);
    for (int i : large) nmax_l = std::max<int64_t>(nmax_l, A[i]->n);
    const size_t ws_stride =
        align_up(align_up((size_t)(nvec + 2) * nmax_s * sizeof(T), 256) + (size_t)nmax_s * sizeof(double), 256);
    const size_t gws_stride = ngangs ?
        align_up(align_up((size_t)(nvec + 2) * nmax_l * sizeof(T), 256) + (size_t)nmax_l * sizeof(double), 256) : 0;
    size_t off = 0;
    const size_t o_sys = off; off += align_up(sizeof(BatchSys) * count, 256);
    const size_t o_ordl = off; off += align_up(sizeof(int) * std::max<size_t>(1, large.size()), 256);
    const size_t o_ords = off; off += align_up(sizeof(int) * std::max<size_t>(1, small.size()), 256);
    const size_t o_res = off; off += align_up(sizeof(DevResult) * count, 256);
    const size_t o_ctr = off; off += 256;
    const size_t o_gbar = off; off += align_up(sizeof(unsigned) * 32 * std::max(1, ngangs), 256);
    const size_t o_gab = off; off += align_up(sizeof(int) * std::max(1, ngangs), 256);
    const size_t o_gslot = off; off += align_up(sizeof(int) * std::max(1, ngangs), 256);
    const size_t o_gpart = off; off += align_up(sizeof(double) * (kMaxL + 1) * G * kMaxDots * std::max(1, ngangs), 256);
    const size_t o_gnpart = off; off += align_up(sizeof(double) * G * kNormSlots * std::max(1, ngangs), 256);
    const size_t o_gws = off; off += gws_stride * ngangs;
    const size_t o_ws = off; off += ws_stride * P;
    if (ctx.bytes < off) {
        if (ctx.mem) { cudaStreamSynchronize(stream); cudaFree(ctx.mem); ctx.mem = nullptr; ctx.bytes = 0; }
        CUDA_TRY(cudaMalloc(&ctx.mem, off));
        ctx.bytes = off;
    }
    if (!ctx.ev0) {
        CUDA_TRY(cudaEventCreate(&ctx.ev0));
        CUDA_TRY(cudaEventCreate(&ctx.ev1));
    }
    DevResult *dres = reinterpret_cast<DevResult *>(ctx.mem + o_res);
    for (int i = 0; i < count; ++i) sys[i].out = dres + i;
    CUDA_TRY(cudaMemcpyAsync(ctx.mem + o_sys, sys.data(), sizeof(BatchSys) * count,
                             cudaMemcpyHostToDevice, stream));
    if (!large.empty())
        CUDA_TRY(cudaMemcpyAsync(ctx.mem + o_ordl, large.data(), sizeof(int) * large.size(),
                                 cudaMemcpyHostToDevice, stream));
    if (!small.empty())
        CUDA_TRY(cudaMemcpyAsync(ctx.mem + o_ords, small.data(), sizeof(int) * small.size(),
                                 cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaMemsetAsync(ctx.mem + o_res, 0, sizeof(DevResult) * count, stream));
    CUDA_TRY(cudaMemsetAsync(ctx.mem + o_ctr, 0, 256, stream));
    CUDA_TRY(cudaMemsetAsync(ctx.mem + o_gbar, 0, o_gpart - o_gbar, stream));   // barriers, aborts, slots
    BatchArgs<T> ba;
    std::memset(&ba, 0, sizeof(ba));
    ba.sys = reinterpret_cast<const BatchSys *>(ctx.mem + o_sys);
    ba.nlarge = ngangs ? (int)large.size() : 0;
    ba.nsmall = (int)small.size();
    ba.order_large = reinterpret_cast<const int *>(ctx.mem + o_ordl);
    ba.order_small = reinterpret_cast<const int *>(ctx.mem + o_ords);
    ba.ctr_large = reinterpret_cast<int *>(ctx.mem + o_ctr);
    ba.ctr_small = reinterpret_cast<int *>(ctx.mem + o_ctr + 128);
    ba.ngangs = ngangs;
    ba.G = G;
    ba.gbar = reinterpret_cast<unsigned *>(ctx.mem + o_gbar);
    ba.gabort = reinterpret_cast<int *>(ctx.mem + o_gab);
    ba.gslot = reinterpret_cast<int *>(ctx.mem + o_gslot);
    ba.gpart = reinterpret_cast<double *>(ctx.mem + o_gpart);
    ba.gnpart = reinterpret_cast<double *>(ctx.mem + o_gnpart);
    ba.gws = ctx.mem + o_gws;
    ba.gws_stride = gws_stride;
    ba.ws = ctx.mem + o_ws;
    ba.ws_stride = ws_stride;
    ba.t0 = reinterpret_cast<unsigned long long *>(ctx.mem + o_ctr + 192);
    ba.proto = proto;
    void *args[] = {&ba};
    CUDA_TRY(cudaEventRecord(ctx.ev0, stream));
    CUDA_TRY(cudaLaunchCooperativeKernel(func, dim3(P), dim3(kBlock), args, 0, stream));
    CUDA_TRY(cudaEventRecord(ctx.ev1, stream));
    std::vector<DevResult> hres(count);
    unsigned long long t0 = 0;
    CUDA_TRY(cudaMemcpyAsync(hres.data(), dres, sizeof(DevResult) * count, cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaMemcpyAsync(&t0, ba.t0, sizeof(t0), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, ctx.ev0, ctx.ev1));
    plcg_status first = PLCG_OK;
    for (int i = 0; i < count; ++i) {
        const DevResult &o = hres[i];
        if (results) {
            results[i].status = o.status;
            results[i].iters = o.iters;
            results[i].spmvs = o.spmvs;
            results[i].restarts = o.restarts;
            results[i].refinements = o.refinements;
            results[i].recursive_relres = o.recursive_relres;
            results[i].true_relres = o.true_relres;
            results[i].seconds = ms * 1e-3;
            // from the launch's start to this system's result (device timer)
            results[i].latency = o.t_end_ns >= t0 ? (double)(o.t_end_ns - t0) * 1e-9 : 0.0;
        }
        if (first == PLCG_OK && o.status != PLCG_OK) first = (plcg_status)o.status;
    }
    if (first != PLCG_OK) return fail(first, "at least one system of the batch did not converge");
    return PLCG_OK;
}

extern "C" plcg_status plcg_solve_batched(int count, plcg_matrix *const *A, const double *const *b,
                                          double *const *x, const double *lmin, const double *lmax,
                                          const plcg_params *prm, plcg_result *results)
{
    if (count < 0) return fail(PLCG_ERR_INVALID, "plcg_solve_batched: count < 0");
    if (count == 0) return PLCG_OK;
    if (!A || !b || !x || !prm) return fail(PLCG_ERR_INVALID, "plcg_solve_batched: NULL argument");
    for (int i = 0; i < count; ++i) {
        if (!A[i] || !b[i] || !x[i]) return fail(PLCG_ERR_INVALID, "system %d: NULL argument", i);
        if ((reinterpret_cast<uintptr_t>(b[i]) | reinterpret_cast<uintptr_t>(x[i])) & 15)
            return fail(PLCG_ERR_INVALID, "system %d: b and x must be 16-byte aligned", i);
        if (A[i]->kind != kOpStencil)
            return fail(PLCG_ERR_UNIMPL, "plcg_solve_batched: system %d is not a stencil operator", i);
        if (A[i]->device != A[0]->device)
            return fail(PLCG_ERR_INVALID, "plcg_solve_batched: systems on different devices");
        if (prm && prm->precond == PLCG_PRECOND_JACOBI && !(A[i]->st.center > 0.0))
            return fail(PLCG_ERR_INVALID, "system %d: Jacobi needs a positive stencil center", i);
    }
    plcg_status st = check_params(A[0], prm);
    if (st != PLCG_OK) return st;
    if (prm->method == PLCG_METHOD_PLCG && prm->l > 4)
        return fail(PLCG_ERR_UNIMPL, "plcg_solve_batched: l must be 1..4");
    if (prm->method == PLCG_METHOD_PLCG && prm->dots_2l1)
        return fail(PLCG_ERR_UNIMPL, "plcg_solve_batched computes the l+1 dot products only (dots_2l1 = 0)");
    CUDA_TRY(cudaSetDevice(A[0]->device));
    if (prm->prec == PLCG_FP64) return run_batched<double>(count, A, b, x, lmin, lmax, prm, results);
    return run_batched<float>(count, A, b, x, lmin, lmax, prm, results);
}

// ------------------------------------------------------------------ serving
// Continuous batching of solves: a scheduler thread admits submitted requests
// in FIFO order whenever their workspace fits the device-memory budget, a
// stream slot is free and their CTAs fit next to the in-flight solves (so
// every cooperative grid can be resident at once and its grid barriers always
// complete); a request that does not fit yet lets later ones that do fit
// pass it for a bounded time (backfilling).  Each admitted request runs as its own persistent launch on its
// own stream; its grid size depends only on the request (its n, kernel and
// the per-request cap), so a request gives the same bits alone or in a mix.
namespace {

struct ServerReq {
    uint64_t ticket = 0;
    plcg_matrix *A = nullptr;
    const double *b = nullptr;
    double *x = nullptr;
    plcg_params prm{};
    double shifts[kMaxL] = {0};
    double sigma[kMaxL] = {0};
    size_t bytes = 0;
    int64_t P = 0;
    double sm_share = 0.0;    // SMs its CTAs occupy: P / (resident CTAs per SM)
    int slot = -1;
    bool done = false;
    plcg_result res{};
    std::chrono::steady_clock::time_point t_submit;
};

}  // namespace

// Admission, request by request in FIFO order (while a stream slot is
// free): a request starts when its workspace fits the remaining budget and
// its CTAs fit next to the running solves (sm_used: SMs their CTAs occupy;
// the first request always fits, its grid being capped at the GPU's
// resident CTAs).  One that does not fit yet is passed by later requests
// that do (backfilling) until it has waited kServerBackfillWindow; then
// admission stops at it, so that a stream of small requests cannot keep it
// out.
constexpr double kServerBackfillWindow = 0.1;   // seconds
enum { kAdmitStart = 0, kAdmitSkip = 1, kAdmitStop = 2 };
static int admit_decision(size_t bytes, double share, double waited_s, size_t mem_free, double sm_used,
                          int num_sms)
{
    const bool fits = bytes <= mem_free && !(sm_used > 0.0 && sm_used + share > num_sms + 1e-9);
    if (fits) return kAdmitStart;
    return waited_s >= kServerBackfillWindow ? kAdmitStop : kAdmitSkip;
}

// Test hook: the admission pass over a queue of n requests (workspace
// bytes[i], SM share[i], waited_s[i] seconds in the queue) given the free
// budget, the SMs in use, the SM count and the free stream slots.  Writes the
// indices of the admitted requests, in admission order, to admitted[] and
// returns their count.
extern "C" int plcg_debug_server_admission(int n, const uint64_t *bytes, const double *share,
                                           const double *waited_s, uint64_t mem_free, double sm_used,
                                           int num_sms, int free_slots, int *admitted)
{
    int k = 0;
    for (int i = 0; i < n && free_slots > 0; ++i) {
        const int d = admit_decision((size_t)bytes[i], share[i], waited_s[i], (size_t)mem_free, sm_used, num_sms);
        if (d == kAdmitStop) break;
        if (d == kAdmitSkip) continue;
        admitted[k++] = i;
        mem_free -= bytes[i];
        sm_used += share[i];
        --free_slots;
    }
    return k;
}

struct plcg_server {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0, used = 0;
    double sm_used = 0.0;
    int max_inflight = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev0, ev1, ev2;   // kernel start, kernel end, result copied
    std::vector<DevResult *> hres;   // pinned, one per slot
    std::vector<int> free_slots;
    std::deque<std::shared_ptr<ServerReq>> queue;
    std::vector<std::shared_ptr<ServerReq>> inflight;
    std::unordered_map<uint64_t, std::shared_ptr<ServerReq>> tickets;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
};

template <typename T>
static plcg_status server_launch(plcg_server *S, ServerReq &q)
{
    const cudaStream_t st = S->streams[q.slot];
    void *ws = nullptr;
    CUDA_TRY(cudaMallocAsync(&ws, q.bytes, st));
    SolveArgs<T> a;
    const void *func = nullptr;
    int64_t P = 0;
    int per_sm = 0;
    size_t bytes = 0, o_out = 0;
    plcg_status s = build_solve<T>(q.A, q.b, q.x, &q.prm, q.sigma, (int)q.P, static_cast<char *>(ws),
                                   &a, &func, &P, &per_sm, &bytes, &o_out);
    if (s == PLCG_OK) {
        CUDA_TRY(cudaEventRecord(S->ev0[q.slot], st));
        s = launch_built<T>(a, func, P, st);
    }
    if (s == PLCG_OK) {
        CUDA_TRY(cudaEventRecord(S->ev1[q.slot], st));
        CUDA_TRY(cudaMemcpyAsync(S->hres[q.slot], a.out, sizeof(DevResult), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaEventRecord(S->ev2[q.slot], st));
    }
    cudaFreeAsync(ws, st);   // stream-ordered: returned once the solve and the copy are done
    return s;
}

static void server_finish(plcg_server *S, const std::shared_ptr<ServerReq> &q, plcg_status launch_st)
{
    if (launch_st == PLCG_OK) {
        const DevResult &o = *S->hres[q->slot];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, S->ev0[q->slot], S->ev1[q->slot]);
        q->res.status = o.status;
        q->res.iters = o.iters;
        q->res.spmvs = o.spmvs;
        q->res.restarts = o.restarts;
        q->res.refinements = o.refinements;
        q->res.recursive_relres = o.recursive_relres;
        q->res.true_relres = o.true_relres;
        q->res.seconds = ms * 1e-3;
    } else {
        q->res.status = launch_st;
    }
    q->res.latency =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - q->t_submit).count();
    S->used -= q->bytes;
    S->sm_used -= q->sm_share;
    S->free_slots.push_back(q->slot);
    q->done = true;
}

static void server_loop(plcg_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progress = false;
        const auto now = std::chrono::steady_clock::now();
        for (auto it = S->queue.begin(); it != S->queue.end() && !S->free_slots.empty();) {
            auto q = *it;
            const int d = admit_decision(q->bytes, q->sm_share,
                                         std::chrono::duration<double>(now - q->t_submit).count(),
                                         S->budget - S->used, S->sm_used, S->num_sms);
            if (d == kAdmitStop) break;
            if (d == kAdmitSkip) {
                ++it;
                continue;
            }
            it = S->queue.erase(it);
            q->slot = S->free_slots.back();
            S->free_slots.pop_back();
            S->used += q->bytes;
            S->sm_used += q->sm_share;
            const plcg_status st = (q->prm.prec != PLCG_FP32_FP64DOT) ? server_launch<double>(S, *q)
                                                              : server_launch<float>(S, *q);
            if (st != PLCG_OK) {
                server_finish(S, q, st);
                S->cv_done.notify_all();
            } else {
                S->inflight.push_back(q);
            }
            progress = true;
        }
        // completions
        for (size_t k = 0; k < S->inflight.size();) {
            auto &q = S->inflight[k];
            if (cudaEventQuery(S->ev2[q->slot]) == cudaSuccess) {
                server_finish(S, q, PLCG_OK);
                S->inflight[k] = S->inflight.back();
                S->inflight.pop_back();
                progress = true;
                S->cv_done.notify_all();
            } else {
                ++k;
            }
        }
        if (S->stop && S->queue.empty() && S->inflight.empty()) break;
        if (!progress) S->cv_sched.wait_for(lk, std::chrono::microseconds(20));
    }
}

extern "C" plcg_status plcg_server_create(size_t mem_budget_bytes, int max_inflight, plcg_server **out)
{
    if (!out) return fail(PLCG_ERR_INVALID, "plcg_server_create: NULL out");
    *out = nullptr;
    if (max_inflight < 0 || max_inflight > 256)
        return fail(PLCG_ERR_INVALID, "max_inflight must be in 0..256");
    plcg_server *S = new plcg_server();
    CUDA_TRY(cudaGetDevice(&S->device));
    CUDA_TRY(cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, S->device));
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    S->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(0.8 * (double)free_b);
    S->max_inflight = max_inflight ? max_inflight : 32;
    // keep freed stream-ordered memory cached in the pool for the next request
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    for (int k = 0; k < S->max_inflight; ++k) {
        cudaStream_t st;
        cudaEvent_t e0, e1, e2;
        DevResult *h = nullptr;
        CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreate(&e0));
        CUDA_TRY(cudaEventCreate(&e1));
        CUDA_TRY(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
        CUDA_TRY(cudaMallocHost(&h, sizeof(DevResult)));
        S->streams.push_back(st);
        S->ev0.push_back(e0);
        S->ev1.push_back(e1);
        S->ev2.push_back(e2);
        S->hres.push_back(h);
        S->free_slots.push_back(S->max_inflight - 1 - k);
    }
    S->th = std::thread(server_loop, S);
    *out = S;
    return PLCG_OK;
}

extern "C" plcg_status plcg_submit(plcg_server *S, plcg_matrix *A, const double *b, double *x,
                                   const plcg_params *prm, uint64_t *ticket)
{
    if (!S || !A || !b || !x || !ticket) return fail(PLCG_ERR_INVALID, "plcg_submit: NULL argument");
    plcg_status st = check_params(A, prm);
    if (st != PLCG_OK) return st;
    if ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15)
        return fail(PLCG_ERR_INVALID, "b and x must be 16-byte aligned");
    if (A->device != S->device) return fail(PLCG_ERR_INVALID, "matrix and server on different devices");
    auto q = std::make_shared<ServerReq>();
    q->A = A;
    q->b = b;
    q->x = x;
    q->prm = *prm;
    if (prm->method == PLCG_METHOD_PLCG) {
        if (prm->shifts) {
            std::memcpy(q->shifts, prm->shifts, prm->l * sizeof(double));
            q->prm.shifts = q->shifts;
        }
        resolve_shifts(A, &q->prm, prm->lmin, prm->lmax, q->sigma);
    }
    // per-request grid cap: at most half of the GPU's resident CTAs, so large
    // requests never lock small ones out
    const void *func = nullptr;
    int64_t P = 0;
    int per_sm = 0;
    size_t bytes = 0, o_out = 0;
    if (prm->prec != PLCG_FP32_FP64DOT) {
        SolveArgs<double> a;
        st = build_solve<double>(A, b, x, &q->prm, q->sigma, 0, nullptr, &a, &func, &P, &per_sm, &bytes, &o_out);
    } else {
        SolveArgs<float> a;
        st = build_solve<float>(A, b, x, &q->prm, q->sigma, 0, nullptr, &a, &func, &P, &per_sm, &bytes, &o_out);
    }
    if (st != PLCG_OK) return st;
    const int cap = std::max(1, (per_sm * S->num_sms) / 2);
    q->P = std::min<int64_t>(P, cap);
    q->sm_share = (double)q->P / per_sm;
    // recompute the byte count for the capped grid (partials scale with P)
    if (prm->prec != PLCG_FP32_FP64DOT) {
        SolveArgs<double> a;
        st = build_solve<double>(A, b, x, &q->prm, q->sigma, (int)q->P, nullptr, &a, &func, &P, &per_sm, &bytes, &o_out);
    } else {
        SolveArgs<float> a;
        st = build_solve<float>(A, b, x, &q->prm, q->sigma, (int)q->P, nullptr, &a, &func, &P, &per_sm, &bytes, &o_out);
    }
    if (st != PLCG_OK) return st;
    q->bytes = bytes;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(PLCG_ERR_INVALID, "server is shutting down");
    if (bytes > S->budget)
        return fail(PLCG_ERR_NOMEM, "request needs %zu bytes of workspace; the budget is %zu", bytes, S->budget);
    q->ticket = S->next_ticket++;
    q->t_submit = std::chrono::steady_clock::now();
    S->queue.push_back(q);
    S->tickets[q->ticket] = q;
    *ticket = q->ticket;
    S->cv_sched.notify_one();
    return PLCG_OK;
}

static plcg_status collect(plcg_server *S, uint64_t ticket, plcg_result *res, bool wait)
{
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail(PLCG_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    auto q = it->second;
    if (!q->done) {
        if (!wait) return PLCG_PENDING;
        S->cv_done.wait(lk, [&] { return q->done; });
    }
    if (res) *res = q->res;
    S->tickets.erase(it);
    if (q->res.status != PLCG_OK) return fail((plcg_status)q->res.status, "request %llu ended with status %d",
                                              (unsigned long long)ticket, q->res.status);
    return PLCG_OK;
}

extern "C" plcg_status plcg_poll(plcg_server *S, uint64_t ticket, plcg_result *res)
{
    if (!S) return fail(PLCG_ERR_INVALID, "plcg_poll: NULL server");
    return collect(S, ticket, res, false);
}

extern "C" plcg_status plcg_wait(plcg_server *S, uint64_t ticket, plcg_result *res)
{
    if (!S) return fail(PLCG_ERR_INVALID, "plcg_wait: NULL server");
    return collect(S, ticket, res, true);
}

extern "C" void plcg_server_destroy(plcg_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_sched.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    for (size_t k = 0; k < S->streams.size(); ++k) {
        cudaStreamSynchronize(S->streams[k]);
        cudaStreamDestroy(S->streams[k]);
        cudaEventDestroy(S->ev0[k]);
        cudaEventDestroy(S->ev1[k]);
        cudaEventDestroy(S->ev2[k]);
        cudaFreeHost(S->hres[k]);
    }
    delete S;
}
