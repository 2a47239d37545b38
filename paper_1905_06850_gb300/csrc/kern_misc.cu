// kern_misc.cu -- kernel dispatch and small helper kernels.
#include "plcg_internal.h"
#include "plcg_kernels.h"

namespace plcg {

const void *kernel_ptr(bool f32, int op, int vec, int l, bool cg, bool sc, bool c32)
{
    if (c32) {   // FP64 vectors, FP32 matrix values (stored-matrix operators only)
        if (f32) return nullptr;
        if (op == kOpCsr) return kptr_m_csr(l, cg, sc);
        if (op == kOpCsrJacobi) return kptr_m_csrj(l, cg, sc);
        if (op == kOpVar27) return kptr_m_v27(l, cg, sc);
        if (op == kOpVar27Jacobi) return kptr_m_v27j(l, cg, sc);
        return nullptr;
    }
    if (!f32) {
        if (op == kOpCsr) return kptr_f64_csr(l, cg, sc);
        if (op == kOpCsrJacobi) return kptr_f64_csrj(l, cg, sc);
        if (op == kOpVar27) return kptr_f64_v27(l, cg, sc);
        if (op == kOpVar27Jacobi) return kptr_f64_v27j(l, cg, sc);
        return vec == 2 ? kptr_f64_st2(l, cg, sc) : kptr_f64_st1(l, cg, sc);
    }
    if (op == kOpCsr) return kptr_f32_csr(l, cg);
    if (op == kOpCsrJacobi) return kptr_f32_csrj(l, cg);
    if (op == kOpVar27) return kptr_f32_v27(l, cg);
    if (op == kOpVar27Jacobi) return kptr_f32_v27j(l, cg);
    return vec == 4 ? kptr_f32_st4(l, cg) : kptr_f32_st1(l, cg);
}

const void *batched_kernel_ptr(bool f32, int l, bool cg, int ctas_per_sm, int rows_per_thread,
                               int vector_width)
{
    if (f32) return batched_kernel_ptr_f32(l, cg, ctas_per_sm, rows_per_thread, vector_width);
    return (ctas_per_sm == 0 && rows_per_thread == 0 && vector_width == 0) ? batched_kernel_ptr_f64(l, cg)
                                                                          : nullptr;
}

// v[i] uniform in [-1, 1): SplitMix64 (Steele, Lea, Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) of (seed + i).
__global__ void fill_random_kernel(double *v, int64_t n, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)i * 0x9e3779b97f4a7c15ull;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        v[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

cudaError_t launch_fill_random(double *v, int64_t n, uint64_t seed, cudaStream_t s)
{
    const int64_t blocks = (n + 255) / 256;
    fill_random_kernel<<<(unsigned)(blocks < 65535 ? (blocks > 0 ? blocks : 1) : 65535), 256, 0, s>>>(v, n, seed);
    return cudaGetLastError();
}

__global__ void round_to_f32_kernel(const double *src, float *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

cudaError_t launch_round_to_f32(const double *src, float *dst, int64_t n, cudaStream_t s)
{
    const int64_t blocks = (n + 255) / 256;
    round_to_f32_kernel<<<(unsigned)(blocks < 65535 ? (blocks > 0 ? blocks : 1) : 65535), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

// Jacobi preconditioner data of a CSR matrix (values of type V): d_r = the
// sum of row r's entries in column r (FP64, in row order), dinv64 = 1 / d_r,
// and copies of both in V.  *bad is set when some d_r is not positive.
template <typename V>
__global__ void jacobi_setup_kernel(const int64_t *rowptr, const int32_t *col, const V *val,
                                    int64_t n, double *dinv64, V *dinv, V *diag, int *bad)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e)
            if (col[e] == r) d += (double)val[e];
        if (!(d > 0.0) || !isfinite(d)) {
            atomicExch(bad, 1);
            d = 1.0;
        }
        const double di = 1.0 / d;
        dinv64[r] = di;
        dinv[r] = (V)di;
        diag[r] = (V)d;
    }
}

cudaError_t launch_jacobi_setup(bool f32, const int64_t *rowptr, const int32_t *col,
                                const void *val, int64_t n, double *dinv64, void *dinv,
                                void *diag, int *bad, cudaStream_t s)
{
    const int64_t blocks = (n + 255) / 256;
    const unsigned g = (unsigned)(blocks < 65535 ? (blocks > 0 ? blocks : 1) : 65535);
    if (f32)
        jacobi_setup_kernel<float><<<g, 256, 0, s>>>(rowptr, col, static_cast<const float *>(val), n,
                                                     dinv64, static_cast<float *>(dinv),
                                                     static_cast<float *>(diag), bad);
    else
        jacobi_setup_kernel<double><<<g, 256, 0, s>>>(rowptr, col, static_cast<const double *>(val), n,
                                                      dinv64, static_cast<double *>(dinv),
                                                      static_cast<double *>(diag), bad);
    return cudaGetLastError();
}

template <typename V>
__global__ void var27_jacobi_setup_kernel(const V *diag, int64_t n, double *dinv64, V *dinv, int *bad)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double d = (double)diag[r];
        if (!(d > 0.0) || !isfinite(d)) {
            atomicExch(bad, 1);
            d = 1.0;
        }
        const double di = 1.0 / d;
        dinv64[r] = di;
        dinv[r] = (V)di;
    }
}

cudaError_t launch_var27_jacobi_setup(bool f32, const void *coef, int64_t n, double *dinv64,
                                      void *dinv, int *bad, cudaStream_t s)
{
    const int64_t blocks = (n + 255) / 256;
    const unsigned g = (unsigned)(blocks < 65535 ? (blocks > 0 ? blocks : 1) : 65535);
    if (f32)
        var27_jacobi_setup_kernel<float><<<g, 256, 0, s>>>(static_cast<const float *>(coef), n, dinv64,
                                                           static_cast<float *>(dinv), bad);
    else
        var27_jacobi_setup_kernel<double><<<g, 256, 0, s>>>(static_cast<const double *>(coef), n, dinv64,
                                                            static_cast<double *>(dinv), bad);
    return cudaGetLastError();
}

// Zero the forward coefficient coef[1+k][c] of every cell c whose neighbour
// c + d_k lies outside the grid (such entries do not act: Dirichlet).
template <typename V>
__global__ void var27_zero_outside_kernel(V *val, int64_t cstride, StencilDesc st)
{
    const int64_t nx = st.nx, ny = st.ny, nz = st.nz, n = nx * ny * nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
        for (int k = 0; k < 13; ++k) {
            const int64_t xn = x + v27_dx(k), yn = y + v27_dy(k), zn = z + v27_dz(k);
            if (xn < 0 || xn >= nx || yn < 0 || yn >= ny || zn >= nz) val[(1 + k) * cstride + c] = V(0);
        }
    }
}

cudaError_t launch_var27_zero_outside(bool f32, void *val, int64_t cstride, const StencilDesc &st, cudaStream_t s)
{
    const int64_t n = (int64_t)st.nx * st.ny * st.nz;
    const int64_t blocks = (n + 255) / 256;
    const unsigned g = (unsigned)(blocks < 65535 ? (blocks > 0 ? blocks : 1) : 65535);
    if (f32)
        var27_zero_outside_kernel<float><<<g, 256, 0, s>>>(static_cast<float *>(val), cstride, st);
    else
        var27_zero_outside_kernel<double><<<g, 256, 0, s>>>(static_cast<double *>(val), cstride, st);
    return cudaGetLastError();
}


// ------------------------------------------------------------------ FP64 rate
// FP64 FMA throughput of the device: every thread runs 8 independent FMA
// chains (x <- x * a + c), enough in flight per warp to keep the FP64 units
// busy; the sums are stored so that no chain is dead code.
__global__ void __launch_bounds__(256) fp64_fma_rate_kernel(double *out, int reps, double a, double c)
{
    double r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = 1e-3 * (double)threadIdx.x + (double)k;
    for (int i = 0; i < reps; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = fma(r[k], a, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += r[k];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace plcg

extern "C" plcg_status plcg_measure_fp64_fma_rate(double *flops_per_s)
{
    using namespace plcg;
    if (!flops_per_s) return PLCG_ERR_INVALID;
    *flops_per_s = 0.0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_rate_kernel, 256, 0) != cudaSuccess) {
        set_last_error("plcg_measure_fp64_fma_rate: device query failed");
        return PLCG_ERR_CUDA;
    }
    const int blocks = sms * per_sm, reps = 1 << 14;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * 256 * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int t = 0; t < 4 && e == cudaSuccess; ++t) {   // the first launch warms up
        e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) {
            fp64_fma_rate_kernel<<<blocks, 256>>>(out, reps, 0.9999999, 1e-7);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && t > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess || !(best > 0.f)) {
        set_last_error(std::string("plcg_measure_fp64_fma_rate: ") + cudaGetErrorString(e));
        return PLCG_ERR_CUDA;
    }
    *flops_per_s = 2.0 * 8.0 * reps * (double)blocks * 256.0 / (best * 1e-3);
    return PLCG_OK;
}

