// kern_misc.cu -- kernel dispatch and small helper kernels.
#include "plcg_internal.h"
#include "plcg_kernels.h"

namespace plcg {

const void *kernel_ptr(bool f32, int op, int vec, int l, bool cg)
{
    if (!f32) {
        if (op == kOpCsr) return kptr_f64_csr(l, cg);
        return vec == 2 ? kptr_f64_st2(l, cg) : kptr_f64_st1(l, cg);
    }
    if (op == kOpCsr) return kptr_f32_csr(l, cg);
    return vec == 4 ? kptr_f32_st4(l, cg) : kptr_f32_st1(l, cg);
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

}  // namespace plcg
