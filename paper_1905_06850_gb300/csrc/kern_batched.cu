// kern_batched.cu -- instantiations of the batched (one system per CTA)
// kernel for l = 1..4, FP64 and FP32 vectors.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *batched_kernel_ptr(bool f32, int l)
{
    if (f32) {
        switch (l) {
        case 1: return reinterpret_cast<const void *>(&batched_kernel<float, 1>);
        case 2: return reinterpret_cast<const void *>(&batched_kernel<float, 2>);
        case 3: return reinterpret_cast<const void *>(&batched_kernel<float, 3>);
        case 4: return reinterpret_cast<const void *>(&batched_kernel<float, 4>);
        default: return nullptr;
        }
    }
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&batched_kernel<double, 1>);
    case 2: return reinterpret_cast<const void *>(&batched_kernel<double, 2>);
    case 3: return reinterpret_cast<const void *>(&batched_kernel<double, 3>);
    case 4: return reinterpret_cast<const void *>(&batched_kernel<double, 4>);
    default: return nullptr;
    }
}

}  // namespace plcg
