// kern_batched_f32v.cu -- instantiations of the batched kernel for T = float
// with 2-wide vector rows in the one-block path (4 CTAs per SM, one row
// group for systems with odd nx): p(l)-CG for l = 1..4 and classic CG.  The
// FP32 default shape of p(1)- and p(2)-CG.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *batched_kernel_ptr_f32_v(int l, bool cg)
{
    if (cg) return reinterpret_cast<const void *>(&batched_kernel<float, 1, true, 4, 1, 2>);
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&batched_kernel<float, 1, false, 4, 1, 2>);
    case 2: return reinterpret_cast<const void *>(&batched_kernel<float, 2, false, 4, 1, 2>);
    case 3: return reinterpret_cast<const void *>(&batched_kernel<float, 3, false, 4, 1, 2>);
    case 4: return reinterpret_cast<const void *>(&batched_kernel<float, 4, false, 4, 1, 2>);
    default: return nullptr;
    }
}

}  // namespace plcg
