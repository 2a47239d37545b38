// kern_batched_f32.cu -- instantiations of the batched kernel for T = float:
// p(l)-CG for l = 1..4 and classic CG (one translation unit per vector type
// so that the build compiles them in parallel).
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *batched_kernel_ptr_f32(int l, bool cg)
{
    if (cg) return reinterpret_cast<const void *>(&batched_kernel<float, 1, true>);
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&batched_kernel<float, 1, false>);
    case 2: return reinterpret_cast<const void *>(&batched_kernel<float, 2, false>);
    case 3: return reinterpret_cast<const void *>(&batched_kernel<float, 3, false>);
    case 4: return reinterpret_cast<const void *>(&batched_kernel<float, 4, false>);
    default: return nullptr;
    }
}

}  // namespace plcg
