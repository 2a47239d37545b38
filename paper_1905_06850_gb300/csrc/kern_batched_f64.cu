// kern_batched_f64.cu -- instantiations of the batched kernel for T = double:
// p(l)-CG for l = 1..4 and classic CG (one translation unit per vector type
// so that the build compiles them in parallel).
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *batched_kernel_ptr_f64(int l, bool cg)
{
    if (cg) return reinterpret_cast<const void *>(&batched_kernel<double, 1, true>);
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&batched_kernel<double, 1, false>);
    case 2: return reinterpret_cast<const void *>(&batched_kernel<double, 2, false>);
    case 3: return reinterpret_cast<const void *>(&batched_kernel<double, 3, false>);
    case 4: return reinterpret_cast<const void *>(&batched_kernel<double, 4, false>);
    default: return nullptr;
    }
}

}  // namespace plcg
