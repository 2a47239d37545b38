// kern_f32_st4.cu -- instantiations of the persistent solvers for T = float,
// VEC = 4, operator kOpStencil (one translation unit per combination so that the
// build compiles them in parallel).
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *kptr_f32_st4(int l, bool cg)
{
    if (cg) return reinterpret_cast<const void *>(&cg_kernel<float, 4, kOpStencil>);
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&plcg_kernel<float, 1, 4, kOpStencil>);
    case 2: return reinterpret_cast<const void *>(&plcg_kernel<float, 2, 4, kOpStencil>);
    case 3: return reinterpret_cast<const void *>(&plcg_kernel<float, 3, 4, kOpStencil>);
    case 4: return reinterpret_cast<const void *>(&plcg_kernel<float, 4, 4, kOpStencil>);
    case 5: return reinterpret_cast<const void *>(&plcg_kernel<float, 5, 4, kOpStencil>);
    case 6: return reinterpret_cast<const void *>(&plcg_kernel<float, 6, 4, kOpStencil>);
    case 7: return reinterpret_cast<const void *>(&plcg_kernel<float, 7, 4, kOpStencil>);
    case 8: return reinterpret_cast<const void *>(&plcg_kernel<float, 8, 4, kOpStencil>);
    default: return nullptr;
    }
}

}  // namespace plcg
