// kern_f32_v27.cu -- instantiations of the persistent solvers for T = float,
// VEC = 1, operator kOpVar27 (the structured 27-point operator); one translation unit per combination so that
// the build compiles them in parallel.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *kptr_f32_v27(int l, bool cg)
{
    if (cg) return reinterpret_cast<const void *>(&cg_kernel<float, 1, kOpVar27>);
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&plcg_kernel<float, 1, 1, kOpVar27>);
    case 2: return reinterpret_cast<const void *>(&plcg_kernel<float, 2, 1, kOpVar27>);
    case 3: return reinterpret_cast<const void *>(&plcg_kernel<float, 3, 1, kOpVar27>);
    case 4: return reinterpret_cast<const void *>(&plcg_kernel<float, 4, 1, kOpVar27>);
    case 5: return reinterpret_cast<const void *>(&plcg_kernel<float, 5, 1, kOpVar27>);
    case 6: return reinterpret_cast<const void *>(&plcg_kernel<float, 6, 1, kOpVar27>);
    case 7: return reinterpret_cast<const void *>(&plcg_kernel<float, 7, 1, kOpVar27>);
    case 8: return reinterpret_cast<const void *>(&plcg_kernel<float, 8, 1, kOpVar27>);
    default: return nullptr;
    }
}

}  // namespace plcg
