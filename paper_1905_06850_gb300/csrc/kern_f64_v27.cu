// kern_f64_v27.cu -- instantiations of the persistent solvers for T = double,
// VEC = 1, operator kOpVar27 (the structured 27-point operator); one translation unit per combination so that
// the build compiles them in parallel.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *kptr_f64_v27(int l, bool cg, bool sc)
{
    if (cg) return reinterpret_cast<const void *>(&cg_kernel<double, 1, kOpVar27>);
    switch (l) {
    case 1:   // sc: the scaled-basis variant (large systems)
        return sc ? reinterpret_cast<const void *>(&plcg_kernel<double, 1, 1, kOpVar27, true>)
                  : reinterpret_cast<const void *>(&plcg_kernel<double, 1, 1, kOpVar27>);
    case 2: return reinterpret_cast<const void *>(&plcg_kernel<double, 2, 1, kOpVar27>);
    case 3: return reinterpret_cast<const void *>(&plcg_kernel<double, 3, 1, kOpVar27>);
    case 4: return reinterpret_cast<const void *>(&plcg_kernel<double, 4, 1, kOpVar27>);
    case 5: return reinterpret_cast<const void *>(&plcg_kernel<double, 5, 1, kOpVar27>);
    case 6: return reinterpret_cast<const void *>(&plcg_kernel<double, 6, 1, kOpVar27>);
    case 7: return reinterpret_cast<const void *>(&plcg_kernel<double, 7, 1, kOpVar27>);
    case 8: return reinterpret_cast<const void *>(&plcg_kernel<double, 8, 1, kOpVar27>);
    default: return nullptr;
    }
}

}  // namespace plcg
