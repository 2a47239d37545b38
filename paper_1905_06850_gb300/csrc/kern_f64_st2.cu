// kern_f64_st2.cu -- instantiations of the persistent solvers for T = double,
// VEC = 2, operator kOpStencil (one translation unit per combination so that the
// build compiles them in parallel).
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *kptr_f64_st2(int l, bool cg, bool sc)
{
    if (cg) return reinterpret_cast<const void *>(&cg_kernel<double, 2, kOpStencil>);
    if (sc && l >= 2 && l <= 5) return kptr_f64_stsc(2, l);   // scaled bases, l = 2..5
    switch (l) {
    case 1:   // sc: the scaled-basis variant (large systems)
        return sc ? reinterpret_cast<const void *>(&plcg_kernel<double, 1, 2, kOpStencil, true>)
                  : reinterpret_cast<const void *>(&plcg_kernel<double, 1, 2, kOpStencil>);
    case 2: return reinterpret_cast<const void *>(&plcg_kernel<double, 2, 2, kOpStencil>);
    case 3: return reinterpret_cast<const void *>(&plcg_kernel<double, 3, 2, kOpStencil>);
    case 4: return reinterpret_cast<const void *>(&plcg_kernel<double, 4, 2, kOpStencil>);
    case 5: return reinterpret_cast<const void *>(&plcg_kernel<double, 5, 2, kOpStencil>);
    case 6: return reinterpret_cast<const void *>(&plcg_kernel<double, 6, 2, kOpStencil>);
    case 7: return reinterpret_cast<const void *>(&plcg_kernel<double, 7, 2, kOpStencil>);
    case 8: return reinterpret_cast<const void *>(&plcg_kernel<double, 8, 2, kOpStencil>);
    default: return nullptr;
    }
}

}  // namespace plcg
