// kern_f64_v27j.cu -- instantiations of the persistent solvers for T = double,
// VEC = 1, operator kOpVar27Jacobi (the structured 27-point operator with M = diag(A)); one translation unit per combination so that
// the build compiles them in parallel.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *kptr_f64_v27j(int l, bool cg, bool sc)
{
    if (cg) return reinterpret_cast<const void *>(&cg_kernel<double, 1, kOpVar27Jacobi>);
    switch (l) {
    case 1:   // sc: the scaled-basis variant (large systems)
        return sc ? reinterpret_cast<const void *>(&plcg_kernel<double, 1, 1, kOpVar27Jacobi, true>)
                  : reinterpret_cast<const void *>(&plcg_kernel<double, 1, 1, kOpVar27Jacobi>);
    case 2: return reinterpret_cast<const void *>(&plcg_kernel<double, 2, 1, kOpVar27Jacobi>);
    case 3: return reinterpret_cast<const void *>(&plcg_kernel<double, 3, 1, kOpVar27Jacobi>);
    case 4: return reinterpret_cast<const void *>(&plcg_kernel<double, 4, 1, kOpVar27Jacobi>);
    case 5: return reinterpret_cast<const void *>(&plcg_kernel<double, 5, 1, kOpVar27Jacobi>);
    case 6: return reinterpret_cast<const void *>(&plcg_kernel<double, 6, 1, kOpVar27Jacobi>);
    case 7: return reinterpret_cast<const void *>(&plcg_kernel<double, 7, 1, kOpVar27Jacobi>);
    case 8: return reinterpret_cast<const void *>(&plcg_kernel<double, 8, 1, kOpVar27Jacobi>);
    default: return nullptr;
    }
}

}  // namespace plcg
