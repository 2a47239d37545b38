// kern_f64_csrj.cu -- instantiations of the persistent solvers for T = double,
// VEC = 1, operator kOpCsrJacobi (CSR with M = diag(A)); one translation unit
// per combination so that the build compiles them in parallel.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *kptr_f64_csrj(int l, bool cg, bool sc)
{
    if (cg) return reinterpret_cast<const void *>(&cg_kernel<double, 1, kOpCsrJacobi>);
    switch (l) {
    case 1:   // sc: the scaled-basis variant (large systems)
        return sc ? reinterpret_cast<const void *>(&plcg_kernel<double, 1, 1, kOpCsrJacobi, true>)
                  : reinterpret_cast<const void *>(&plcg_kernel<double, 1, 1, kOpCsrJacobi>);
    case 2: return reinterpret_cast<const void *>(&plcg_kernel<double, 2, 1, kOpCsrJacobi>);
    case 3: return reinterpret_cast<const void *>(&plcg_kernel<double, 3, 1, kOpCsrJacobi>);
    case 4: return reinterpret_cast<const void *>(&plcg_kernel<double, 4, 1, kOpCsrJacobi>);
    case 5: return reinterpret_cast<const void *>(&plcg_kernel<double, 5, 1, kOpCsrJacobi>);
    case 6: return reinterpret_cast<const void *>(&plcg_kernel<double, 6, 1, kOpCsrJacobi>);
    case 7: return reinterpret_cast<const void *>(&plcg_kernel<double, 7, 1, kOpCsrJacobi>);
    case 8: return reinterpret_cast<const void *>(&plcg_kernel<double, 8, 1, kOpCsrJacobi>);
    default: return nullptr;
    }
}

}  // namespace plcg
