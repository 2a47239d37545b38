// kern_m_v27.cu -- instantiations of the persistent solvers for the
// FP32-matrix path (FP64 vectors, dots and scalars; matrix values stored in
// FP32), VEC = 1, operator kOpVar27 (one translation unit per operator so that
// the build compiles them in parallel).
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

const void *kptr_m_v27(int l, bool cg, bool sc)
{
    if (cg) return reinterpret_cast<const void *>(&cg_kernel<double, 1, kOpVar27, float>);
    switch (l) {
    case 1:   // sc: the scaled-basis variant (large systems)
        return sc ? reinterpret_cast<const void *>(&plcg_kernel<double, 1, 1, kOpVar27, true, float>)
                  : reinterpret_cast<const void *>(&plcg_kernel<double, 1, 1, kOpVar27, false, float>);
    case 2: return reinterpret_cast<const void *>(&plcg_kernel<double, 2, 1, kOpVar27, false, float>);
    case 3: return reinterpret_cast<const void *>(&plcg_kernel<double, 3, 1, kOpVar27, false, float>);
    case 4: return reinterpret_cast<const void *>(&plcg_kernel<double, 4, 1, kOpVar27, false, float>);
    case 5: return reinterpret_cast<const void *>(&plcg_kernel<double, 5, 1, kOpVar27, false, float>);
    case 6: return reinterpret_cast<const void *>(&plcg_kernel<double, 6, 1, kOpVar27, false, float>);
    case 7: return reinterpret_cast<const void *>(&plcg_kernel<double, 7, 1, kOpVar27, false, float>);
    case 8: return reinterpret_cast<const void *>(&plcg_kernel<double, 8, 1, kOpVar27, false, float>);
    default: return nullptr;
    }
}

}  // namespace plcg
