// kern_f64_stsc.cu -- instantiations of the scaled-basis FP64 p(l)-CG solver
// for the stencil operators, l = 2..5 (VEC = 2 and 1; l = 1 is in
// kern_f64_st2.cu / kern_f64_st1.cu), in a translation unit of their own so
// that the build compiles them in parallel.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

template <int VEC>
static const void *stsc(int l)
{
    switch (l) {
    case 2: return reinterpret_cast<const void *>(&plcg_kernel<double, 2, VEC, kOpStencil, true>);
    case 3: return reinterpret_cast<const void *>(&plcg_kernel<double, 3, VEC, kOpStencil, true>);
    case 4: return reinterpret_cast<const void *>(&plcg_kernel<double, 4, VEC, kOpStencil, true>);
    case 5: return reinterpret_cast<const void *>(&plcg_kernel<double, 5, VEC, kOpStencil, true>);
    default: return nullptr;
    }
}

const void *kptr_f64_stsc(int vec, int l) { return vec == 2 ? stsc<2>(l) : stsc<1>(l); }

}  // namespace plcg
