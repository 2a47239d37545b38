// kern_batched_f32b.cu -- instantiations of the batched kernel for T = float
// in the launch shapes with 3 CTAs per SM (registers for larger row-group
// counts): p(l)-CG for l = 1..4 and classic CG.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

template <int RPT>
static const void *batched_f32_shape3(int l, bool cg)
{
    if (cg) return reinterpret_cast<const void *>(&batched_kernel<float, 1, true, 3, RPT, 1>);
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&batched_kernel<float, 1, false, 3, RPT, 1>);
    case 2: return reinterpret_cast<const void *>(&batched_kernel<float, 2, false, 3, RPT, 1>);
    case 3: return reinterpret_cast<const void *>(&batched_kernel<float, 3, false, 3, RPT, 1>);
    case 4: return reinterpret_cast<const void *>(&batched_kernel<float, 4, false, 3, RPT, 1>);
    default: return nullptr;
    }
}

const void *batched_kernel_ptr_f32_3(int l, bool cg, int rows_per_thread)
{
    if (rows_per_thread == 1) return batched_f32_shape3<1>(l, cg);
    if (rows_per_thread == 2) return batched_f32_shape3<2>(l, cg);
    if (rows_per_thread == 4) return batched_f32_shape3<4>(l, cg);
    return nullptr;
}

}  // namespace plcg
