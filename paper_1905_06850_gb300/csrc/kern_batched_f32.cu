// kern_batched_f32.cu -- instantiations of the batched kernel for T = float:
// p(l)-CG for l = 1..4 and classic CG, in the default launch shape and the
// shapes with 4 CTAs per SM and one row per thread (the 3-CTA shapes are in
// kern_batched_f32b.cu and the 2-wide vector rows, the default of p(1)- and
// p(2)-CG, in kern_batched_f32v.cu, so that the build compiles them in
// parallel).
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

template <int MINB, int RPT>
static const void *batched_f32_shape(int l, bool cg)
{
    if (cg) return reinterpret_cast<const void *>(&batched_kernel<float, 1, true, MINB, RPT, 1>);
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&batched_kernel<float, 1, false, MINB, RPT, 1>);
    case 2: return reinterpret_cast<const void *>(&batched_kernel<float, 2, false, MINB, RPT, 1>);
    case 3: return reinterpret_cast<const void *>(&batched_kernel<float, 3, false, MINB, RPT, 1>);
    case 4: return reinterpret_cast<const void *>(&batched_kernel<float, 4, false, MINB, RPT, 1>);
    default: return nullptr;
    }
}

const void *batched_kernel_ptr_f32(int l, bool cg, int ctas_per_sm, int rows_per_thread, int vector_width)
{
    if (ctas_per_sm == 0 && rows_per_thread == 0 && vector_width == 0) {   // each method's default
        if (cg) return reinterpret_cast<const void *>(&batched_kernel<float, 1, true>);
        switch (l) {
        case 1:
        case 2: return batched_kernel_ptr_f32_v(l, false);
        case 3: return reinterpret_cast<const void *>(&batched_kernel<float, 3, false>);
        case 4: return reinterpret_cast<const void *>(&batched_kernel<float, 4, false>);
        default: return nullptr;
        }
    }
    if (vector_width == 2)
        return (ctas_per_sm == 4 && rows_per_thread == 1) ? batched_kernel_ptr_f32_v(l, cg) : nullptr;
    if (vector_width != 1) return nullptr;
    if (ctas_per_sm == 4) {
        if (rows_per_thread == 1) return batched_f32_shape<4, 1>(l, cg);
        if (rows_per_thread == 2) return batched_f32_shape<4, 2>(l, cg);
        if (rows_per_thread == 4) return batched_f32_shape<4, 4>(l, cg);
        return nullptr;
    }
    return batched_kernel_ptr_f32_3(l, cg, rows_per_thread);
}

}  // namespace plcg
