// kern_cluster_f32.cu -- instantiations of the cluster-resident solver for
// small systems (the grid is one thread-block cluster), T = float: the
// stencil (VEC = 4 and 1) and CSR operators, p(l)-CG for l = 1..4 and
// classic CG.
#include "solver.cuh"
#include "plcg_kernels.h"

namespace plcg {

template <int VEC, int OP>
static const void *cluster_ptr_f32(int l, bool cg)
{
    if (cg) return reinterpret_cast<const void *>(&plcg_cluster_kernel<float, 1, VEC, OP, true>);
    switch (l) {
    case 1: return reinterpret_cast<const void *>(&plcg_cluster_kernel<float, 1, VEC, OP, false>);
    case 2: return reinterpret_cast<const void *>(&plcg_cluster_kernel<float, 2, VEC, OP, false>);
    case 3: return reinterpret_cast<const void *>(&plcg_cluster_kernel<float, 3, VEC, OP, false>);
    case 4: return reinterpret_cast<const void *>(&plcg_cluster_kernel<float, 4, VEC, OP, false>);
    default: return nullptr;
    }
}

const void *kptr_cluster_f32(int op, int vec, int l, bool cg)
{
    if (op == kOpStencil) return vec == 4 ? cluster_ptr_f32<4, kOpStencil>(l, cg)
                                        : cluster_ptr_f32<1, kOpStencil>(l, cg);
    if (op == kOpCsr && vec == 1) return cluster_ptr_f32<1, kOpCsr>(l, cg);
    return nullptr;
}

}  // namespace plcg
