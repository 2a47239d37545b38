// plcg_kernels.h -- host-visible entry points of the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/plcg.h"

namespace plcg {

// Address of the persistent solver for (FP32 path?, operator, vector width,
// pipeline length l, classic CG?, scaled bases?, FP32 matrix values under
// FP64 vectors?); nullptr when not instantiated.
const void *kernel_ptr(bool f32, int op, int vec, int l, bool cg, bool sc = false, bool c32 = false);

// Address of the batched kernel for p(l)-CG (l = 1..4) or classic CG in a
// launch shape (CTAs per SM the registers are sized for, row groups per
// thread, vector width; 0, 0, 0 = the method's default; other shapes exist
// for FP32 only: 3 or 4 CTAs per SM with 1, 2 or 4 row groups and width 1,
// or 4 CTAs per SM, 1 row group and width 2); nullptr when absent.
const void *batched_kernel_ptr(bool f32, int l, bool cg, int ctas_per_sm = 0, int rows_per_thread = 0,
                               int vector_width = 0);
const void *batched_kernel_ptr_f32(int l, bool cg, int ctas_per_sm, int rows_per_thread, int vector_width);
const void *batched_kernel_ptr_f32_3(int l, bool cg, int rows_per_thread);
const void *batched_kernel_ptr_f32_v(int l, bool cg);
const void *batched_kernel_ptr_f64(int l, bool cg);

// Per-translation-unit getters used by kernel_ptr.
const void *kptr_f64_st2(int l, bool cg, bool sc);
const void *kptr_f64_st1(int l, bool cg, bool sc);
const void *kptr_f64_stsc(int vec, int l);
const void *kptr_f64_csr(int l, bool cg, bool sc);
const void *kptr_f32_st4(int l, bool cg);
const void *kptr_f32_st1(int l, bool cg);
const void *kptr_f32_csr(int l, bool cg);
const void *kptr_f64_csrj(int l, bool cg, bool sc);
const void *kptr_f32_csrj(int l, bool cg);
const void *kptr_f64_v27(int l, bool cg, bool sc);
const void *kptr_f32_v27(int l, bool cg);
const void *kptr_f64_v27j(int l, bool cg, bool sc);
const void *kptr_f32_v27j(int l, bool cg);
// The cluster-resident small-system solver (stencil and CSR operators,
// l = 1..4 or classic CG); nullptr when not instantiated.
const void *kptr_cluster_f64(int op, int vec, int l, bool cg);
const void *kptr_cluster_f32(int op, int vec, int l, bool cg);
const void *kptr_m_csr(int l, bool cg, bool sc);
const void *kptr_m_csrj(int l, bool cg, bool sc);
const void *kptr_m_v27(int l, bool cg, bool sc);
const void *kptr_m_v27j(int l, bool cg, bool sc);

// Sets the thread-local message returned by plcg_last_error().
void set_last_error(const std::string &msg);

// A stencil solve run exactly as plcg_solve would run it (argument checks,
// shifts, kernel, launch shape, kernel arguments), but with its workspace in
// the caller's device memory [base, base + cap) instead of an allocation.
// A solve whose workspace would exceed cap returns PLCG_ERR_INVALID naming
// both sizes (`who` prefixes the messages).  Synchronous.
plcg_status solve_stencil_fixed(const plcg_stencil_desc *desc, const double *b, double *x,
                                const plcg_params *prm, plcg_result *res, void *stream, char *base,
                                size_t cap, const char *who);

// Jacobi data of a CSR matrix: dinv64 = 1 / diag (FP64), dinv and diag in
// the stored value type (float if f32); *bad = 1 if a diagonal entry is not
// positive.
cudaError_t launch_jacobi_setup(bool f32, const int64_t *rowptr, const int32_t *col,
                                const void *val, int64_t n, double *dinv64, void *dinv,
                                void *diag, int *bad, cudaStream_t s);

// Jacobi data of the structured 27-point operator (diagonal = coef[0..n)):
// dinv64 = 1 / diag (FP64), dinv in the stored type; *bad = 1 if an entry
// is not positive.
cudaError_t launch_var27_jacobi_setup(bool f32, const void *coef, int64_t n, double *dinv64,
                                      void *dinv, int *bad, cudaStream_t s);

// v[i] = a pseudo-random value in [-1, 1) from (seed, i) (SplitMix64).
cudaError_t launch_fill_random(double *v, int64_t n, uint64_t seed, cudaStream_t s);

// dst[i] = (float) src[i] on the device.
cudaError_t launch_var27_zero_outside(bool f32, void *val, int64_t cstride, const StencilDesc &st,
                                      cudaStream_t s);
cudaError_t launch_round_to_f32(const double *src, float *dst, int64_t n, cudaStream_t s);

}  // namespace plcg
