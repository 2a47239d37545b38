// solver.cuh -- the persistent single-launch solvers of libplcg.so (sm_103a).
//
// One cooperative launch runs a whole solve: ||b||, residuals, every
// iteration of every segment (Algorithm 1 of Cools et al., EuroMPI'19, with
// M = I, or classic CG), restarts after square-root breakdowns (Sec. 2.2) and,
// on the FP32 path, the FP64 refinement loop.  Thread blocks (CTAs) own
// interleaved units of rows; one bounded grid barrier separates iterations
// (the SpMV of iteration i+1 reads neighbours written in iteration i).
//
// The global reduction of Alg. 2 (MPI_Iallreduce, consumed by MPI_Wait l
// iterations later) becomes: each CTA writes its FP64 dot partials into ring
// slot i mod (l+1) before the barrier, and at iteration i+l every CTA sums the
// slot's partials itself in a fixed order, so all CTAs hold bit-identical
// G entries and run the O(l^2) scalar work (K2, K3, K6 scalars) redundantly,
// with no extra barrier and no single-CTA serialisation.
#pragma once

#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include <type_traits>

#include "fxsum.h"
#include "plcg_internal.h"

namespace plcg {

// plcg_status values used on the device (mirrors include/plcg.h).
enum : int { kStOk = 0, kStBreakdown = -4, kStMaxit = -5, kStNonfinite = -6, kStTimeout = -7 };

constexpr int kMaxRefine = 64;   // FP32 path: cap on FP64 refinement steps

// ------------------------------------------------------------------------
// Memory-model helpers for the grid barrier.
// ------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(volatile const int *)p; }

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded grid-wide barrier.  Every CTA adds 1 to *bar; the barrier of epoch
// e is passed when *bar reaches e * gridDim.x.  Returns false when the poll
// bound ran out (the CTA then sets the abort flag) or another CTA aborted;
// the caller must then leave the kernel.  force_timeout adds one phantom
// arrival to the target so that the wait runs out (test hook).
__device__ __forceinline__ bool group_barrier(unsigned *bar, unsigned &epoch, unsigned members,
                                              unsigned long long limit, int force,
                                              int *abort_flag, int *s_ok)
{
    // bar.sync orders the CTA's writes before thread 0's release-add (release
    // is cumulative over what happened before it); the acquire-load that sees
    // the last arrival orders the reads after the trailing bar.sync.
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1u;
        const unsigned target = epoch * members + (force ? 1u : 0u);
        red_release_add_u32(bar, 1u);
        int ok = 1;
        unsigned long long polls = 0;
        while ((int)(ld_acquire_u32(bar) - target) < 0) {
            if ((++polls & 31) == 0) {
                if (ld_volatile(abort_flag)) { ok = 0; break; }
                if (polls > limit) { atomicExch(abort_flag, 1); ok = 0; break; }
                __nanosleep(32);
            }
        }
        if (ok && ld_volatile(abort_flag)) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned &epoch,
                                             unsigned long long limit, int force,
                                             int *abort_flag, int *s_ok)
{
    return group_barrier(bar, epoch, gridDim.x, limit, force, abort_flag, s_ok);
}

// ------------------------------------------------------------------------
// Bulk-copy staging (TMA, cp.async.bulk) with an mbarrier in shared memory.
// ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders generic-proxy writes that this thread has observed (another CTA's
// global stores of the previous iteration, acquired through the grid
// barrier) before its later async-proxy (bulk copy) reads.
__device__ __forceinline__ void fence_proxy_async_all()
{
    asm volatile("fence.proxy.async;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) completing its bytes on the mbarrier.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of the mbarrier; false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit)
{
    for (unsigned long long k = 0; k <= limit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------------------
// Reductions (fixed order, so every CTA gets the same bits).
// ------------------------------------------------------------------------
// A warp instruction on GB300's FP64 units occupies them for ~16 cycles, so
// the warp stage is a reduce-scatter butterfly: with NP = ND rounded up to a
// power of two, step j exchanges half of each lane's NP >> j remaining sums
// with lane ^ (16 >> j) and adds the other half, until every lane holds one
// sum; plain butterfly steps finish.  NP - 1 + 5 - log2(NP) FP64 adds per
// lane instead of 5 ND.  Dot q ends in lane q << (5 - log2(NP)).
template <int ND>
__device__ __forceinline__ double warp_reduce_scatter(const double (&v)[ND], int lane)
{
    constexpr int P = ND <= 1 ? 0 : ND <= 2 ? 1 : ND <= 4 ? 2 : ND <= 8 ? 3 : ND <= 16 ? 4 : 5;
    constexpr int NP = 1 << P;
    double w[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) w[q] = q < ND ? v[q] : 0.0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int o = 16 >> j;
        const int half = NP >> (j + 1);
        const bool upper = (lane & o) != 0;   // keep the upper half of the remaining sums
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const double send = upper ? w[q] : w[q + half];
            const double keep = upper ? w[q + half] : w[q];
            w[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    double t = w[0];
#pragma unroll
    for (int o = 16 >> P; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

template <int ND>
__device__ __forceinline__ void block_sum(double (&v)[ND], double *s_red, double *s_out)
{
    constexpr int P = ND <= 1 ? 0 : ND <= 2 ? 1 : ND <= 4 ? 2 : ND <= 8 ? 3 : ND <= 16 ? 4 : 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double t = warp_reduce_scatter<ND>(v, lane);
    if ((lane & ((32 >> P) - 1)) == 0) {
        const int q = lane >> (5 - P);
        if (q < ND) s_red[warp * ND + q] = t;
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        // pairwise over the warps (a dependent FP64 add costs ~64 cycles on GB300)
        double w8[kBlock / 32];
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) w8[w] = s_red[w * ND + threadIdx.x];
#pragma unroll
        for (int h = kBlock / 64; h >= 1; h >>= 1)
#pragma unroll
            for (int w = 0; w < h; ++w) w8[w] += w8[w + h];
        s_out[threadIdx.x] = w8[0];
    }
    __syncthreads();
}

// Sum over `count` CTAs of part[c * stride + q], q < ND; result in s_out[q].
template <int ND>
__device__ __forceinline__ void partials_sum(const double *part, int count, int stride,
                                             double *s_red, double *s_out)
{
    double v[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) v[q] = 0.0;
    for (int c = threadIdx.x; c < count; c += kBlock) {
#pragma unroll
        for (int q = 0; q < ND; ++q) v[q] += __ldcg(part + (size_t)c * stride + q);
    }
    block_sum<ND>(v, s_red, s_out);
}

template <int ND>
__device__ __forceinline__ void grid_partials_sum(const double *part, int stride, double *s_red,
                                                  double *s_out)
{
    partials_sum<ND>(part, (int)gridDim.x, stride, s_red, s_out);
}

// One warp: sum over `count` CTAs of part[c * stride + q] for Q0 <= q < ND
// in a fixed order (lane-strided partial sums, then the reduce-scatter
// butterfly); dst[q] (shared memory) gets the sums, 0 for q < Q0; then the
// warp syncs.
template <int ND, int Q0 = 0>
__device__ __forceinline__ void warp_partials_sum(const double *part, int count, int stride,
                                                  double *dst)
{
    constexpr int NA = ND - Q0;
    constexpr int P = NA <= 1 ? 0 : NA <= 2 ? 1 : NA <= 4 ? 2 : NA <= 8 ? 3 : NA <= 16 ? 4 : 5;
    const int lane = threadIdx.x & 31;
    double v[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) v[q] = 0.0;
    for (int c = lane; c < count; c += 32) {
#pragma unroll
        for (int q = 0; q < NA; ++q) v[q] += __ldcg(part + (size_t)c * stride + Q0 + q);
    }
    const double t = warp_reduce_scatter<NA>(v, lane);
    if ((lane & ((32 >> P) - 1)) == 0) {
        const int q = lane >> (5 - P);
        if (q < NA) dst[Q0 + q] = t;
    }
    if (lane < Q0) dst[lane] = 0.0;
    __syncwarp();
}

// The dots of the partial ring a scalar step needs: all 2l+1 positions with
// the 2l+1-dot variant, positions l .. 2l with the l+1 dots of Sec. 2.2.
template <int ND>
__device__ __forceinline__ void warp_dots_sum(const double *part, int count, int stride, bool all,
                                              double *dst)
{
    if (all) warp_partials_sum<ND, 0>(part, count, stride, dst);
    else warp_partials_sum<ND, (ND - 1) / 2>(part, count, stride, dst);
}

// ------------------------------------------------------------------------
// Vector loads/stores of VEC consecutive elements (128-bit when VEC*sizeof = 16).
// ------------------------------------------------------------------------
template <typename V, int VEC>
__device__ __forceinline__ void vld(const V *p, V (&o)[VEC])
{
    if constexpr (VEC == 1) {
        o[0] = *p;
    } else if constexpr (sizeof(V) == 8 && VEC == 2) {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else if constexpr (sizeof(V) == 4 && VEC == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (sizeof(V) == 4 && VEC == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = p[v];
    }
}

template <typename V, int VEC>
__device__ __forceinline__ void vldg(const V *p, V (&o)[VEC])   // read-only data (b, CSR)
{
    if constexpr (VEC == 1) {
        o[0] = __ldg(p);
    } else if constexpr (sizeof(V) == 8 && VEC == 2) {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = t.x; o[1] = t.y;
    } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = __ldg(p + v);
    }
}

template <typename V, int VEC>
__device__ __forceinline__ void vst(V *p, const V (&o)[VEC])
{
    if constexpr (VEC == 1) {
        *p = o[0];
    } else if constexpr (sizeof(V) == 8 && VEC == 2) {
        *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    } else if constexpr (sizeof(V) == 4 && VEC == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (sizeof(V) == 4 && VEC == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
    } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) p[v] = o[v];
    }
}

// ------------------------------------------------------------------------
// Operand loaders for the SpMV: one vector, or r + beta * p (classic CG).
// ------------------------------------------------------------------------
template <typename V>
struct Ld1 {
    const V *z;
    template <int VEC>
    __device__ __forceinline__ void vec(uint32_t g, V (&o)[VEC]) const { vld<V, VEC>(z + g, o); }
    __device__ __forceinline__ V one(uint32_t g) const { return z[g]; }
};

template <typename V>
struct LdAxpy {           // value = a[g] + beta * b[g]
    const V *a;
    const V *b;
    V beta;
    template <int VEC>
    __device__ __forceinline__ void vec(uint32_t g, V (&o)[VEC]) const
    {
        V t[VEC];
        vld<V, VEC>(a + g, o);
        vld<V, VEC>(b + g, t);
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = fma(beta, t[v], o[v]);
    }
    __device__ __forceinline__ V one(uint32_t g) const { return fma(beta, b[g], a[g]); }
};

template <typename V>
struct LdFirst {          // value = a[g] (CG first step, p_0 = r_0)
    const V *a;
    template <int VEC>
    __device__ __forceinline__ void vec(uint32_t g, V (&o)[VEC]) const { vld<V, VEC>(a + g, o); }
    __device__ __forceinline__ V one(uint32_t g) const { return a[g]; }
};

// ------------------------------------------------------------------------
// Stored matrix values into the arithmetic type.  GB300 converts between
// FP32 and FP64 on its narrow FP64 units, which the FP64 sweeps already keep
// busy, so an FP32 value is widened to FP64 with integer operations: the
// sign, the exponent rebiased by 1023 - 127 = 896 and the 23 mantissa bits
// placed in the two 32-bit halves of the double.  Exact for zeros and every
// normal FP32 value; FP32 subnormals (below 2^-126) read as signed zero.
// ------------------------------------------------------------------------
__device__ __forceinline__ double widen_f32(float f)
{
    const uint32_t u = __float_as_uint(f);
    const bool normal = (u & 0x7f800000u) != 0u;
    const uint32_t hi = (u & 0x80000000u) | (normal ? ((u & 0x7fffffffu) >> 3) + (896u << 20) : 0u);
    const uint32_t lo = normal ? (u << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

template <typename V, typename C>
__device__ __forceinline__ V coef_cast(C c)
{
    if constexpr (sizeof(V) == 8 && sizeof(C) == 4) return widen_f32(c);
    else return (V)c;
}

// ------------------------------------------------------------------------
// Operators.  apply() returns the centre values c and w = (A z) for the VEC
// rows g0 .. g0+VEC-1 (stencil: nx % VEC == 0, so they share y and z).
// ------------------------------------------------------------------------
// Centre values c and neighbour sums nb of the VEC rows g0 .. g0+VEC-1, so
// that (A z)_g = center * c + off * nb.  Row indices are 32-bit (n < 2^31):
// one multiply-add forms each address.
template <typename V, int VEC, class Ld>
__device__ __forceinline__ void stencil_parts(const StencilDesc &st, const Ld &ld, uint32_t g0,
                                              V (&c)[VEC], V (&nb)[VEC])
{
    const uint32_t nx = (uint32_t)st.nx, ny = (uint32_t)st.ny;
    // coordinates of row g0: x fastest, then y, then z
    const uint32_t line = (__umulhi(g0, st.dnx.m) + g0) >> st.dnx.s;
    const uint32_t x0 = g0 - line * nx;
    const uint32_t zc = (__umulhi(line, st.dny.m) + line) >> st.dny.s;
    const uint32_t y = line - zc * ny;
    ld.template vec<VEC>(g0, c);
    const V left = (x0 > 0) ? ld.one(g0 - 1) : V(0);
    const V right = (x0 + VEC < nx) ? ld.one(g0 + VEC) : V(0);
    if constexpr (std::is_same<V, double>::value && VEC >= 2) {
        // FP64, two rows per thread (systems of more than 16384 rows, bound
        // by the FP64 pipe): the neighbour sum on the integer units
        // (fxsum.h), the out-of-grid neighbours as zeros.  One row per
        // thread (small systems, bound by latency) keeps the FP64
        // additions, whose dependent chain is shorter.
        V ym[VEC], yp[VEC], zm[VEC], zp[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) ym[v] = yp[v] = zm[v] = zp[v] = V(0);
        if (y > 0) ld.template vec<VEC>(g0 - nx, ym);
        if (y + 1 < ny) ld.template vec<VEC>(g0 + nx, yp);
        if (st.dim == 3) {
            const uint32_t nxy = nx * ny;
            if (zc > 0) ld.template vec<VEC>(g0 - nxy, zm);
            if (zc + 1 < (uint32_t)st.nz) ld.template vec<VEC>(g0 + nxy, zp);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const double x[6] = {(v > 0) ? c[v - 1] : left, (v < VEC - 1) ? c[v + 1] : right,
                                     ym[v], yp[v], zm[v], zp[v]};
                nb[v] = fx_sum(x);
            }
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const double x[4] = {(v > 0) ? c[v - 1] : left, (v < VEC - 1) ? c[v + 1] : right,
                                     ym[v], yp[v]};
                nb[v] = fx_sum(x);
            }
        }
        return;
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v)
        nb[v] = ((v > 0) ? c[v - 1] : left) + ((v < VEC - 1) ? c[v + 1] : right);
    V t[VEC];
    if (y > 0) {
        ld.template vec<VEC>(g0 - nx, t);
#pragma unroll
        for (int v = 0; v < VEC; ++v) nb[v] += t[v];
    }
    if (y + 1 < ny) {
        ld.template vec<VEC>(g0 + nx, t);
#pragma unroll
        for (int v = 0; v < VEC; ++v) nb[v] += t[v];
    }
    if (st.dim == 3) {
        const uint32_t nxy = nx * ny;
        if (zc > 0) {
            ld.template vec<VEC>(g0 - nxy, t);
#pragma unroll
            for (int v = 0; v < VEC; ++v) nb[v] += t[v];
        }
        if (zc + 1 < (uint32_t)st.nz) {
            ld.template vec<VEC>(g0 + nxy, t);
#pragma unroll
            for (int v = 0; v < VEC; ++v) nb[v] += t[v];
        }
    }
}

template <typename V, int VEC, class Ld>
__device__ __forceinline__ void stencil_apply(const StencilDesc &st, V cC, V cO, const Ld &ld,
                                              uint32_t g0, V (&c)[VEC], V (&w)[VEC])
{
    V nb[VEC];
    stencil_parts<V, VEC>(st, ld, g0, c, nb);
#pragma unroll
    for (int v = 0; v < VEC; ++v) w[v] = fma(cO, nb[v], cC * c[v]);
}

// Row g of the structured symmetric 27-point operator (VEC = 1): the full
// (A z)_g = a_gg z_g + sum over the 13 forward offsets d of
// w_d(g) z_{g+d} + w_d(g-d) z_{g-d}, where w_d(c) = coef[1+k][c] is the
// entry A[c, c+d] and the backward entry comes from the neighbour by
// symmetry; neighbours outside the grid are skipped (Dirichlet).  C is the
// stored coefficient type.
template <typename V, typename C, class Ld>
__device__ __forceinline__ V var27_row(const StencilDesc &st, const C *coef, int64_t stride,
                                       const Ld &ld, uint32_t g)
{
    const uint32_t nx = (uint32_t)st.nx, ny = (uint32_t)st.ny, nz = (uint32_t)st.nz;
    const uint32_t nxy = nx * ny;
    const size_t n = (size_t)stride;
    const uint32_t line = (__umulhi(g, st.dnx.m) + g) >> st.dnx.s;
    const uint32_t x = g - line * nx;
    const uint32_t zc = (__umulhi(line, st.dny.m) + line) >> st.dny.s;
    const uint32_t y = line - zc * ny;
    const bool xm = x > 0, xp = x + 1 < nx, ym = y > 0, yp = y + 1 < ny, zm = zc > 0, zp = zc + 1 < nz;
    V s = coef_cast<V>(__ldg(coef + g)) * ld.one(g);
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        const int dz = v27_dz(k), dy = v27_dy(k), dx = v27_dx(k);
        const uint32_t off = (uint32_t)(dz * (int)nxy + dy * (int)nx + dx);   // > 0
        const bool fwd = (dx > 0 ? xp : dx < 0 ? xm : true) && (dy > 0 ? yp : dy < 0 ? ym : true) &&
                         (dz > 0 ? zp : true);
        const bool bwd = (dx > 0 ? xm : dx < 0 ? xp : true) && (dy > 0 ? ym : dy < 0 ? yp : true) &&
                         (dz > 0 ? zm : true);
        const C *ck = coef + (size_t)(1 + k) * n;
        if (fwd) s = fma(coef_cast<V>(__ldg(ck + g)), ld.one(g + off), s);
        if (bwd) s = fma(coef_cast<V>(__ldg(ck + (g - off))), ld.one(g - off), s);
    }
    return s;
}

// CSR row (VEC = 1).  C is the stored value type (float or double).
template <typename V, typename C, class Ld>
__device__ __forceinline__ V csr_row(const CsrDesc &A, const Ld &ld, uint32_t row)
{
    const C *val = static_cast<const C *>(A.val);
    const int64_t e0 = __ldg(A.rowptr + row), e1 = __ldg(A.rowptr + row + 1);
    V s = V(0);
    for (int64_t e = e0; e < e1; ++e) s = fma(coef_cast<V>(__ldg(val + e)), ld.one(__ldg(A.col + e)), s);
    return s;
}

// A CSR row whose entries were staged in shared memory (scol / sval), from
// the row's staged entry range [k0, k1).
template <typename V, typename C, class Ld>
__device__ __forceinline__ V csr_row_k(const int32_t *scol, const C *sval, uint32_t k0, uint32_t k1, const Ld &ld)
{
    V s = V(0);
    for (uint32_t k = k0; k < k1; ++k) s = fma(coef_cast<V>(sval[k]), ld.one((uint32_t)scol[k]), s);
    return s;
}

// Per-CTA tiles of the structured 27-point operator, one per sweep unit of
// rows [r0, r1) (dynamic shared memory: v27_hdr(SB) bytes of header -- the
// NB mbarriers in 16-byte pairs and, without SB, the 13 base pointers of the
// backward loads -- then NB buffers of kSlots slots of kV27Slot elements):
// slots 0..13 the diagonal and forward coefficients of the unit's rows; with
// SB slots 14..26 the backward coefficients (forward array k at rows g - d_k,
// by symmetry); then nine slots' room for z around the unit: its nine line
// segments ((dz, dy) in {-1,0,1}^2, x - 1 .. x + 1), or its three plane
// segments (each the lines dy = -1..1 of plane dz with their x halo); then
// the unit's rows of NV vector operands (the steady-state sweep's; other
// sweeps load those from global memory).  One bulk copy per slot (a plane
// segment fills three), each rounded out to 16 bytes; the rounding puts
// element g of a backward or z slot at a shift that is fixed for the whole
// solve (the arrays and ring vectors start on 256-byte boundaries and units
// on multiples of 4 rows), so the shifts are computed once; forward and
// vector slots start at their first row.  The sweep keeps the next NB - 1
// units' copies in flight while it computes from the current buffer.
// Without SB the backward coefficients come through L2, loaded before the
// wait for the unit's copies.  A unit whose copies would leave the arrays'
// allocations falls back to global loads (vectors are padded to 256 bytes,
// so their rounded copies always stay inside).
template <typename T, int NV, bool SB>
struct Var27Tile {
    static constexpr int A = 16 / (int)sizeof(T);   // elements per 16 bytes
    static constexpr int NB = v27_bufs(SB);          // buffers
    static constexpr int kZ = SB ? 27 : 14;          // first z slot
    static constexpr int kV = v27_op_slots(SB);      // first vector slot
    static constexpr int kSlots = kV + NV;
    static constexpr int kBuf = kSlots * kV27Slot;   // elements per buffer
    uint64_t *bar;                                   // bar[0 .. NB-1]
    const T **bwd;                                   // without SB: bwd[k] + g, backward coefficient k of row g
    T *slot0;
    uint32_t parity = 0;          // bit b: the phase buffer b waits for next
    uint32_t shb = 0, shz = 0;    // 2-bit shifts of the backward and z slots
    // z staging: the nine line segments in slots of their own, or (zm, when
    // a plane's three lines with their x halo fit three slots: nx <= 275)
    // one copy per plane dz holding the lines dy = -1, 0, 1 nx apart, so a
    // unit takes 3 z copies instead of 9; ys = the distance between the
    // line segments of one plane in the tile
    bool zm = false;
    int ys = kV27Slot;
    __device__ __forceinline__ explicit Var27Tile(unsigned char *dsm)
        : bar(reinterpret_cast<uint64_t *>(dsm)),
          bwd(reinterpret_cast<const T **>(dsm + 16 * ((NB + 1) / 2))),
          slot0(reinterpret_cast<T *>(dsm + v27_hdr(SB)))
    {
    }
    // Needs a __syncthreads() before the first issue().
    __device__ __forceinline__ void init(const StencilDesc &st, const T *coef, int64_t cstride, bool merge_z)
    {
        const int64_t nx = st.nx, nxy = (int64_t)st.nx * st.ny;
        if (threadIdx.x == 0)
            for (int b = 0; b < NB; ++b) mbar_init(bar + b, kSlots);
        if (!SB && threadIdx.x < 13) {
            const int k = threadIdx.x;
            bwd[k] = coef + (1 + k) * cstride - (v27_dz(k) * nxy + v27_dy(k) * nx + v27_dx(k));
        }
        for (int k = 0; k < 13; ++k) {
            const int off = v27_dz(k) * (int)nxy + v27_dy(k) * (int)nx + v27_dx(k);
            shb |= (uint32_t)(((-off) % A + A) % A) << (2 * k);
        }
        zm = merge_z && 2 * nx + kBlock + 2 * A + 2 <= 3 * kV27Slot;
        ys = zm ? (int)nx : kV27Slot;
        for (int q = 0; q < 9; ++q) {
            // the row at the start of the z copy that holds line q, relative to r0
            const int d = zm ? (q / 3 - 1) * (int)nxy - (int)nx - 1
                             : (q / 3 - 1) * (int)nxy + (q % 3 - 1) * (int)nx - 1;
            shz |= (uint32_t)((d % A + A) % A) << (2 * q);
        }
    }
    // The slot this thread stages when the first nthreads threads (whole
    // warps) sweep; kSlots or more: none.  The slots are dealt round-robin
    // over those warps (slot = lane * warps + warp): the bulk copies that one
    // warp instruction issues for several lanes go out one after another, so
    // each warp issues only a few of the unit's copies (128^3 Jacobi
    // p(1)-CG 15.1 -> 13.0 ms against threads 0 .. kSlots-1 owning them).
    __device__ __forceinline__ static int my_slot(int nthreads)
    {
        const int w = (int)(threadIdx.x >> 5), nw = nthreads >> 5;
        return w < nw ? (int)(threadIdx.x & 31) * nw + w : kSlots;
    }
    __device__ __forceinline__ static bool issues(int nthreads) { return my_slot(nthreads) < kSlots; }
    __device__ __forceinline__ int sb(int k) const { return (int)((shb >> (2 * k)) & 3u); }
    __device__ __forceinline__ int sz(int q) const { return (int)((shz >> (2 * q)) & 3u); }
    // Vector slot j of buffer buf (element t = row r0 + t).
    __device__ __forceinline__ const T *vec(int buf, int j) const
    {
        return slot0 + buf * kBuf + (kV + j) * kV27Slot;
    }
    // a_gg of row r0 + t (the diagonal slot).
    __device__ __forceinline__ T diag(int buf, int t) const { return slot0[buf * kBuf + t]; }
    // Without SB: the backward coefficients of row g (issued before wait():
    // their L2 latency overlaps the copies').
    __device__ __forceinline__ void backward(uint32_t g, T (&bw)[13]) const
    {
        if constexpr (!SB) {
#pragma unroll
            for (int k = 0; k < 13; ++k) bw[k] = __ldg(bwd[k] + g);
        }
    }
    // The copy plan of one slot for the current sweep: the copy of unit
    // [r0, r1) reads [base + (r0 + loff) elements, base + (r1 + hoff)
    // elements), rounded out to 16 bytes, which must lie inside [lo, hi) and
    // fit cap bytes, into element dst of the buffer; base == null: no copy.
    // Written by prepare() and read by issue() in the slot's owner thread
    // only (no barrier between them), kept in shared memory after the
    // buffers rather than in registers.
    struct Plan {
        const char *base, *lo, *hi;
        int loff, hoff, dst, cap;
    };
    __device__ __forceinline__ Plan *plans() const { return reinterpret_cast<Plan *>(slot0 + NB * kBuf); }
    // The plans of this sweep (every thread calls it; owners write): the
    // operator slots from coef (allocation [clo, chi)) and z (the ring's
    // allocation [zlo, zhi)), the vector slots from vsrc(j) when `vecs`.
    template <class VSrc>
    __device__ __forceinline__ void prepare(bool vecs, const VSrc &vsrc, const StencilDesc &st, const T *coef,
                                            int64_t cstride, const char *clo, const char *chi, const T *z,
                                            const char *zlo, const char *zhi, int nthreads)
    {
        const int sl = my_slot(nthreads);
        if (sl >= kSlots) return;
        const int nx = st.nx, nxy = st.nx * st.ny;
        Plan p{nullptr, clo, chi, 0, 0, sl * kV27Slot, kV27Slot * (int)sizeof(T)};
        if (sl < 14) {
            p.base = reinterpret_cast<const char *>(coef + sl * cstride);
        } else if (sl < kZ) {
            const int k = sl - 14;
            const int off = v27_dz(k) * nxy + v27_dy(k) * nx + v27_dx(k);
            p.base = reinterpret_cast<const char *>(coef + (1 + k) * cstride);
            p.loff = p.hoff = -off;   // may start in the zero halo before the arrays
        } else if (sl < kV) {
            const int q = sl - kZ;
            p.lo = zlo;
            p.hi = zhi;
            if (zm) {   // planes dz = q - 1 in slots kZ, kZ + 3, kZ + 6; no copy for q >= 3
                if (q < 3) {
                    p.base = reinterpret_cast<const char *>(z);
                    p.loff = (q - 1) * nxy - nx - 1;
                    p.hoff = (q - 1) * nxy + nx + 1;
                    p.dst = kZ * kV27Slot + q * 3 * kV27Slot;
                    p.cap = 3 * kV27Slot * (int)sizeof(T);
                }
            } else {
                const int d = (q / 3 - 1) * nxy + (q % 3 - 1) * nx;
                p.base = reinterpret_cast<const char *>(z);
                p.loff = d - 1;
                p.hoff = d + 1;
            }
        } else if (vecs) {   // whole rows from their start; padded to 256 bytes: always inside
            p.base = reinterpret_cast<const char *>(vsrc(sl - kV));
            p.lo = nullptr;
            p.hi = reinterpret_cast<const char *>(~uintptr_t(0));
        }
        plans()[sl] = p;
    }
    // Start staging rows [r0, r1) in buffer buf by this sweep's plans
    // (`want` false: nothing to stage, the barrier alone).  Each slot has one
    // owner thread among the first `nthreads` (my_slot): the owners check
    // that their 16-byte-rounded ranges stay inside their allocations, the
    // first `nthreads` threads agree on the result with a barrier reduction
    // (which also orders every read of the buffer's previous unit before the
    // new copies: those reads have completed into registers, and the
    // async-proxy writes follow the barrier), and every owner issues its copy,
    // arriving on the buffer's mbarrier (init count kSlots) with its bytes.
    // Returns false when the unit is to be read from global memory;
    // otherwise every thread calls wait() before reading the tile.
    __device__ __forceinline__ bool issue(int buf, bool want, uint32_t r0, uint32_t r1, int nthreads)
    {
        const int sl = my_slot(nthreads);
        uintptr_t b0 = 0, b1 = 0;
        int dst = 0;
        int ok = 1;
        if (sl < kV && !want) ok = 0;
        if (sl < kSlots && want) {
            const Plan p = plans()[sl];
            dst = p.dst;
            const int64_t lo = (int64_t)r0 + p.loff, hi = (int64_t)r1 + p.hoff;
            if (p.base && hi > lo) {
                b0 = reinterpret_cast<uintptr_t>(p.base + lo * (int64_t)sizeof(T)) & ~uintptr_t(15);
                b1 = (reinterpret_cast<uintptr_t>(p.base + hi * (int64_t)sizeof(T)) + 15) & ~uintptr_t(15);
                ok = b0 >= reinterpret_cast<uintptr_t>(p.lo) && b1 <= reinterpret_cast<uintptr_t>(p.hi) &&
                     b1 - b0 <= (uintptr_t)p.cap;
            }
        }
        int all;
        asm volatile("{\n\t.reg .pred p, q;\n\t"
                     "setp.ne.s32 p, %1, 0;\n\t"
                     "bar.red.and.pred q, 1, %2, p;\n\t"
                     "selp.s32 %0, 1, 0, q;\n\t}"
                     : "=r"(all) : "r"(ok), "r"(nthreads) : "memory");
        if (!all) return false;
        if (sl < kSlots) {
            const uint32_t bytes = (uint32_t)(b1 - b0);
            mbar_arrive_expect_tx(bar + buf, bytes);
            if (bytes)
                bulk_copy_g2s(slot0 + buf * kBuf + dst, reinterpret_cast<const void *>(b0), bytes, bar + buf);
        }
        return true;
    }
    // Wait for the copies issue() started (bounded: on timeout the abort flag
    // is raised and the wait repeated once, so no copy is left in flight).
    __device__ __forceinline__ void wait(int buf, unsigned long long limit, int *abort_flag)
    {
        const uint32_t ph = (parity >> buf) & 1u;
        if (!mbar_wait(bar + buf, ph, limit)) {
            atomicExch(abort_flag, 1);
            mbar_wait(bar + buf, ph, limit);
        }
        parity ^= 1u << buf;
    }
    // (A z)_g for row g = r0 + t of the unit staged in buffer buf (z's centre
    // value in *zc; without SB, bw holds backward()'s coefficients of the
    // row).  No boundary tests: entries towards cells outside the grid are
    // stored as zero and every z value a copy brings in is finite (z itself,
    // or the zero halos around the ring vectors).
    template <typename V>
    __device__ __forceinline__ V row(int buf, int t, const T (&bw)[13], V *zc) const
    {
        const T *slot = slot0 + buf * kBuf;
        const T *zs = slot + kZ * kV27Slot;
        auto zat = [&](int dz, int dy, int dx) -> V {
            const int q = (dz + 1) * 3 + (dy + 1);
            return (V)zs[(dz + 1) * 3 * kV27Slot + (dy + 1) * ys + t + 1 + dx + sz(q)];
        };
        const V c = zat(0, 0, 0);
        *zc = c;
        V s = (V)slot[t] * c;
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            const int dz = v27_dz(k), dy = v27_dy(k), dx = v27_dx(k);
            s = fma((V)slot[(1 + k) * kV27Slot + t], zat(dz, dy, dx), s);
            const V b = SB ? (V)slot[(14 + k) * kV27Slot + t + sb(k)] : (V)bw[k];
            s = fma(b, zat(-dz, -dy, -dx), s);
        }
        return s;
    }
};

// Per-warp staging of CSR entries in shared memory (dynamic shared memory,
// layout in plcg_internal.h).  Every warp stages the entries of its own 32
// rows of a sweep unit -- a contiguous range, since the rows are -- with one
// bulk copy for the column indices and one for the values, completing on
// the warp's mbarrier, and waits only for them: the CTA's warps are
// independent copy/compute pipelines, so one warp's copy overlaps the others'
// arithmetic.
template <typename T>
struct CsrStage {
    uint64_t *bar;
    int32_t *col;
    T *val;
    uint32_t parity = 0;      // phase parity of bar for the warp's next staged rows
    __device__ __forceinline__ explicit CsrStage(unsigned char *dsm)
    {
        const int w = threadIdx.x >> 5;
        bar = reinterpret_cast<uint64_t *>(dsm) + w;
        col = reinterpret_cast<int32_t *>(dsm + 128) + w * kCsrStageWarpCap;
        val = reinterpret_cast<T *>(dsm + 128 + 8 * 4 * kCsrStageWarpCap) + w * kCsrStageWarpCap;
    }
    // One thread per warp initialises the warp's mbarrier (then a CTA barrier).
    __device__ __forceinline__ void init()
    {
        if ((threadIdx.x & 31) == 0) mbar_init(bar, 1);
    }
    // The row pointers of the warp's rows [r0, r1) (r1 - r0 <= 32), loaded
    // one unit ahead so that their latency overlaps the current unit: one
    // broadcast load of rowptr[r0] and one coalesced load of this lane's row
    // end rowptr[min(r0 + lane + 1, r1)].
    struct Rows {
        int64_t start, end;
    };
    __device__ __forceinline__ static Rows rows_load(const CsrDesc &csr, uint32_t r0, uint32_t r1)
    {
        const uint32_t lane = threadIdx.x & 31;
        return {__ldg(csr.rowptr + r0), __ldg(csr.rowptr + min(r0 + lane + 1, r1))};
    }
    // The warp's entry range [e0, e1) and this lane's row [rs, re) from the
    // loads (every lane of the warp calls it: shuffles).
    __device__ __forceinline__ static void rows_bounds(const Rows &p, int64_t *e0, int64_t *e1, int64_t *rs,
                                                       int64_t *re)
    {
        const int64_t up = __shfl_up_sync(0xffffffffu, p.end, 1);
        *e0 = p.start;
        *e1 = __shfl_sync(0xffffffffu, p.end, 31);
        *rs = (threadIdx.x & 31) ? up : p.start;
        *re = p.end;
    }
    // Stage the entries [e0, e1) of the warp's rows (rows_bounds), rounded
    // out to 16 bytes (the arrays carry the padding), issued by lane 0 once
    // every lane is done with the previous rows' entries; every lane waits.
    // Returns false (read global memory) when the range exceeds the warp's
    // buffer; *e0s is the global position of the first staged entry.
    __device__ __forceinline__ bool stage_range(const CsrDesc &csr, int64_t e0, int64_t e1, int64_t *e0s,
                                                unsigned long long limit, int *abort_flag)
    {
        *e0s = e0 & ~int64_t(3);
        const int64_t cnt = ((e1 + 3) & ~int64_t(3)) - *e0s;
        const bool on = cnt > 0 && cnt <= kCsrStageWarpCap;
        __syncwarp();
        if (on) {
            if ((threadIdx.x & 31) == 0) {
                // the lanes' reads of the previous rows' entries were consumed
                // before the __syncwarp above, so the copy cannot overtake them
                const uint32_t cb = (uint32_t)cnt * 4u, vb = (uint32_t)cnt * (uint32_t)sizeof(T);
                mbar_arrive_expect_tx(bar, cb + vb);
                bulk_copy_g2s(col, csr.col + *e0s, cb, bar);
                bulk_copy_g2s(val, static_cast<const T *>(csr.val) + *e0s, vb, bar);
            }
            if (!mbar_wait(bar, parity, limit)) {
                atomicExch(abort_flag, 1);          // the solve ends at the next barrier
                mbar_wait(bar, parity, limit);      // the copy in flight lands first
            }
            parity ^= 1u;
        }
        return on;
    }
};

// (c, nb) with (A z)_g = kc * c + kn * nb: stencil (center, off), CSR (0, 1).
template <typename V, typename C, int VEC, int OP, class Ld>
__device__ __forceinline__ void op_parts(const StencilDesc &st, const CsrDesc &csr, const Ld &ld,
                                         uint32_t g0, V (&c)[VEC], V (&nb)[VEC])
{
    if constexpr (OP == kOpStencil) {
        stencil_parts<V, VEC>(st, ld, g0, c, nb);
    } else if constexpr (op_is_var27(OP)) {
        static_assert(VEC == 1, "27-point rows are one per thread");
        c[0] = ld.one(g0);
        nb[0] = var27_row<V, C>(st, static_cast<const C *>(csr.val), csr.stride, ld, g0);
    } else {
        static_assert(VEC == 1, "CSR rows are one per thread");
        c[0] = ld.one(g0);
        nb[0] = csr_row<V, C>(csr, ld, g0);
    }
}

template <typename V, typename C, int VEC, int OP, class Ld>
__device__ __forceinline__ void op_apply(const StencilDesc &st, const CsrDesc &csr, V cC, V cO,
                                         const Ld &ld, uint32_t g0, V (&c)[VEC], V (&w)[VEC])
{
    if constexpr (OP == kOpStencil) {
        stencil_apply<V, VEC>(st, cC, cO, ld, g0, c, w);
    } else if constexpr (op_is_var27(OP)) {
        static_assert(VEC == 1, "27-point rows are one per thread");
        c[0] = ld.one(g0);
        w[0] = var27_row<V, C>(st, static_cast<const C *>(csr.val), csr.stride, ld, g0);
    } else {
        static_assert(VEC == 1, "CSR rows are one per thread");
        c[0] = ld.one(g0);
        w[0] = csr_row<V, C>(csr, ld, g0);
    }
}

// ------------------------------------------------------------------------
// Shared-memory state of one CTA.
// ------------------------------------------------------------------------
template <typename T>
struct Coef {
    int mode;                 // 0: fill (i < l), 1: recurrences (i >= l)
    int k6;                   // 0: none, 1: phat_0 = v_0, 2: x and phat update (phat_m = eta_m p_m)
    int end;                  // -1: continue, else SegEnd
    int fmode;                // final sweep: 0 x += f1 phat; 1 lucky (m >= 1); 2 lucky (m = 0)
    int prev0;                // z^(0)_{m-1} exists
    int ncopy;
    long long kseg;           // k of the iterate the segment returns (when end >= 0)
    T sig, invd, al, bm;
    T uc, unb;                // K4 coefficients of z^(l)_i and of the SpMV's neighbour part
    T ak[kMaxL];
    T wu[kMaxL], wb[kMaxL];   // K4, basis k < l: coefficients of z^(k+1) and of z^(k)_{prev}
    int unit;                 // scaled bases: unb and wu[0] are exactly 1 (steady sweep form)
    T zx, pv, pp;
    T f1, f2;
    int dsrc[kMaxDots];       // 0 off, 1 memory, 2 new u, 3 new v, 4 z^(l)_i, 5 z^(l)_{i-1}
    const T *dptr[kMaxDots];
    const T *zl_cur;
    const T *zl_prev;
    T *zl_new;
    const T *cur[kMaxL];
    const T *prv[kMaxL];
    T *nw[kMaxL];
    T *cpy[kMaxL];
    const T *v0;              // final sweep: z^(0)_m
};

// The fields of Coef the iteration sweep reads, as a register copy for the
// one-CTA path (see the sweep); the rarely used cpy and dptr stay in shared
// memory.
template <typename T, int L>
struct SweepCoef {
    int mode, k6, prev0, ncopy;
    T sig, invd, al, bm, uc, unb, zx, pv, pp;
    T ak[L], wu[L], wb[L];
    int unit;
    int dsrc[2 * L + 1];
    const T *zl_cur, *zl_prev;
    T *zl_new;
    const T *cur[L], *prv[L];
    T *nw[L];
    __device__ __forceinline__ SweepCoef(const Coef<T> &c)
        : mode(c.mode), k6(c.k6), prev0(c.prev0), ncopy(c.ncopy), sig(c.sig), invd(c.invd),
          al(c.al), bm(c.bm), uc(c.uc), unb(c.unb), zx(c.zx), pv(c.pv), pp(c.pp), zl_cur(c.zl_cur),
          zl_prev(c.zl_prev),
          zl_new(c.zl_new), unit(c.unit)
    {
#pragma unroll
        for (int k = 0; k < L; ++k) {
            ak[k] = c.ak[k];
            wu[k] = c.wu[k];
            wb[k] = c.wb[k];
            cur[k] = c.cur[k];
            prv[k] = c.prv[k];
            nw[k] = c.nw[k];
        }
#pragma unroll
        for (int q = 0; q <= 2 * L; ++q) dsrc[q] = c.dsrc[q];
    }
};

template <typename T>
struct Smem {
    double red[(kBlock / 32) * kMaxDots];
    double out[kMaxDots + 2];
    double raw[kMaxDots];
    double G[kMaxL + 1][kMaxDots];   // finalised columns c-l .. c (column c at c mod (l+1))
    double Ginv[kMaxL + 1];          // 1 / g_{c,c} of those columns
    double gam[kMaxL + 1], del[kMaxL + 1], idel[kMaxL + 1];   // gamma_j, delta_j, 1 / delta_j
    double eta[2], zeta[2], ieta[2]; // eta_m, zeta_m, 1 / eta_m
    double scs[16], iscs[16];        // scaled bases: s_j of z^(l)_j (j mod 16) and reciprocals
    double sct[kMaxL][16];           // ... t^(k)_j of z^(k)_j, k < l (j mod 16)
    double isct[kMaxL][16];          // ... and their reciprocals
    double ikn;                      // 1 / kn
    double bring[kMaxL + 1][kMaxDots];   // one-CTA group: reduced dots of the last l+1 iterations
    double bnorm[2];
    double raw2[kMaxDots];           // the scalar warp's copy of a reduced dot column
    Coef<T> cfb[2];                  // coefficients of iterations i (i & 1) and i + 1
    long long stg_e0;                // CSR staging: global position of the unit's first staged entry
    int stg_on;                      // CSR staging: this unit's entries are in shared memory
    int ok;
};

template <typename T> struct Eps;
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };
template <> struct Eps<float> { static constexpr double v = (double)FLT_EPSILON; };

// Vector j of basis k's ring: slot j mod depth[k] (j < 2^31; the modulo by
// the invariant depth uses the host-prepared multiply-shift divisor).
template <typename T>
__device__ __forceinline__ T *ring(const SolveArgs<T> &a, int k, long long j)
{
    const uint32_t jj = (uint32_t)j;
    const uint32_t q = (__umulhi(jj, a.ddiv[k].m) + jj) >> a.ddiv[k].s;
    return a.zring + (a.base[k] + (int64_t)(jj - q * (uint32_t)a.depth[k])) * a.vstride;
}

// ------------------------------------------------------------------------
// Execution groups.  A solve runs either on the whole grid (one system per
// launch; CTAs meet at a bounded grid barrier and exchange FP64 partials
// through global memory) or on one CTA (batched solves: one system per CTA;
// __syncthreads is the barrier and the reduced dots stay in shared memory).
// ------------------------------------------------------------------------
template <typename T>
struct GridGroup {
    unsigned epoch = 0;
    __device__ __forceinline__ int64_t unit0() const { return blockIdx.x; }
    __device__ __forceinline__ int64_t ustep() const { return gridDim.x; }
    __device__ __forceinline__ bool leader() const { return blockIdx.x == 0; }
    __device__ __forceinline__ bool sync(const SolveArgs<T> &a, Smem<T> &s)
    {
        return grid_barrier(a.bar, epoch, a.poll_limit, a.force_timeout, &a.out->abort, &s.ok);
    }
    // this CTA's reduced dots (s.out[0..nd)) into ring slot `slot`
    __device__ __forceinline__ void put_dots(const SolveArgs<T> &a, Smem<T> &s, int slot, int nd)
    {
        if ((int)threadIdx.x < nd)
            a.part[((size_t)slot * gridDim.x + blockIdx.x) * kMaxDots + threadIdx.x] = s.out[threadIdx.x];
    }
    // sum over CTAs of ring slot `slot` into dst[0..ND)
    template <int ND>
    __device__ __forceinline__ void get_dots(const SolveArgs<T> &a, Smem<T> &s, int slot, double *dst)
    {
        // warp 0 sums (few FP64 instructions: GB300's FP64 units are narrow),
        // the CTA barrier publishes the result
        if (threadIdx.x < 32)
            warp_partials_sum<ND>(a.part + (size_t)slot * gridDim.x * kMaxDots, (int)gridDim.x, kMaxDots, dst);
        __syncthreads();
    }
    // one warp sums ring slot `slot` over the CTAs into dst (every CTA's warp
    // adds in the same order, so all CTAs get the same bits)
    template <int ND>
    __device__ __forceinline__ void get_dots_warp(const SolveArgs<T> &a, Smem<T> &, int slot,
                                                  double *dst)
    {
        warp_dots_sum<ND>(a.part + (size_t)slot * gridDim.x * kMaxDots, (int)gridDim.x, kMaxDots,
                          a.dots_2l1 != 0, dst);
    }
    __device__ __forceinline__ void put_norms(const SolveArgs<T> &a, Smem<T> &s)
    {
        if (threadIdx.x == 0) {
            a.npart[(size_t)blockIdx.x * kNormSlots + 0] = s.out[0];
            a.npart[(size_t)blockIdx.x * kNormSlots + 1] = s.out[1];
        }
    }
    __device__ __forceinline__ void get_norms(const SolveArgs<T> &a, Smem<T> &s)
    {
        grid_partials_sum<2>(a.npart, kNormSlots, s.red, s.out);
    }
};

template <typename T>
struct BlockGroup {
    __device__ __forceinline__ int64_t unit0() const { return 0; }
    __device__ __forceinline__ int64_t ustep() const { return 1; }
    __device__ __forceinline__ bool leader() const { return true; }
    __device__ __forceinline__ bool sync(const SolveArgs<T> &, Smem<T> &)
    {
        __syncthreads();
        return true;
    }
    __device__ __forceinline__ void put_dots(const SolveArgs<T> &, Smem<T> &s, int slot, int nd)
    {
        if ((int)threadIdx.x < nd) s.bring[slot][threadIdx.x] = s.out[threadIdx.x];
    }
    template <int ND>
    __device__ __forceinline__ void get_dots(const SolveArgs<T> &, Smem<T> &s, int slot, double *dst)
    {
        if ((int)threadIdx.x < ND) dst[threadIdx.x] = s.bring[slot][threadIdx.x];
        __syncthreads();
    }
    // the scalar warp of this very CTA reads the ring in shared memory
    template <int ND>
    __device__ __forceinline__ void get_dots_warp(const SolveArgs<T> &, Smem<T> &s, int slot,
                                                  double *dst)
    {
        for (int q = threadIdx.x & 31; q < ND; q += 32) dst[q] = s.bring[slot][q];
        __syncwarp();
    }
    __device__ __forceinline__ void put_norms(const SolveArgs<T> &, Smem<T> &s)
    {
        if (threadIdx.x < 2) s.bnorm[threadIdx.x] = s.out[threadIdx.x];
    }
    __device__ __forceinline__ void get_norms(const SolveArgs<T> &, Smem<T> &s)
    {
        if (threadIdx.x < 2) s.out[threadIdx.x] = s.bnorm[threadIdx.x];
        __syncthreads();
    }
};

// ------------------------------------------------------------------------
// Thread-block clusters: the whole grid is one cluster of up to 16 CTAs on
// neighbouring SMs, which the hardware schedules together.  Its barrier
// (barrier.cluster, release/acquire at cluster scope, which orders the
// CTAs' global and shared memory accesses) replaces the grid barrier, and
// each CTA's reduced dots stay in its own shared memory, where the others
// read them through distributed shared memory (mapa + ld.shared::cluster).
// ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_size()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster (warp-converged).
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The double at the same shared-memory offset as *p in CTA `rank` of the cluster.
__device__ __forceinline__ double ld_dsmem(const double *p, uint32_t rank)
{
    uint32_t ra;
    double v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_addr(p)), "r"(rank));
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
    return v;
}

// One warp: dst[q] = sum over the cluster's CTAs of their src[q], Q0 <= q < ND,
// in a fixed order (lane c reads CTA c, then the reduce-scatter butterfly),
// so every CTA gets the same bits; dst[q] = 0 for q < Q0.
template <int ND, int Q0 = 0>
__device__ __forceinline__ void cluster_dots_sum(const double *src, double *dst)
{
    constexpr int NA = ND - Q0;
    constexpr int P = NA <= 1 ? 0 : NA <= 2 ? 1 : NA <= 4 ? 2 : NA <= 8 ? 3 : NA <= 16 ? 4 : 5;
    const int lane = threadIdx.x & 31;
    const uint32_t nc = cluster_size();
    double v[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) v[q] = ((uint32_t)lane < nc) ? ld_dsmem(src + Q0 + q, (uint32_t)lane) : 0.0;
    const double t = warp_reduce_scatter<NA>(v, lane);
    if ((lane & ((32 >> P) - 1)) == 0) {
        const int q = lane >> (5 - P);
        if (q < NA) dst[Q0 + q] = t;
    }
    if (lane < Q0) dst[lane] = 0.0;
    __syncwarp();
}

template <typename T>
struct ClusterGroup {
    __device__ __forceinline__ int64_t unit0() const { return cluster_rank(); }
    __device__ __forceinline__ int64_t ustep() const { return cluster_size(); }
    __device__ __forceinline__ bool leader() const { return cluster_rank() == 0; }
    // no bounded wait to expire: every CTA takes the same branches (the
    // scalars are bit-identical), so all arrive at every barrier
    __device__ __forceinline__ bool sync(const SolveArgs<T> &, Smem<T> &)
    {
        cluster_barrier();
        return true;
    }
    __device__ __forceinline__ void put_dots(const SolveArgs<T> &, Smem<T> &s, int slot, int nd)
    {
        if ((int)threadIdx.x < nd) s.bring[slot][threadIdx.x] = s.out[threadIdx.x];
    }
    template <int ND>
    __device__ __forceinline__ void get_dots(const SolveArgs<T> &, Smem<T> &s, int slot, double *dst)
    {
        if (threadIdx.x < 32) cluster_dots_sum<ND>(&s.bring[slot][0], dst);
        __syncthreads();
    }
    template <int ND>
    __device__ __forceinline__ void get_dots_warp(const SolveArgs<T> &a, Smem<T> &s, int slot, double *dst)
    {
        if (a.dots_2l1) cluster_dots_sum<ND, 0>(&s.bring[slot][0], dst);
        else cluster_dots_sum<ND, (ND - 1) / 2>(&s.bring[slot][0], dst);
    }
    __device__ __forceinline__ void put_norms(const SolveArgs<T> &, Smem<T> &s)
    {
        if (threadIdx.x < 2) s.bnorm[threadIdx.x] = s.out[threadIdx.x];
    }
    __device__ __forceinline__ void get_norms(const SolveArgs<T> &, Smem<T> &s)
    {
        if (threadIdx.x < 32) cluster_dots_sum<2>(&s.bnorm[0], s.out);
        __syncthreads();
    }
};

// A gang: G CTAs of one cooperative launch solving one system together
// (batched solves of large systems); bounded barrier and FP64 partials of its
// own, so gangs proceed independently of each other.
template <typename T>
struct GangGroup {
    int rank, G;
    unsigned *bar;
    unsigned epoch;
    double *part;             // [(l+1) slots][G][kMaxDots]
    double *npart;            // [G][kNormSlots]
    int *abort_flag;
    unsigned long long limit;
    __device__ __forceinline__ int64_t unit0() const { return rank; }
    __device__ __forceinline__ int64_t ustep() const { return G; }
    __device__ __forceinline__ bool leader() const { return rank == 0; }
    __device__ __forceinline__ bool sync(const SolveArgs<T> &, Smem<T> &s)
    {
        return group_barrier(bar, epoch, (unsigned)G, limit, 0, abort_flag, &s.ok);
    }
    __device__ __forceinline__ void put_dots(const SolveArgs<T> &, Smem<T> &s, int slot, int nd)
    {
        if ((int)threadIdx.x < nd)
            part[((size_t)slot * G + rank) * kMaxDots + threadIdx.x] = s.out[threadIdx.x];
    }
    template <int ND>
    __device__ __forceinline__ void get_dots(const SolveArgs<T> &, Smem<T> &s, int slot, double *dst)
    {
        if (threadIdx.x < 32) warp_partials_sum<ND>(part + (size_t)slot * G * kMaxDots, G, kMaxDots, dst);
        __syncthreads();
    }
    template <int ND>
    __device__ __forceinline__ void get_dots_warp(const SolveArgs<T> &a, Smem<T> &, int slot,
                                                  double *dst)
    {
        warp_dots_sum<ND>(part + (size_t)slot * G * kMaxDots, G, kMaxDots, a.dots_2l1 != 0, dst);
    }
    __device__ __forceinline__ void put_norms(const SolveArgs<T> &, Smem<T> &s)
    {
        if (threadIdx.x == 0) {
            npart[(size_t)rank * kNormSlots + 0] = s.out[0];
            npart[(size_t)rank * kNormSlots + 1] = s.out[1];
        }
    }
    __device__ __forceinline__ void get_norms(const SolveArgs<T> &, Smem<T> &s)
    {
        partials_sum<2>(npart, G, kNormSlots, s.red, s.out);
    }
};

// ------------------------------------------------------------------------
// Scalar step of iteration i (one thread of every CTA; all CTAs compute the
// same bits).  K2: finalise column c = i-l+1 of G (Algorithm 1) and its
// breakdown check; K3: gamma_{i-l}, delta_{i-l}; K6 scalars: lambda, eta,
// zeta and the stop test.
// A dependent FP64 operation costs ~64 cycles on GB300 and a division or a
// square root ~500, so the step is ordered for latency: the vector pointers
// (integer work) first; then gamma, the K6 scalars (which do not need
// g_{c,c}) and 1/sqrt(arg) are all in flight before the breakdown branch;
// g_{c,c} = arg / sqrt(arg) and 1/delta_m = g_{m,m} / (g_{c,c} delta_{m-l})
// come from that one reciprocal square root with the cached 1/delta, so
// the critical path holds one rsqrt and one reciprocal (1/eta_m, off the
// rsqrt's path).
// ------------------------------------------------------------------------
template <typename T, int L>
__device__ __forceinline__ void step_vectors(Coef<T> &cf, const SolveArgs<T> &a, int i)
{
    const int m = i - L;
    const bool rec = i >= L;
    cf.zl_cur = ring(a, L, i);
    cf.zl_prev = (i >= 1) ? ring(a, L, i - 1) : nullptr;
    cf.zl_new = ring(a, L, i + 1);
    if (!rec) {
        for (int k = i + 1; k <= L - 1; ++k) cf.cpy[cf.ncopy++] = ring(a, k, i + 1);
    } else {
#pragma unroll
        for (int k = 0; k < L; ++k) {
            cf.cur[k] = ring(a, k, m + k);
            cf.prv[k] = (m + k - 1 >= 0) ? ring(a, k, m + k - 1) : nullptr;
            cf.nw[k] = ring(a, k, m + k + 1);
        }
    }
    // K5 operands: position q is row j = i-2l+1+q of column i+1 (Algorithm 1, K5)
#pragma unroll
    for (int q = 0; q <= 2 * L; ++q) {
        const int j = i - 2 * L + 1 + q;
        int src = 0;
        const T *ptr = nullptr;
        if (j >= 0) {
            if (q < L) {
                if (a.dots_2l1) { src = 1; ptr = ring(a, 0, j); }
            } else if (q == L) {
                if (rec) src = 3;
                else { src = 1; ptr = ring(a, 0, j); }
            } else {
                if (j == i + 1) src = 2;
                else if (j == i) src = 4;
                else if (j == i - 1 && rec) src = 5;
                else { src = 1; ptr = ring(a, L, j); }
            }
        }
        cf.dsrc[q] = src;
        cf.dptr[q] = ptr;
    }
}

// Scaled bases (FP64).  The sweep stores Z_j = z^(l)_j / s_j and, for each
// basis k < l, W^(k)_j = z^(k)_j / t^(k)_j, and the direction
// P_m = phat_m / t^(0)_m, with the scales chosen so that K4 needs no
// multiply for one term of each recurrence: s_{i+1} = s_i kn / delta_m and
// t^(k)_{m+k+1} = t^(k+1)_{m+k+1} / delta_m (t^(l) being s), times a power
// of two (2^e, 2^f_k) only when a product leaves [2^-256, 2^256]; with
// (A z)_g = kc z_g + kn nb_g,
//   Z_{i+1} = nb(Z_i) + ((kc - gamma_m) / kn) Z_i - (delta_{m-1} s_{i-1} / (kn s_i)) Z_{i-1}
//   W^(k)_{m+k+1} = U + (sigma_k - gamma_m)(t^(k)_{m+k} / u) W^(k)_{m+k}
//                     - delta_{m-1} (t^(k)_{m+k-1} / u) W^(k)_{m+k-1}
// where U = W^(k+1)_{m+k+1} (Z_i for k = l - 1) has the scale u (each term
// divided by 2^e or 2^f_k when that is not 1: the general sweep form then).
// The host picks this variant (SC) for 2^19 rows or more (l <= 5 on the
// stencils, l = 1 elsewhere): below that the step's extra latency outweighs
// the FP64 multiplies per row it saves.  The K5 dots of scaled vectors are
// multiplied back by their scales here, so G, gamma, delta, eta and zeta are
// those of the unscaled algorithm; K6 folds t^(0) into its scalars.  Same
// iterates in exact arithmetic.  Scale rings of 16 hold every index a step
// reads: s over 2l values, t^(0) over 2l + 1 (l <= 5).
template <typename T, int L>
constexpr bool kScaledBases = (sizeof(T) == 8 && L <= 5);

template <typename T, int L, bool SC>
__device__ __forceinline__ void scalar_step_body(Smem<T> &s, Coef<T> &cf, const double *raw,
                                                 const SolveArgs<T> &a, int i, double rn,
                                                 double tau, long long budget, T kc, T kn)
{
    cf.end = -1;
    cf.fmode = 0;
    cf.ncopy = 0;
    cf.unit = 0;
    const int m = i - L;
    step_vectors<T, L>(cf, a, i);
    constexpr bool kScaled = SC && kScaledBases<T, L>;
    const bool scl = kScaled && kn != T(0);
    if (i < L) {
        cf.mode = 0;
        cf.k6 = 0;
        cf.sig = (T)a.sigma[i];
        if (kScaled && i == 0) {   // a segment starts from unscaled vectors (the fill phase's)
            for (int j = 0; j <= L; ++j) {
                s.scs[j] = s.iscs[j] = 1.0;
                for (int k = 0; k < L; ++k) s.sct[k][j] = s.isct[k][j] = 1.0;
            }
            s.ikn = scl ? 1.0 / (double)kn : 0.0;
        }
        return;
    }
    const int c = i - L + 1;
    double *col = s.G[c % (L + 1)];
    // scales of this step: s_i, s_{i-1}, t_m = t^(0)_m, t_{m-1} (with
    // reciprocals kept beside them: no division on the step's path)
    double s_i = 1.0, s_im1 = 1.0, t_m = 1.0, t_mm1 = 1.0, is_i = 1.0, it_m = 1.0, s_c = 1.0;
    if (scl) {
        s_i = s.scs[i & 15];
        is_i = s.iscs[i & 15];
        s_im1 = s.scs[(i - 1) & 15];
        s_c = s.scs[c & 15];
        t_m = s.sct[0][m & 15];
        it_m = s.isct[0][m & 15];
        t_mm1 = (m >= 1) ? s.sct[0][(m - 1) & 15] : 1.0;
    }
    auto g = [&](int j, int cc) -> double {
        if (j < 0 || j < cc - 2 * L || j > cc) return 0.0;
        return s.G[cc % (L + 1)][j - cc + 2 * L];
    };
    auto ginv = [&](int j) -> double { return s.Ginv[j % (L + 1)]; };
    auto del = [&](int j) -> double { return j < 0 ? 0.0 : s.del[j % (L + 1)]; };
    auto idel = [&](int j) -> double { return s.idel[j % (L + 1)]; };
    auto gam = [&](int j) -> double { return s.gam[j % (L + 1)]; };
    // raw column c (dots of iteration i-l): position q is row j = c-2l+q;
    // scaled bases: u_c = s_c Z_c against t^(0)_j W^(0)_j (q <= l) or s_j Z_j
#pragma unroll
    for (int q = 0; q <= 2 * L; ++q) {
        const int j = c - 2 * L + q;
        double v = (j >= 0) ? raw[q] : 0.0;
        if (scl && j >= 0) v *= s_c * (q <= L ? s.sct[0][j & 15] : s.scs[j & 15]);
        col[q] = v;
    }
    const int lo = (c - 2 * L > 0) ? c - 2 * L : 0;
    if (!a.dots_2l1)   // Sec. 2.2: g_{j,c} = g_{c-l,j+l} for j = c-2l .. c-l-1
        for (int j = lo; j <= c - L - 1; ++j) col[j - c + 2 * L] = g(c - L, j + L);
    for (int j = (c - L + 1 > 0 ? c - L + 1 : 0); j <= c - 1; ++j) {
        double t = col[j - c + 2 * L];
        for (int k = lo; k <= j - 1; ++k) t -= g(k, j) * col[k - c + 2 * L];
        col[j - c + 2 * L] = t * ginv(j);
    }
    const double graw = col[2 * L];
    double arg = graw;
    for (int k = lo; k <= c - 1; ++k) arg -= col[k - c + 2 * L] * col[k - c + 2 * L];
    const double rg = rsqrt(arg);          // NaN or inf when arg <= 0: unused then
    const double gmm = g(m, m), igmm = ginv(m);
    const double gmc = col[m - c + 2 * L];
    const double dm1 = del(m - 1);        // delta_{m-1} (0 for m = 0)
    double gm;
    if (m < L)
        gm = (gmc + a.sigma[m] * gmm - (m >= 1 ? g(m - 1, m) * dm1 : 0.0)) * igmm;
    else
        gm = (gmm * gam(m - L) + gmc * del(m - L) - g(m - 1, m) * dm1) * igmm;
    s.gam[m % (L + 1)] = gm;
    // K6 scalars for m >= 1 (Sec. 2.1): lambda_m, eta_m, zeta_m need no g_{c,c}
    double lam = 0.0, em = gm, iem = 0.0, zm = 0.0;
    if (m >= 1) {
        lam = dm1 * s.ieta[(m - 1) & 1];
        em = gm - lam * dm1;
        iem = 1.0 / em;
        zm = -lam * s.zeta[(m - 1) & 1];
    }
    const double thr = 64.0 * Eps<T>::v * fabs(graw);
    if (!isfinite(arg) || !isfinite(gm)) {
        cf.end = kSegNonfinite;
        cf.kseg = m;
        return;
    }
    if (arg <= thr) {
        if (arg >= -thr) {   // lucky breakdown: x_{m+1} is exact in this Krylov space
            if (m == 0) {
                s.eta[0] = gm;
                s.zeta[0] = rn;
                cf.fmode = 2;
                cf.pv = (T)(1.0 / gm);
                cf.f2 = (T)rn;
            } else {
                // p_{m-1} = phat_{m-1} / eta_{m-1}; p_m = (v_m - delta_{m-1} p_{m-1}) / eta_m
                // (scaled bases: v_m = t_m W_m, phat_{m-1} = t_{m-1} P_{m-1})
                const double iep = s.ieta[(m - 1) & 1];
                cf.fmode = 1;
                cf.f1 = (T)(s.zeta[(m - 1) & 1] * iep * t_mm1);
                cf.pv = (T)(iem * t_m);
                cf.pp = (T)(-dm1 * iem * iep * t_mm1);
                cf.f2 = (T)zm;
            }
            cf.end = kSegLucky;
            cf.kseg = m + 1;
        } else {             // breakdown: keep x_m and restart
            cf.fmode = 0;
            cf.f1 = (T)((m >= 1) ? s.zeta[(m - 1) & 1] * s.ieta[(m - 1) & 1] * t_mm1 : 0.0);
            cf.end = kSegBreakdown;
            cf.kseg = m;
        }
        cf.v0 = ring(a, 0, m);
        return;
    }
    // g_{c,c} = sqrt(arg) and the recurrence coefficients from 1/sqrt(arg):
    // delta_m = g_{c,c} [delta_{m-l}] / g_{m,m}, 1/delta_m = g_{m,m} / (g_{c,c} [delta_{m-l}])
    const double gcc = arg * rg;
    col[2 * L] = gcc;
    s.Ginv[c % (L + 1)] = rg;
    const double invd = (m < L) ? rg * gmm : rg * gmm * idel(m - L);
    const double dm = (m < L) ? gcc * igmm : gcc * del(m - L) * igmm;
    s.del[m % (L + 1)] = dm;
    s.idel[m % (L + 1)] = invd;
    cf.mode = 1;
    cf.prev0 = (m >= 1);
    if (scl) {
        // scaled bases: the new scales, 2^e and 2^f_k keeping them in range
        auto pow2 = [](int k) -> double {   // 2^k, |k| < 1000
            return __longlong_as_double((long long)(1023 + k) << 52);
        };
        auto out_of_range = [](double v) -> bool { return !(fabs(v) >= 0x1p-256 && fabs(v) <= 0x1p256); };
        const double bs = invd * (double)kn * s_i;
        const int e = out_of_range(bs) ? -ilogb(bs) : 0;
        const double pe = pow2(-e), ivk = pe * s.ikn;
        s.scs[(i + 1) & 15] = bs * pow2(e);
        s.iscs[(i + 1) & 15] = dm * s.ikn * is_i * pe;
        cf.invd = (T)ivk;
        cf.al = (T)(-gm * ivk);
        cf.uc = (T)(((double)kc - gm) * ivk);
        cf.unb = (T)pe;
        cf.bm = (T)((m >= 1) ? -dm1 * (s_im1 * is_i) * ivk : 0.0);
        int unit = (e == 0);
#pragma unroll
        for (int k = 0; k < L; ++k) {
            // basis k: current z^(k)_{m+k}, previous z^(k)_{m+k-1}, new z^(k)_{m+k+1};
            // U = z^(k+1)_{m+k+1} (z^(l)_i for k = l - 1) with scale u
            const int jc = m + k, jn = m + k + 1;
            const double u = (k == L - 1) ? s_i : s.sct[k + 1][jn & 15];
            const double iu = (k == L - 1) ? is_i : s.isct[k + 1][jn & 15];
            const double tc = s.sct[k][jc & 15];
            const double tp = (jc >= 1) ? s.sct[k][(jc - 1) & 15] : 1.0;
            const double bt = invd * u;
            const int f = out_of_range(bt) ? -ilogb(bt) : 0;
            const double pf = pow2(-f);
            s.sct[k][jn & 15] = bt * pow2(f);
            s.isct[k][jn & 15] = dm * iu * pf;
            cf.ak[k] = (T)((a.sigma[k] - gm) * (tc * iu) * pf);
            cf.wu[k] = (T)pf;
            cf.wb[k] = (T)((m >= 1) ? -dm1 * (tp * iu) * pf : 0.0);
            unit &= (f == 0);
        }
        cf.unit = unit;
    } else {
        cf.invd = (T)invd;
        cf.al = (T)(-gm * invd);
        cf.bm = (T)((m >= 1) ? -dm1 * invd : 0.0);
        // (A z)_g = kc z_g + kn nb_g: K4's coefficients of z^(l)_i and nb, once
        // here instead of per row in the sweep
        cf.uc = fma(kc, cf.invd, cf.al);
        cf.unb = kn * cf.invd;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            cf.ak[k] = (T)((a.sigma[k] - gm) * invd);
            cf.wu[k] = cf.invd;
            cf.wb[k] = cf.bm;
        }
    }
    // K6 on the scaled direction phat_m = eta_m p_m (one FMA per row fewer):
    // phat_0 = v_0, phat_m = v_m - (delta_{m-1} / eta_{m-1}) phat_{m-1},
    // x_m = x_{m-1} + (zeta_{m-1} / eta_{m-1}) phat_{m-1}
    if (i == L) {
        s.eta[0] = gm;
        s.zeta[0] = rn;
        s.ieta[0] = 1.0 / gm;
        cf.k6 = 1;
    } else {
        const double iep = s.ieta[(m - 1) & 1];
        cf.k6 = 2;
        // scaled bases: P_m = phat_m / t_m = W_m - (delta_{m-1}/eta_{m-1})(t_{m-1}/t_m) P_{m-1}
        cf.zx = (T)(s.zeta[(m - 1) & 1] * iep * t_mm1);
        cf.pp = (T)(-dm1 * iep * (t_mm1 * it_m));
        s.eta[m & 1] = em;
        s.ieta[m & 1] = iem;
        s.zeta[m & 1] = zm;
        if (!isfinite(zm)) {
            cf.end = kSegNonfinite;
            cf.kseg = m;
            return;
        }
        if (fabs(zm) < tau || m >= budget) {
            cf.end = (fabs(zm) < tau) ? kSegConverged : kSegMaxit;
            cf.fmode = 0;
            cf.f1 = cf.zx;
            cf.kseg = m;
            cf.v0 = ring(a, 0, m);
            return;
        }
    }
}

template <typename T, int L, bool SC>
__device__ __noinline__ void scalar_step_call(Smem<T> &s, Coef<T> &cf, const double *raw,
                                              const SolveArgs<T> &a, int i, double rn, double tau,
                                              long long budget, T kc, T kn)
{
    scalar_step_body<T, L, SC>(s, cf, raw, a, i, rn, tau, budget, kc, kn);
}

// The scalar step inline, except in the FP32 whole-grid kernels: there the
// sweep runs at 80 registers (3 CTAs per SM) and an inlined scalar step
// changes its register allocation enough to cost ~15% at 256^3 (measured);
// the out-of-line call costs ~0.3 us per iteration, which the FP64 and
// one-CTA paths (latency-bound on small systems) keep.
template <typename T, int L, bool OOL, bool SC>
__device__ __forceinline__ void scalar_step(Smem<T> &s, Coef<T> &cf, const double *raw,
                                            const SolveArgs<T> &a, int i, double rn, double tau,
                                            long long budget, T kc, T kn)
{
    if constexpr (OOL) scalar_step_call<T, L, SC>(s, cf, raw, a, i, rn, tau, budget, kc, kn);
    else scalar_step_body<T, L, SC>(s, cf, raw, a, i, rn, tau, budget, kc, kn);
}

// Per-thread accumulator of one dot product over the units a thread sweeps.
// FP64 vectors: one FMA per term into the FP64 sum.  FP32 vectors: the
// compensated dot product Dot2 of Ogita, Rump & Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26(6), 2005 -- Dekker's TwoProduct (via FMA)
// per term and Knuth's TwoSum into a running FP32 pair (s, t) -- flushed
// into the FP64 sum every kFlushUnits units.  A pair then covers at most
// kFlushUnits * VEC * RPT <= 512 terms, whose error bound (Ogita et al.,
// Thm. 5.3) is eps_32 |sum| + gamma_n^2 sum |terms| with gamma_512^2 < 1e-8:
// below the rounding of the FP32 vectors themselves.  A flush is two
// conversions and two adds on GB300's FP64 units, where a warp instruction
// occupies them for ~16 cycles, so flushes are kept rare.
constexpr int kFlushUnits = 32;

template <typename T, int VEC>
struct DotAcc {
    double acc = 0.0;
    float s = 0.f, t = 0.f;
    __device__ __forceinline__ void add(const T (&x)[VEC], const T (&y)[VEC])
    {
        if constexpr (sizeof(T) == 8) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc = fma(x[v], y[v], acc);
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const float h = __fmul_rn(x[v], y[v]);
                const float lo = __fmaf_rn(x[v], y[v], -h);
                const float s2 = __fadd_rn(s, h);
                const float bb = __fsub_rn(s2, s);
                const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb)), __fsub_rn(h, bb));
                s = s2;
                t = __fadd_rn(t, __fadd_rn(e, lo));
            }
        }
    }
    __device__ __forceinline__ void flush()
    {
        if constexpr (sizeof(T) == 4) {
            acc = (acc + (double)s) + (double)t;
            s = 0.f;
            t = 0.f;
        }
    }
};

// ------------------------------------------------------------------------
// Residual sweep: r = b - A x (FP64; the stored operator values widened),
// this CTA's ||r||^2 and ||b||^2 in s.out[0..1] -- with the Jacobi
// preconditioner the natural norms r^T M^{-1} r and b^T M^{-1} b (Sec. 2.2,
// "Residual norm in p(l)-CG").  Units of kBlock * V64 rows.
// ------------------------------------------------------------------------
template <typename T, int VEC, int OP, class Grp, typename C = T>
__device__ void residual_sweep(const SolveArgs<T> &a, Smem<T> &s, const Grp &grp)
{
    constexpr int V64 = (VEC >= 2) ? 2 : 1;
    constexpr int UNIT = kBlock * V64;
    const int64_t n = a.n;
    const int64_t nunits = (n + UNIT - 1) / UNIT;
    const double cC = (double)(T)a.st.center, cO = (double)(T)a.st.off;
    double acc[2] = {0.0, 0.0};
    Ld1<double> ld{a.x};
    for (int64_t u = grp.unit0(); u < nunits; u += grp.ustep()) {
        const uint32_t g0 = (uint32_t)(u * UNIT + (int64_t)threadIdx.x * V64);
        if (g0 >= (uint32_t)n) continue;
        double c[V64], w[V64], bv[V64];
        if constexpr (OP == kOpStencil) {
            stencil_apply<double, V64>(a.st, cC, cO, ld, g0, c, w);
        } else if constexpr (op_is_var27(OP)) {
            c[0] = a.x[g0];
            w[0] = var27_row<double, C>(a.st, static_cast<const C *>(a.csr.val), a.csr.stride, ld, g0);
        } else {
            c[0] = a.x[g0];
            w[0] = csr_row<double, C>(a.csr, ld, g0);
        }
        vldg<double, V64>(a.b + g0, bv);
        double rv[V64];
#pragma unroll
        for (int v = 0; v < V64; ++v) {
            rv[v] = bv[v] - w[v];
            if constexpr (op_is_jacobi(OP)) {
                const double mi = __ldg(a.dinv64 + g0 + v);
                acc[0] = fma(bv[v] * mi, bv[v], acc[0]);
                acc[1] = fma(rv[v] * mi, rv[v], acc[1]);
            } else {
                acc[0] = fma(bv[v], bv[v], acc[0]);
                acc[1] = fma(rv[v], rv[v], acc[1]);
            }
        }
        vst<double, V64>(a.r + g0, rv);
    }
    block_sum<2>(acc, s.red, s.out);
}

template <typename T>
__device__ __forceinline__ void write_result(const SolveArgs<T> &a, int status, long long iters,
                                             long long spmvs, long long restarts,
                                             long long refinements, double recres, double normb,
                                             double last_rn)
{
    DevResult *o = a.out;
    o->status = (ld_volatile(&o->abort) && status == kStOk) ? kStTimeout : status;
    o->iters = iters;
    o->spmvs = spmvs;
    o->restarts = restarts;
    o->refinements = refinements;
    o->recursive_relres = (normb > 0.0) ? recres / normb : 0.0;
    o->true_relres = (normb > 0.0) ? last_rn / normb : 0.0;
    o->t_end_ns = global_timer_ns();
}

// K5 operand of dot q in the steady state (l+1 dots, i >= l+1): the same
// choice scalar_step makes, as a compile-time function of q: 0 no dot,
// 1 ring vector z^(l)_j from memory, 2 the new z^(l)_{i+1}, 3 the new
// z^(0)_{i-l+1}, 4 z^(l)_i, 5 z^(l)_{i-1}.
template <int L>
__device__ __forceinline__ constexpr int steady_dot_src(int q)
{
    return q < L ? 0 : q == L ? 3 : q == 2 * L ? 2 : q == 2 * L - 1 ? 4 : q == 2 * L - 2 ? 5 : 1;
}

// ------------------------------------------------------------------------
// p(l)-CG: a whole solve on one group (grid or CTA).
// ------------------------------------------------------------------------
// D1: the l + 1 dots of Sec. 2.2 only (the 2l + 1 option compiled out: the
// sweep then carries no accumulators for positions 0 .. l-1).
template <typename T, int L, int VEC, int OP, class Grp, int RPT = 1, bool SC = false, typename CT = T,
          bool D1 = false>
__device__ void plcg_body(const SolveArgs<T> &a, Smem<T> &s, Grp &grp)
{
    const bool d2 = !D1 && a.dots_2l1;   // the 2l + 1 dots
    constexpr int UNIT = kBlock * VEC;
    constexpr bool kF32 = (sizeof(T) == 4);
    constexpr bool kOolScalar = kF32 && std::is_same<Grp, GridGroup<T>>::value;
    // FP64 p(1)-CG keeps its bases scaled (see scalar_step_body): two FP64
    // multiplies per row fewer in the FP64-bound sweep
    constexpr bool kScaled = SC && kScaledBases<T, L>;
    // CSR on the whole grid: each sweep unit's entries are bulk-copied into
    // shared memory (one contiguous range per unit) before its rows are read
    constexpr bool kStage = op_is_csr(OP) && std::is_same<Grp, GridGroup<T>>::value && RPT == 1;
    extern __shared__ __align__(128) unsigned char plcg_dsm[];
    CsrStage<CT> stage(plcg_dsm);
    if constexpr (kStage) {
        stage.init();
        __syncthreads();
    }
    // structured 27-point operator on the whole grid, FP32: each sweep unit's
    // coefficients and z^(l) lines are staged as a shared-memory tile (the
    // FP64 sweep is bound by the FP64 units and measured faster without)
    constexpr bool kTile = op_is_var27(OP) && std::is_same<Grp, GridGroup<T>>::value && RPT == 1 &&
                           sizeof(T) == 4 && sizeof(CT) == 4;
    constexpr int kNV = kTile ? v27_vec_slots(L, op_is_jacobi(OP)) : 0;
    using Tile = Var27Tile<T, kNV, kV27StageBwdPlcg>;
    Tile tile(plcg_dsm);
    if constexpr (kTile) {
        tile.init(a.st, static_cast<const T *>(a.csr.val), a.csr.stride, kV27MergeZPlcg);
        __syncthreads();
        // zero the halo before ring vector 0 and the span after every ring
        // vector (rows n .. vstride-1): the tiles' z-line copies reach into
        // them and multiply what they find by zero coefficients (the grid
        // barrier after the first residual sweep orders these stores before
        // any copy)
        const int64_t span = a.vstride - a.n, nz = a.halo + (int64_t)a.nring * span;
        for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < nz; e += (int64_t)gridDim.x * kBlock) {
            if (e < a.halo) {
                a.zring[e - a.halo] = T(0);
            } else {
                const int64_t i = (e - a.halo) / span;
                a.zring[i * a.vstride + a.n + (e - a.halo - i * span)] = T(0);
            }
        }
    }
    const int64_t n = a.n;
    const int64_t nunits = (n + UNIT - 1) / UNIT;
    const int tid = threadIdx.x;
    const T cC = (T)a.st.center, cO = (T)a.st.off;
    // (A z)_g = kc * c + kn * nb (see op_parts)
    const T kc = (OP == kOpStencil) ? cC : T(0), kn = (OP == kOpStencil) ? cO : T(1);
    // xi: the iterate K6 updates (FP64 path: x itself; FP32 path: the inner
    // correction d of the refinement step)
    T *xi = kF32 ? a.rc : reinterpret_cast<T *>(a.x);

    long long iters = 0, spmvs = 0, restarts = 0, refinements = 0, segments = 0;
    int last_end = kSegConverged;
    double normb = 0.0, recres = 0.0, last_rn = 0.0;
    int status = kStOk;

#define PLCG_SYNC()                                                                          \
    do {                                                                                     \
        if (!grp.sync(a, s)) {                                                               \
            status = kStTimeout;                                                             \
            goto finish;                                                                     \
        }                                                                                    \
    } while (0)

    for (;;) {
        // ---- true residual r = b - A x and its norm (Algorithm 1 initialization / the final check)
        residual_sweep<T, VEC, OP, Grp, CT>(a, s, grp);
        grp.put_norms(a, s);
        spmvs++;
        PLCG_SYNC();
        grp.get_norms(a, s);
        if (segments == 0) normb = sqrt(s.out[0]);
        const double rn = sqrt(s.out[1]);
        last_rn = rn;
        if (normb == 0.0) {
            // b = 0: x = 0 is the solution
            for (int64_t u = grp.unit0(); u * kBlock < n; u += grp.ustep()) {
                const int64_t g = u * kBlock + tid;
                if (g < n) a.x[g] = 0.0;
            }
            status = kStOk;
            break;
        }
        if (!isfinite(normb) || !isfinite(rn)) { status = kStNonfinite; break; }
        if (rn < a.rtol * normb) { status = kStOk; recres = (segments == 0) ? rn : recres; break; }
        if (iters >= a.maxit) { status = kStMaxit; break; }
        if (segments > 0) {
            if (kF32 && (last_end == kSegConverged || last_end == kSegLucky)) {
                if (++refinements > kMaxRefine) { status = kStMaxit; break; }
            } else {
                if (restarts >= a.max_restarts) {
                    status = (last_end == kSegMaxit) ? kStMaxit : kStBreakdown;
                    break;
                }
                restarts++;
            }
        }
        const double tau = kF32 ? fmax(a.inner_floor * rn, 0.5 * a.rtol * normb) : a.rtol * normb;
        const long long budget = a.maxit - iters;

        // ---- Algorithm 1, initialization: z^(k)_0 := M^{-1} r_0 / nu for every
        // k, nu = sqrt((r_0, M^{-1} r_0)); u_0 = M z^(l)_0 is never stored; g_00 := 1
        {
            const double inv = 1.0 / rn;
            for (int64_t u = grp.unit0(); u < nunits; u += grp.ustep()) {
                const int64_t g0 = u * UNIT + (int64_t)tid * VEC;
                if (g0 >= n) continue;
                T z[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    if constexpr (op_is_jacobi(OP))
                        z[v] = (T)(a.r[g0 + v] * __ldg(a.dinv64 + g0 + v) * inv);
                    else
                        z[v] = (T)(a.r[g0 + v] * inv);
                }
#pragma unroll
                for (int k = 0; k <= L; ++k) vst<T, VEC>(ring(a, k, 0) + g0, z);
                if constexpr (kF32) {
                    T zero[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) zero[v] = T(0);
                    vst<T, VEC>(xi + g0, zero);
                }
            }
            if (tid == 0) {
#pragma unroll
                for (int q = 0; q < kMaxDots; ++q) s.G[0][q] = 0.0;
                s.G[0][2 * L] = 1.0;
                s.Ginv[0] = 1.0;
            }
        }
        PLCG_SYNC();

        // Coefficients of iteration 0 (fill phase: no dot products needed yet).
        // Afterwards, the coefficients of iteration i + 1 need the dots of
        // iteration i + 1 - l.  Serial mode (l = 1, or lookahead off): after the
        // barrier that ends iteration i, every CTA sums those partials and
        // thread 0 runs the scalar step while the others wait.  Lookahead mode
        // (l >= 2): those dots are already complete during iteration i, so the
        // last warp of every CTA computes them while the other warps sweep --
        // Alg. 2's overlap of the global reduction (MPI_Iallreduce ... MPI_Wait
        // l iterations later) with the local work, on one GPU.
        const bool la = (L >= 2) && a.lookahead;
        const int nsw = la ? kBlock - 32 : kBlock;   // threads that sweep
        if (tid == 0) scalar_step<T, L, kOolScalar, SC>(s, s.cfb[0], s.raw, a, 0, rn, tau, budget, kc, kn);
        __syncthreads();
        for (long long i = 0;; ++i) {
            const Coef<T> &cf = s.cfb[i & 1];
            if (cf.end >= 0) {
                // ---- final vector update of the segment
                if (cf.end != kSegNonfinite) {
                    for (int64_t u = grp.unit0(); u < nunits; u += grp.ustep()) {
                        const int64_t g0 = u * UNIT + (int64_t)tid * VEC;
                        if (g0 >= n) continue;
                        T xv[VEC], pv[VEC];
                        vld<T, VEC>(xi + g0, xv);
                        if (cf.fmode == 0) {
                            if (cf.f1 != T(0)) {
                                vld<T, VEC>(a.p + g0, pv);
#pragma unroll
                                for (int v = 0; v < VEC; ++v) xv[v] = fma(cf.f1, pv[v], xv[v]);
                            }
                        } else {
                            T vv[VEC];
                            vld<T, VEC>(cf.v0 + g0, vv);
                            if (cf.fmode == 1) {
                                vld<T, VEC>(a.p + g0, pv);
#pragma unroll
                                for (int v = 0; v < VEC; ++v) {
                                    xv[v] = fma(cf.f1, pv[v], xv[v]);
                                    const T pn = fma(cf.pv, vv[v], cf.pp * pv[v]);
                                    xv[v] = fma(cf.f2, pn, xv[v]);
                                }
                            } else {
#pragma unroll
                                for (int v = 0; v < VEC; ++v) xv[v] = fma(cf.f2, cf.pv * vv[v], xv[v]);
                            }
                        }
                        if constexpr (kF32) {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) a.x[g0 + v] += (double)xv[v];
                        } else {
                            vst<T, VEC>(xi + g0, xv);
                        }
                    }
                }
                iters += cf.kseg;
                last_end = cf.end;
                segments++;
                if (cf.end == kSegNonfinite) { status = kStNonfinite; goto finish; }
                recres = (cf.end == kSegLucky || cf.end == kSegBreakdown) ? 0.0
                       : fabs(s.zeta[cf.kseg & 1]);
                PLCG_SYNC();
                break;
            }

            if (la && tid >= nsw) {
                // scalar warp: the coefficients of iteration i + 1
                if (i + 1 >= L)
                    grp.template get_dots_warp<2 * L + 1>(a, s, (int)((i + 1 - L) % (L + 1)), s.raw2);
                if ((tid & 31) == 0)
                    scalar_step<T, L, kOolScalar, SC>(s, s.cfb[(i + 1) & 1], s.raw2, a, (int)(i + 1), rn, tau, budget,
                                                  kc, kn);
                __syncwarp();
            }
            // ---- one full iteration sweep: K1, K4, K5 (partials), K6.  A thread
            // owns RPT row groups of VEC rows per unit (stride kBlock * VEC) and
            // issues every load of all of them before any store (the vectors are
            // distinct, but the compiler cannot know), so its HBM/L2 reads
            // overlap in flight.
            // The coefficients live in shared memory and the vector stores go
            // through generic pointers the compiler cannot prove disjoint from
            // it, so every field read after a store is re-loaded.  The one-CTA
            // path (RPT > 1, few warps) copies them into registers; the grid
            // path keeps them in shared memory, where re-loads cost less than
            // the registers (and occupancy) a copy would take.
            using CoefRef = std::conditional_t<(RPT > 1), SweepCoef<T, L>, const Coef<T> &>;
            using StRef = std::conditional_t<(RPT > 1), StencilDesc, const StencilDesc &>;
            CoefRef C = cf;
            StRef st = a.st;
            const CsrDesc &csr = a.csr;
            T *const pvec = a.p;
            DotAcc<T, VEC> dac[2 * L + 1];
            const uint32_t nn = (uint32_t)n;                      // n < 2^31
            const uint32_t usw = (uint32_t)(nsw * VEC * RPT);      // rows per sweep unit
            const uint32_t nunits_s = (tid < nsw) ? (nn + usw - 1) / usw : 0u;
            // Steady state -- every iteration of a segment after the first l + 1:
            // the recurrences run, K6 updates p and x, z^(0)_{m-1} exists and the
            // K5 operands follow a fixed pattern.  That case gets its own loop
            // with those tests and the operand selection resolved at compile time.
            const bool steady = C.mode == 1 && C.k6 == 2 && C.prev0 && !d2;
            auto sweep = [&](auto steady_tag) {
                constexpr bool S = decltype(steady_tag)::value;
                const bool rec = S || C.mode == 1;
                const int k6 = S ? 2 : C.k6;
                const bool prev0 = S || C.prev0;
                int since_flush = 0;
                // 27-point tiles: the first unit's copies start here, each
                // following unit's at the top of the one before it
                const char *tclo = a.cf_lo, *tchi = a.cf_hi;
                int tb = 0;             // buffer of the current unit
                uint32_t stg_q = 0;     // bit b: buffer b's unit is staged (copies in flight or landed)
                // the steady sweep's vector operands ride along in the tile
                constexpr bool SV = S && kNV > 0;
                auto vsrc = [&](int j) -> const T * {
                    if (j == 0) return C.zl_prev;
                    if (j <= L) return C.cur[j - 1];
                    if (j <= 2 * L) return C.prv[j - 1 - L];
                    if (j == 2 * L + 1) return pvec;
                    if (j == 2 * L + 2) return static_cast<const T *>(xi);
                    return static_cast<const T *>(csr.dinv);
                };
                // stage unit uu (if it exists) in buffer bb
                auto tile_issue = [&](int bb, uint32_t uu) {
                    const bool more = uu < nunits_s;
                    const bool on = tile.issue(bb, more, more ? uu * usw : 0u, more ? min(uu * usw + usw, nn) : 0u,
                                               nsw);
                    stg_q = (stg_q & ~(1u << bb)) | ((on ? 1u : 0u) << bb);
                };
                if constexpr (kTile) {   // the first NB - 1 units
                    // z^(l)_i and the vectors were written by generic stores
                    // before the grid barrier that began this sweep; nothing
                    // the copies read is written during it.  One proxy fence
                    // per issuing thread orders those stores before all of
                    // the sweep's copies.
                    if (Tile::issues(nsw)) fence_proxy_async_all();
                    tile.prepare(SV, vsrc, st, static_cast<const T *>(csr.val), csr.stride, tclo, tchi, C.zl_cur,
                                 a.ws_lo, a.ws_hi, nsw);
                    if ((uint32_t)grp.unit0() < nunits_s)
                        for (int bb = 0; bb < Tile::NB - 1; ++bb)
                            tile_issue(bb, (uint32_t)grp.unit0() + (uint32_t)bb * (uint32_t)grp.ustep());
                }
                typename CsrStage<CT>::Rows rp_next{0, 0};   // the warp's next unit's row pointers
                if constexpr (kStage) {
                    const uint32_t w0 = (uint32_t)grp.unit0() * usw + (uint32_t)(tid & ~31);
                    if (a.stage && w0 < nn) rp_next = CsrStage<CT>::rows_load(csr, w0, min(w0 + 32u, nn));
                }
                for (uint32_t u = (uint32_t)grp.unit0(); u < nunits_s; u += (uint32_t)grp.ustep()) {
                    uint32_t g0[RPT];
                    bool ok[RPT];
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        g0[r] = u * usw + ((uint32_t)r * nsw + tid) * VEC;
                        ok[r] = g0[r] < nn;
                    }
                    bool stg = false;
                    int64_t e0s = 0, rs = 0, re = 0;
                    if constexpr (kStage) {   // this warp's 32 rows of the unit
                        const uint32_t w0 = u * usw + (uint32_t)(tid & ~31);
                        if (a.stage && w0 < nn) {
                            const typename CsrStage<CT>::Rows rp = rp_next;
                            const uint32_t wn = w0 + (uint32_t)grp.ustep() * usw;
                            if (u + (uint32_t)grp.ustep() < nunits_s && wn < nn)
                                rp_next = CsrStage<CT>::rows_load(csr, wn, min(wn + 32u, nn));
                            int64_t e0, e1;
                            CsrStage<CT>::rows_bounds(rp, &e0, &e1, &rs, &re);
                            stg = stage.stage_range(csr, e0, e1, &e0s, a.poll_limit, &a.out->abort);
                        }
                    }
                    T bw[13];   // the tiled unit's backward coefficients (row g0[0])
                    if constexpr (kTile) {    // the copies NB - 1 units ahead; this unit's tile
                        stg = (stg_q >> tb) & 1u;
                        tile_issue((tb + Tile::NB - 1) % Tile::NB,
                                   u + (uint32_t)(Tile::NB - 1) * (uint32_t)grp.ustep());
                        if (stg && ok[0]) tile.backward(g0[0], bw);
                        if (stg) tile.wait(tb, a.poll_limit, &a.out->abort);
                    }
                    // -- loads
                    T c[RPT][VEC], nb[RPT][VEC], zp[RPT][VEC], cur[RPT][L][VEC], pk[RPT][L][VEC];
                    T pv[RPT][VEC], xv[RPT][VEC];
                    T dg[RPT];   // Jacobi: a_gg, for u_{i+1} = M z^(l)_{i+1}
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) zp[r][v] = T(0);
                        dg[r] = T(1);
                        if (!ok[r]) continue;
                        if constexpr (kStage) {   // K1 operands
                            if (stg) {
                                c[r][0] = C.zl_cur[g0[r]];
                                nb[r][0] = csr_row_k<T, CT>(stage.col, stage.val, (uint32_t)(rs - e0s),
                                                            (uint32_t)(re - e0s), Ld1<T>{C.zl_cur});
                            } else {
                                op_parts<T, CT, VEC, OP>(st, csr, Ld1<T>{C.zl_cur}, g0[r], c[r], nb[r]);
                            }
                        } else if constexpr (kTile) {
                            // K1 from the tile after the loads below
                        } else {
                            op_parts<T, CT, VEC, OP>(st, csr, Ld1<T>{C.zl_cur}, g0[r], c[r], nb[r]);
                        }
                        if constexpr (kTile) {
                            if (SV && stg) {   // the steady sweep's vectors, from the tile
                                const int t = (int)(g0[r] - u * usw);
                                zp[r][0] = tile.vec(tb, 0)[t];
#pragma unroll
                                for (int k = 0; k < L; ++k) {
                                    cur[r][k][0] = tile.vec(tb, 1 + k)[t];
                                    pk[r][k][0] = tile.vec(tb, 1 + L + k)[t];
                                }
                                pv[r][0] = tile.vec(tb, 2 * L + 1)[t];
                                xv[r][0] = tile.vec(tb, 2 * L + 2)[t];
                                if constexpr (op_is_jacobi(OP)) {
                                    c[r][0] = tile.vec(tb, 2 * L + 3)[t];   // 1 / a_gg for now
                                    dg[r] = tile.diag(tb, t);                // a_gg: the diagonal slot
                                }
                                continue;
                            }
                            if constexpr (op_is_jacobi(OP)) {   // 1 / a_gg for now
                                if (stg) {
                                    c[r][0] = __ldg(static_cast<const T *>(csr.dinv) + g0[r]);
                                    dg[r] = tile.diag(tb, (int)(g0[r] - u * usw));
                                } else {
                                    c[r][0] = __ldg(static_cast<const T *>(csr.dinv) + g0[r]);
                                    dg[r] = coef_cast<T>(__ldg(static_cast<const CT *>(csr.diag) + g0[r]));
                                }
                            }
                        } else if constexpr (op_is_jacobi(OP)) {
                            // K1 with M = diag(A): z^(l)_{i+1} is built from M^{-1} A z^(l)_i
                            nb[r][0] *= __ldg(static_cast<const T *>(csr.dinv) + g0[r]);
                            dg[r] = coef_cast<T>(__ldg(static_cast<const CT *>(csr.diag) + g0[r]));
                        }
                        if (rec) {
                            vld<T, VEC>(C.zl_prev + g0[r], zp[r]);
#pragma unroll
                            for (int k = 0; k < L; ++k) vld<T, VEC>(C.cur[k] + g0[r], cur[r][k]);
#pragma unroll
                            for (int k = 0; k < L; ++k) {
                                if (k > 0 || prev0) {
                                    vld<T, VEC>(C.prv[k] + g0[r], pk[r][k]);
                                } else {
#pragma unroll
                                    for (int v = 0; v < VEC; ++v) pk[r][k][v] = T(0);
                                }
                            }
                        }
                        if (k6 == 2) {
                            vld<T, VEC>(pvec + g0[r], pv[r]);
                            vld<T, VEC>(xi + g0[r], xv[r]);
                        }
                    }
                    if constexpr (kTile) {   // K1 from the tile
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            if (!ok[r]) continue;
                            const T di = c[r][0];
                            if (stg) {
                                T zc;
                                nb[r][0] = tile.template row<T>(tb, (int)(g0[r] - u * usw), bw, &zc);
                                c[r][0] = zc;
                            } else {
                                op_parts<T, CT, VEC, OP>(st, csr, Ld1<T>{C.zl_cur}, g0[r], c[r], nb[r]);
                            }
                            if constexpr (op_is_jacobi(OP)) nb[r][0] *= di;
                        }
                    }
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        if (!ok[r]) continue;
                        // -- compute
                        T un[VEC], nw[L][VEC];
                        if (!rec) {
                            // u_{i+1} = A z^(l)_i - sigma_i z^(l)_i
#pragma unroll
                            for (int v = 0; v < VEC; ++v) un[v] = fma(kc - C.sig, c[r][v], kn * nb[r][v]);
                        } else {
                            // K4: z^(l)_{i+1} = (A z^(l)_i - gamma z^(l)_i - delta' z^(l)_{i-1}) / delta
                            // and z^(k)_{i-l+k+1}, k < l (Algorithm 1, K4)
                            const T uc = C.uc, un_nb = C.unb;
                            if (kScaled && S && C.unit) {
                                // scaled bases, steady state: the coefficients of nb
                                // and of each recurrence's U term are 1
#pragma unroll
                                for (int v = 0; v < VEC; ++v) un[v] = fma(uc, c[r][v], fma(C.bm, zp[r][v], nb[r][v]));
#pragma unroll
                                for (int k = 0; k < L; ++k)
#pragma unroll
                                    for (int v = 0; v < VEC; ++v) {
                                        const T up = (k == L - 1) ? c[r][v] : cur[r][k + 1][v];
                                        nw[k][v] = fma(C.ak[k], cur[r][k][v], fma(C.wb[k], pk[r][k][v], up));
                                    }
                            } else {
#pragma unroll
                                for (int v = 0; v < VEC; ++v)
                                    un[v] = fma(uc, c[r][v], fma(un_nb, nb[r][v], C.bm * zp[r][v]));
#pragma unroll
                                for (int k = 0; k < L; ++k)
#pragma unroll
                                    for (int v = 0; v < VEC; ++v) {
                                        const T up = (k == L - 1) ? c[r][v] : cur[r][k + 1][v];
                                        nw[k][v] = fma(up, C.wu[k], fma(C.ak[k], cur[r][k][v], C.wb[k] * pk[r][k][v]));
                                    }
                            }
                        }
                        // K6: p and the iterate (Algorithm 1, K6)
                        if (k6 == 1) {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) pv[r][v] = cur[r][0][v];
                        } else if (k6 == 2) {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                xv[r][v] = fma(C.zx, pv[r][v], xv[r][v]);
                                pv[r][v] = fma(C.pp, pv[r][v], cur[r][0][v]);
                            }
                        }
                        // -- stores
                        vst<T, VEC>(C.zl_new + g0[r], un);
                        if (!rec) {
                            for (int k = 0; k < C.ncopy; ++k) vst<T, VEC>(cf.cpy[k] + g0[r], un);
                        } else {
#pragma unroll
                            for (int k = 0; k < L; ++k) vst<T, VEC>(C.nw[k] + g0[r], nw[k]);
                        }
                        if (k6 >= 1) vst<T, VEC>(pvec + g0[r], pv[r]);
                        if (k6 == 2) vst<T, VEC>(xi + g0[r], xv[r]);
                        // -- K5: partial dot products with u_{i+1} = M z^(l)_{i+1}
                        // (M = I: z^(l)_{i+1} itself)
                        T uM[VEC];
#pragma unroll
                        for (int v = 0; v < VEC; ++v) uM[v] = op_is_jacobi(OP) ? un[v] * dg[r] : un[v];
#pragma unroll
                        for (int q = 0; q <= 2 * L; ++q) {
                            if (D1 && q < L) continue;
                            const int src = S ? steady_dot_src<L>(q) : C.dsrc[q];
                            if (src == 0) continue;
                            T o[VEC];
                            if (src == 1) {
                                vld<T, VEC>(cf.dptr[q] + g0[r], o);
                            } else {
#pragma unroll
                                for (int v = 0; v < VEC; ++v)
                                    o[v] = (src == 2) ? un[v] : (src == 3) ? nw[0][v] : (src == 4) ? c[r][v]
                                         : zp[r][v];
                            }
                            dac[q].add(uM, o);
                        }
                    }
                    if (++since_flush == kFlushUnits) {
#pragma unroll
                        for (int q = 0; q <= 2 * L; ++q)
                            if ((!D1 || q >= L) && (!S || steady_dot_src<L>(q) != 0)) dac[q].flush();   // dots in use
                        since_flush = 0;
                    }
                    tb = (tb + 1) % Tile::NB;
                }
            };
            if (steady) sweep(std::true_type{});
            else sweep(std::false_type{});
            double acc[2 * L + 1];
#pragma unroll
            for (int q = 0; q <= 2 * L; ++q) {
                if (q >= L || d2) dac[q].flush();   // positions < l: only with 2l+1 dots
                acc[q] = dac[q].acc;
            }
            spmvs++;
            // MPI_Iallreduce(..., req(i)): publish this CTA's partials in slot i mod (l+1)
            if (d2) {
                block_sum<2 * L + 1>(acc, s.red, s.out);
            } else {
                // the l+1 dots of Sec. 2.2 (positions l .. 2l); the others are
                // filled from the symmetry of G when the column is finalised
                double sub[L + 1];
#pragma unroll
                for (int q = 0; q <= L; ++q) sub[q] = acc[L + q];
                block_sum<L + 1>(sub, s.red, s.out + L);
                if (tid < L) s.out[tid] = 0.0;
            }
            grp.put_dots(a, s, (int)(i % (L + 1)), 2 * L + 1);
            PLCG_SYNC();
            if (!la) {   // MPI_Wait(req(i+1-l)) and the scalar step, serially (warp 0)
                if (tid < 32) {
                    if (i + 1 >= L)
                        grp.template get_dots_warp<2 * L + 1>(a, s, (int)((i + 1 - L) % (L + 1)), s.raw);
                    if (tid == 0)
                        scalar_step<T, L, kOolScalar, SC>(s, s.cfb[(i + 1) & 1], s.raw, a, (int)(i + 1), rn, tau,
                                                      budget, kc, kn);
                }
                __syncthreads();
            }
        }
    }
finish:
    if (grp.leader() && tid == 0)
        write_result(a, status, iters, spmvs, restarts, refinements, recres, normb, last_rn);
    __syncthreads();
#undef PLCG_SYNC
}

// ------------------------------------------------------------------------
// Classic CG (Hestenes-Stiefel) on one group: two synchronisations per
// iteration (after (p, Ap) and after (r, r)).  With the Jacobi preconditioner
// (kOpCsrJacobi) the recursive vector is z = M^{-1} r instead of r: q holds
// M^{-1} A p, z -= alpha q, and rho = (r, z) = sum a_gg z_g^2.  p lives in a ring of two
// vectors because the SpMV of step k reads neighbours of p_{k-1} while p_k is
// written.  q = A p is in a.p; the recursive residual is r itself on the FP64
// path and a.rc (FP32) on the FP32 path, whose inner iterate is the ring's
// third vector.
// ------------------------------------------------------------------------
template <typename T, int VEC, int OP, class Grp, int RPT = 1, typename CT = T>
__device__ void cg_body(const SolveArgs<T> &a, Smem<T> &s, Grp &grp)
{
    constexpr int UNIT = kBlock * VEC;
    constexpr int USWEEP = UNIT * RPT;
    constexpr bool kF32 = (sizeof(T) == 4);
    const int64_t n = a.n;
    const int64_t nunits = (n + UNIT - 1) / UNIT;
    const int tid = threadIdx.x;
    const T cC = (T)a.st.center, cO = (T)a.st.off;
    T *pr[2] = {a.zring, a.zring + n};
    T *q = a.p;
    std::conditional_t<(RPT > 1), StencilDesc, const StencilDesc &> st = a.st;
    const CsrDesc &csr = a.csr;
    T *rc = kF32 ? a.rc : reinterpret_cast<T *>(a.r);
    T *xi = kF32 ? a.zring + 2 * n : reinterpret_cast<T *>(a.x);
    const uint32_t nn = (uint32_t)n;   // n < 2^31
    // CSR on the whole grid, FP32: the SpMV sweep stages each unit's entries
    // (as in p(l)-CG).  FP64 CG runs without: its 3 CTAs per SM would not fit
    // the FP64 staging buffer (measured: 2 CTAs with staging are slower).
    constexpr bool kStage = op_is_csr(OP) && std::is_same<Grp, GridGroup<T>>::value && RPT == 1 &&
                            sizeof(T) == 4;
    extern __shared__ __align__(128) unsigned char plcg_dsm[];
    CsrStage<CT> stage(plcg_dsm);
    if constexpr (kStage) {
        stage.init();
        __syncthreads();
    }
    // structured 27-point operator on the whole grid, FP32: p_k = z_k +
    // beta p_{k-1} gets a sweep of its own (in place, in ring vector 0, which
    // carries the zero halos), and the SpMV reads p through the shared-memory
    // tiles of the p(l)-CG sweep -- one barrier more per iteration instead of
    // forming p at all 27 stencil points (Table 1 charges CG and p(l)-CG the
    // same SpMV)
    constexpr bool kTileCG = op_is_var27(OP) && std::is_same<Grp, GridGroup<T>>::value && RPT == 1 &&
                             sizeof(T) == 4 && sizeof(CT) == 4;
    // FP64 on the whole grid: the same separate p sweep, since GB300's FP64
    // units, not HBM, bound the FP64 sweeps and forming p on the fly costs an
    // FP64 FMA at every stencil point or matrix entry (one pass more, 7 of 18
    // FP64 instructions per row fewer on the 7-point stencil)
    constexpr bool kSepP = kTileCG || (sizeof(T) == 8 && std::is_same<Grp, GridGroup<T>>::value && RPT == 1);
    using Tile = Var27Tile<T, 0, kV27StageBwdCg>;
    Tile tile(plcg_dsm);
    if constexpr (kSepP) {
        pr[0] = pr[1] = a.zring;   // p updated in place
        if constexpr (kF32) xi = a.zring + 2 * a.vstride;
    }
    if constexpr (kTileCG) {
        tile.init(a.st, static_cast<const T *>(csr.val), csr.stride, kV27MergeZCg);
        __syncthreads();
        // zero the halo before ring vector 0 and the span after every ring
        // vector: the tiles' z copies reach into them (the grid barrier after
        // the first residual sweep orders these stores before any copy)
        const int64_t span = a.vstride - a.n, nzr = a.halo + (int64_t)a.nring * span;
        for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < nzr; e += (int64_t)gridDim.x * kBlock) {
            if (e < a.halo) {
                a.zring[e - a.halo] = T(0);
            } else {
                const int64_t i = (e - a.halo) / span;
                a.zring[i * a.vstride + a.n + (e - a.halo - i * span)] = T(0);
            }
        }
    }

    long long iters = 0, spmvs = 0, restarts = 0, refinements = 0, segments = 0;
    int last_end = kSegConverged;
    double normb = 0.0, recres = 0.0, last_rn = 0.0;
    int status = kStOk;

#define CG_SYNC()                                                                            \
    do {                                                                                     \
        if (!grp.sync(a, s)) {                                                               \
            status = kStTimeout;                                                             \
            goto finish;                                                                     \
        }                                                                                    \
    } while (0)

    for (;;) {
        residual_sweep<T, VEC, OP, Grp, CT>(a, s, grp);
        grp.put_norms(a, s);
        spmvs++;
        CG_SYNC();
        grp.get_norms(a, s);
        if (segments == 0) normb = sqrt(s.out[0]);
        const double rn = sqrt(s.out[1]);
        last_rn = rn;
        if (normb == 0.0) {
            for (int64_t u = grp.unit0(); u * kBlock < n; u += grp.ustep()) {
                const int64_t g = u * kBlock + tid;
                if (g < n) a.x[g] = 0.0;
            }
            status = kStOk;
            break;
        }
        if (!isfinite(normb) || !isfinite(rn)) { status = kStNonfinite; break; }
        if (rn < a.rtol * normb) { status = kStOk; break; }
        if (iters >= a.maxit) { status = kStMaxit; break; }
        if (segments > 0) {
            if (kF32 && last_end == kSegConverged) {
                if (++refinements > kMaxRefine) { status = kStMaxit; break; }
            } else {
                if (restarts >= a.max_restarts) {
                    status = (last_end == kSegMaxit) ? kStMaxit : kStBreakdown;
                    break;
                }
                restarts++;
            }
        }
        const double tau = kF32 ? fmax(a.inner_floor * rn, 0.5 * a.rtol * normb) : a.rtol * normb;
        const long long budget = a.maxit - iters;
        double rr = rn * rn;
        if constexpr (kF32) {
            // rc = (float) r (Jacobi: (float) M^{-1} r), d = 0, rr from the
            // rounded values
            DotAcc<T, VEC> d0;
            for (int64_t u = grp.unit0(); u < nunits; u += grp.ustep()) {
                const int64_t g0 = u * UNIT + (int64_t)tid * VEC;
                if (g0 >= n) continue;
                T z[VEC], zero[VEC], zm[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    if constexpr (op_is_jacobi(OP)) {
                        z[v] = (T)(a.r[g0 + v] * __ldg(a.dinv64 + g0 + v));
                        zm[v] = z[v] * coef_cast<T>(__ldg(static_cast<const CT *>(csr.diag) + g0 + v));
                    } else {
                        z[v] = (T)a.r[g0 + v];
                        zm[v] = z[v];
                    }
                    zero[v] = T(0);
                }
                d0.add(zm, z);
                d0.flush();
                vst<T, VEC>(rc + g0, z);
                vst<T, VEC>(xi + g0, zero);
            }
            double acc[1] = {d0.acc};
            block_sum<1>(acc, s.red, s.out);
            grp.put_dots(a, s, 0, 1);
            CG_SYNC();
            grp.template get_dots<1>(a, s, 0, s.raw);
            rr = s.raw[0];
        } else if constexpr (op_is_jacobi(OP)) {
            // FP64 path: z = M^{-1} r in r's place; rr = (r, M^{-1} r) = rn^2
            for (int64_t u = grp.unit0(); u < nunits; u += grp.ustep()) {
                const int64_t g = u * UNIT + (int64_t)tid;
                if (g < n) a.r[g] *= __ldg(a.dinv64 + g);
            }
            CG_SYNC();
        }
        long long k = 0;
        int end;
        double beta = 0.0;
        for (;;) {
            if (!isfinite(rr)) { end = kSegNonfinite; break; }
            if (sqrt(rr) < tau) { end = kSegConverged; break; }
            if (k >= budget) { end = kSegMaxit; break; }
            // ---- p_k = r_k + beta_{k-1} p_{k-1};  q = A p_k;  (p_k, q)
            T *pn = pr[(k + 1) & 1];
            const T *po = pr[k & 1];
            DotAcc<T, VEC> d1;
            int since_flush = 0;
            const int64_t nunits_s = (n + USWEEP - 1) / USWEEP;
            if constexpr (kSepP) {
                // p_k in place
                for (int64_t u = grp.unit0(); u < nunits; u += grp.ustep()) {
                    const int64_t g0 = u * UNIT + (int64_t)tid * VEC;
                    if (g0 >= n) continue;
                    T pv[VEC], zv[VEC];
                    vld<T, VEC>(rc + g0, zv);
                    if (k == 0) {
                        vst<T, VEC>(pn + g0, zv);
                    } else {
                        vld<T, VEC>(pn + g0, pv);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) pv[v] = fma((T)beta, pv[v], zv[v]);
                        vst<T, VEC>(pn + g0, pv);
                    }
                }
                CG_SYNC();
            }
            if constexpr (kSepP && !kTileCG) {
                // q = A p_k and (p_k, A p_k) from the stored p
                for (uint32_t u = (uint32_t)grp.unit0(); u < (uint32_t)nunits; u += (uint32_t)grp.ustep()) {
                    const uint32_t g0 = u * (uint32_t)UNIT + (uint32_t)tid * VEC;
                    if (g0 >= nn) continue;
                    T c[VEC], w[VEC];
                    op_apply<T, CT, VEC, OP>(st, csr, cC, cO, Ld1<T>{pn}, g0, c, w);
                    d1.add(c, w);
                    if constexpr (op_is_jacobi(OP)) w[0] *= __ldg(static_cast<const T *>(csr.dinv) + g0);
                    vst<T, VEC>(q + g0, w);
                    if (++since_flush == kFlushUnits) { d1.flush(); since_flush = 0; }
                }
            } else if constexpr (kTileCG) {
                const uint32_t usw = (uint32_t)kBlock;
                int tb = 0;
                uint32_t stg_q = 0;
                auto novec = [](int) -> const T * { return nullptr; };
                auto tile_issue = [&](int bb, uint32_t uu) {
                    const bool more = uu < (uint32_t)nunits;
                    const bool on = tile.issue(bb, more, more ? uu * usw : 0u,
                                               more ? min(uu * usw + usw, nn) : 0u, kBlock);
                    stg_q = (stg_q & ~(1u << bb)) | ((on ? 1u : 0u) << bb);
                };
                // p was written by generic stores before the barrier above; one
                // proxy fence per issuing thread orders them before the copies
                if (Tile::issues(kBlock)) fence_proxy_async_all();
                tile.prepare(false, novec, st, static_cast<const T *>(csr.val), csr.stride, a.cf_lo, a.cf_hi, pn,
                             a.ws_lo, a.ws_hi, kBlock);
                if ((uint32_t)grp.unit0() < (uint32_t)nunits)
                    for (int bb = 0; bb < Tile::NB - 1; ++bb)
                        tile_issue(bb, (uint32_t)grp.unit0() + (uint32_t)bb * (uint32_t)grp.ustep());
                for (uint32_t u = (uint32_t)grp.unit0(); u < (uint32_t)nunits; u += (uint32_t)grp.ustep()) {
                    const bool stg = (stg_q >> tb) & 1u;
                    tile_issue((tb + Tile::NB - 1) % Tile::NB, u + (uint32_t)(Tile::NB - 1) * (uint32_t)grp.ustep());
                    const uint32_t g = u * usw + (uint32_t)tid;
                    T bw[13];
                    if (stg && g < nn) tile.backward(g, bw);
                    if (stg) tile.wait(tb, a.poll_limit, &a.out->abort);
                    if (g < nn) {
                        T c[VEC], w[VEC];
                        T mi = T(1);   // Jacobi: 1 / a_gg
                        if (stg) {
                            T zc;
                            w[0] = tile.template row<T>(tb, tid, bw, &zc);
                            c[0] = zc;
                            // the correctly rounded reciprocal of the diagonal
                            // slot: the stored inverse diagonal's value
                            if constexpr (op_is_jacobi(OP)) mi = __frcp_rn(tile.diag(tb, tid));
                        } else {
                            op_parts<T, CT, VEC, OP>(st, csr, Ld1<T>{pn}, g, c, w);
                            if constexpr (op_is_jacobi(OP)) mi = __ldg(static_cast<const T *>(csr.dinv) + g);
                        }
                        d1.add(c, w);
                        if constexpr (op_is_jacobi(OP)) w[0] *= mi;   // q = M^{-1} A p
                        vst<T, VEC>(q + g, w);
                    }
                    if (++since_flush == kFlushUnits) { d1.flush(); since_flush = 0; }
                    tb = (tb + 1) % Tile::NB;
                }
            } else {
                typename CsrStage<CT>::Rows rp_next{0, 0};   // the warp's next unit's row pointers
                if constexpr (kStage) {
                    const uint32_t w0 = (uint32_t)grp.unit0() * USWEEP + (uint32_t)(tid & ~31);
                    if (a.stage && w0 < nn) rp_next = CsrStage<CT>::rows_load(csr, w0, min(w0 + 32u, nn));
                }
                for (uint32_t u = (uint32_t)grp.unit0(); u < (uint32_t)nunits_s; u += (uint32_t)grp.ustep()) {
                    T c[RPT][VEC], w[RPT][VEC], mi[RPT];
                    uint32_t g0[RPT];
                    bool stg = false;
                    int64_t e0s = 0, rs = 0, re = 0;
                    if constexpr (kStage) {   // this warp's 32 rows of the unit
                        const uint32_t w0 = u * USWEEP + (uint32_t)(tid & ~31);
                        if (a.stage && w0 < nn) {
                            const typename CsrStage<CT>::Rows rp = rp_next;
                            const uint32_t wn = w0 + (uint32_t)grp.ustep() * USWEEP;
                            if (u + (uint32_t)grp.ustep() < (uint32_t)nunits_s && wn < nn)
                                rp_next = CsrStage<CT>::rows_load(csr, wn, min(wn + 32u, nn));
                            int64_t e0, e1;
                            CsrStage<CT>::rows_bounds(rp, &e0, &e1, &rs, &re);
                            stg = stage.stage_range(csr, e0, e1, &e0s, a.poll_limit, &a.out->abort);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        g0[r] = u * USWEEP + ((uint32_t)r * kBlock + tid) * VEC;
                        if (g0[r] >= nn) continue;
                        if (stg) {
                            const uint32_t k0 = (uint32_t)(rs - e0s), k1 = (uint32_t)(re - e0s);
                            if (k == 0) {
                                const LdFirst<T> ld{rc};
                                c[r][0] = ld.one(g0[r]);
                                w[r][0] = csr_row_k<T, CT>(stage.col, stage.val, k0, k1, ld);
                            } else {
                                const LdAxpy<T> ld{rc, po, (T)beta};
                                c[r][0] = ld.one(g0[r]);
                                w[r][0] = csr_row_k<T, CT>(stage.col, stage.val, k0, k1, ld);
                            }
                        } else if (k == 0) {
                            op_apply<T, CT, VEC, OP>(st, csr, cC, cO, LdFirst<T>{rc}, g0[r], c[r], w[r]);
                        } else {
                            op_apply<T, CT, VEC, OP>(st, csr, cC, cO, LdAxpy<T>{rc, po, (T)beta}, g0[r], c[r], w[r]);
                        }
                        if constexpr (op_is_jacobi(OP))
                            mi[r] = __ldg(static_cast<const T *>(csr.dinv) + g0[r]);
                    }
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        if (g0[r] >= nn) continue;
                        vst<T, VEC>(pn + g0[r], c[r]);
                        d1.add(c[r], w[r]);
                        if constexpr (op_is_jacobi(OP)) w[r][0] *= mi[r];   // q = M^{-1} A p
                        vst<T, VEC>(q + g0[r], w[r]);
                    }
                    if (++since_flush == kFlushUnits) { d1.flush(); since_flush = 0; }
                }
            }
            d1.flush();
            spmvs++;
            double acc[1] = {d1.acc};
            block_sum<1>(acc, s.red, s.out);
            grp.put_dots(a, s, 0, 1);
            CG_SYNC();
            grp.template get_dots<1>(a, s, 0, s.raw);
            const double pq = s.raw[0];
            if (!(pq > 0.0)) { end = isfinite(pq) ? kSegBreakdown : kSegNonfinite; break; }
            const double alpha = rr / pq;
            const T al = (T)alpha;
            // ---- x += alpha p; r -= alpha q; (r, r)
            DotAcc<T, VEC> d2;
            since_flush = 0;
            for (uint32_t u = (uint32_t)grp.unit0(); u < (uint32_t)nunits_s; u += (uint32_t)grp.ustep()) {
                T pv[RPT][VEC], qv[RPT][VEC], xv[RPT][VEC], rv[RPT][VEC], dv[RPT][VEC];
                uint32_t g0[RPT];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    g0[r] = u * USWEEP + ((uint32_t)r * kBlock + tid) * VEC;
                    if (g0[r] >= nn) continue;
                    vld<T, VEC>(pn + g0[r], pv[r]);
                    vld<T, VEC>(q + g0[r], qv[r]);
                    vld<T, VEC>(xi + g0[r], xv[r]);
                    vld<T, VEC>(rc + g0[r], rv[r]);
                    if constexpr (op_is_jacobi(OP)) {
                        CT dc[VEC];
                        vldg<CT, VEC>(static_cast<const CT *>(csr.diag) + g0[r], dc);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) dv[r][v] = coef_cast<T>(dc[v]);
                    }
                }
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    if (g0[r] >= nn) continue;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        xv[r][v] = fma(al, pv[r][v], xv[r][v]);
                        rv[r][v] = fma(-al, qv[r][v], rv[r][v]);
                    }
                    vst<T, VEC>(xi + g0[r], xv[r]);
                    vst<T, VEC>(rc + g0[r], rv[r]);
                    if constexpr (op_is_jacobi(OP)) {   // rho = (r, z) = sum a_gg z_g^2
#pragma unroll
                        for (int v = 0; v < VEC; ++v) dv[r][v] *= rv[r][v];
                        d2.add(dv[r], rv[r]);
                    } else {
                        d2.add(rv[r], rv[r]);
                    }
                }
                if (++since_flush == kFlushUnits) { d2.flush(); since_flush = 0; }
            }
            d2.flush();
            double acc2[1] = {d2.acc};
            block_sum<1>(acc2, s.red, s.out);
            grp.put_dots(a, s, 1, 1);
            CG_SYNC();
            grp.template get_dots<1>(a, s, 1, s.raw);
            const double rr_new = s.raw[0];
            beta = rr_new / rr;
            if (a.trace && segments == 0 && k < a.trace_cap && grp.leader() && tid == 0) {
                a.trace[2 * k] = alpha;   // the Lanczos coefficients of the (preconditioned) operator
                a.trace[2 * k + 1] = beta;
            }
            rr = rr_new;
            ++k;
        }
        iters += k;
        last_end = end;
        segments++;
        recres = sqrt(rr);
        if (end == kSegNonfinite) { status = kStNonfinite; goto finish; }
        if constexpr (kF32) {   // x += d
            for (int64_t u = grp.unit0(); u < nunits; u += grp.ustep()) {
                const int64_t g0 = u * UNIT + (int64_t)tid * VEC;
                if (g0 >= n) continue;
                T xv[VEC];
                vld<T, VEC>(xi + g0, xv);
#pragma unroll
                for (int v = 0; v < VEC; ++v) a.x[g0 + v] += (double)xv[v];
            }
        }
        CG_SYNC();
    }
finish:
    if (grp.leader() && tid == 0)
        write_result(a, status, iters, spmvs, restarts, refinements, recres, normb, last_rn);
    __syncthreads();
#undef CG_SYNC
}

// ------------------------------------------------------------------------
// Single-system kernels: the whole grid solves one system (cooperative
// launch, so that every CTA is resident and the grid barrier can complete).
// ------------------------------------------------------------------------
// CTAs per SM the register budget is sized for: three for FP32 with l <= 2
// and for the FP64 p(1)-CG stencil sweep with scaled bases and two rows per
// thread (latency-bound once its neighbour sum runs on the integer units:
// 3D 256^3 161.7 -> 138.5 ms at 85 registers with 72 bytes of spills,
// against 128 registers at two CTAs per SM), two otherwise; the 27-point tiles' buffers (about 47 KB each) leave room
// for one CTA per SM with four of them (two with two).
template <typename T, int L, int OP, bool SC = false, int VEC = 1>
constexpr int kPlcgMinBlocks = (sizeof(T) == 4 && op_is_var27(OP)) ? 2
                               : (sizeof(T) == 4 && L <= 2)       ? 3
                               : (SC && L == 1 && OP == kOpStencil && VEC == 2) ? 3
                                                                                : 2;

// CT: the stored type of the matrix values (T, or float under FP64 vectors:
// the FP32-matrix path).
template <typename T, int L, int VEC, int OP, bool SC = false, typename CT = T>
__global__ void __launch_bounds__(kBlock, (kPlcgMinBlocks<T, L, OP, SC, VEC>))
plcg_kernel(SolveArgs<T> a)
{
    __shared__ Smem<T> s;
    GridGroup<T> grp;
    plcg_body<T, L, VEC, OP, GridGroup<T>, 1, SC, CT>(a, s, grp);
}

template <typename T, int VEC, int OP, typename CT = T>
__global__ void __launch_bounds__(kBlock, 3) cg_kernel(SolveArgs<T> a)
{
    __shared__ Smem<T> s;
    GridGroup<T> grp;
    cg_body<T, VEC, OP, GridGroup<T>, 1, CT>(a, s, grp);
}

// Small systems: the grid is one thread-block cluster (ClusterGroup), launched
// with a cluster dimension equal to the grid.  Every CTA passes a last
// cluster barrier before it exits, so none leaves while another may still
// read its shared memory.
template <typename T, int L, int VEC, int OP, bool CG>
__global__ void __launch_bounds__(kBlock, 1) plcg_cluster_kernel(SolveArgs<T> a)
{
    __shared__ Smem<T> s;
    ClusterGroup<T> grp;
    if constexpr (CG) cg_body<T, VEC, OP, ClusterGroup<T>>(a, s, grp);
    else plcg_body<T, L, VEC, OP, ClusterGroup<T>>(a, s, grp);
    cluster_barrier();
}

// ------------------------------------------------------------------------
// Batched kernel: many independent stencil systems in one persistent
// (cooperative) launch.  The first ngangs * G CTAs form gangs of G CTAs that
// take the systems of the "large" list (largest estimated work first) and
// solve each one together; every CTA -- gang members once that list is
// exhausted -- then takes systems of the "small" list one per CTA, with
// __syncthreads as its barrier.  Converged systems retire at once and free
// their CTA or gang for the next system.
// ------------------------------------------------------------------------
// Launch shape of the batched kernel, per method: CTAs per SM (the
// register budget), row groups per thread and vector width VW in the
// one-CTA path, where a CTA streams a whole system and latency is hidden by
// warps and by loads in flight per thread.  VW = 2: each thread takes pairs
// of adjacent rows as 2-wide vectors in systems whose nx is even (the
// others take the row-group path).  Chosen by timing the 4096-system
// workload on GB300 over 2-6 CTAs per SM, 1, 2 or 4 row groups and vector
// widths 1 and 2: 4 CTAs per SM for every method; 4 row groups for classic
// CG and p(1)-CG, 1 for p(l >= 2)-CG (FP64); in FP32, 2-wide rows for p(1)-
// and p(2)-CG (44.8 and 59.4 ms against 47.0 and 60.8 ms with one row per
// thread), 2-wide rows being slower for p(3)-CG (77.4 ms against 74.6) and
// classic CG (58.9 against 56.9), and 4-wide rows spilling registers.
template <int L, bool CG> constexpr int kBatchMinBlocks = 4;
template <int L, bool CG> constexpr int kBatchRPT = (CG || L == 1) ? 4 : 1;
// Other launch shapes (CTAs per SM the registers are sized for, row groups
// per thread, vector width) are instantiated for the FP32 path; the batched
// autotuner picks among them (plcg_set_batched_launch).

template <typename T>
__device__ __forceinline__ void batch_args(const BatchArgs<T> &ba, const BatchSys &sy, T *ws,
                                           SolveArgs<T> &a)
{
    a = ba.proto;
    a.n = (int64_t)sy.nx * sy.ny * sy.nz;
    a.st.dim = sy.dim;
    a.st.nx = sy.nx;
    a.st.ny = sy.ny;
    a.st.nz = sy.nz;
    a.st.dnx = sy.dnx;
    a.st.dny = sy.dny;
    a.st.center = sy.center;
    a.st.off = sy.off;
    a.b = sy.b;
    a.x = sy.x;
    a.out = sy.out;
    for (int j = 0; j < kMaxL; ++j) a.sigma[j] = sy.sigma[j];
    // workspace: ring vectors, p, rc (type T), then r (FP64)
    const int64_t nv = a.n;
    a.zring = ws;
    a.vstride = nv;
    int nvec = 0;
    for (int j = 0; j <= kMaxL; ++j) nvec += (j <= a.l) ? a.depth[j] : 0;
    if (a.method == 1) nvec = 3;
    a.p = ws + (size_t)nvec * nv;
    a.rc = a.p + nv;
    a.r = reinterpret_cast<double *>(reinterpret_cast<char *>(ws) +
                                     ((((size_t)(nvec + 2) * nv * sizeof(T)) + 255) / 256) * 256);
}

template <typename T, int L, bool CG, int MINB = kBatchMinBlocks<L, CG>, int RPT = kBatchRPT<L, CG>, int VW = 1>
__global__ void __launch_bounds__(kBlock, MINB) batched_kernel(BatchArgs<T> ba)
{
    __shared__ Smem<T> s;
    __shared__ int s_next;
    // the current system's arguments, in shared memory: every thread reads
    // the same fields, and a per-thread copy (~600 bytes) in local memory
    // would not stay in L1 with 1024 threads per SM
    __shared__ SolveArgs<T> sa;
    const int b = blockIdx.x;
    if (b == 0 && threadIdx.x == 0) *ba.t0 = global_timer_ns();
    if (b < ba.ngangs * ba.G) {
        const int gang = b / ba.G;
        GangGroup<T> grp;
        grp.rank = b % ba.G;
        grp.G = ba.G;
        grp.bar = ba.gbar + (size_t)gang * 32;
        grp.epoch = 0;
        grp.part = ba.gpart + (size_t)gang * (kMaxL + 1) * ba.G * kMaxDots;
        grp.npart = ba.gnpart + (size_t)gang * ba.G * kNormSlots;
        grp.abort_flag = ba.gabort + gang;
        grp.limit = ba.proto.poll_limit;
        T *ws = reinterpret_cast<T *>(ba.gws + (size_t)gang * ba.gws_stride);
        for (;;) {
            if (grp.rank == 0 && threadIdx.x == 0) {
                const int k = atomicAdd(ba.ctr_large, 1);
                ba.gslot[gang] = (k < ba.nlarge) ? ba.order_large[k] : -1;
            }
            if (!grp.sync(ba.proto, s)) return;   // a broken gang barrier ends this gang
            if (threadIdx.x == 0) s_next = ld_volatile(ba.gslot + gang);
            __syncthreads();
            const int sysi = s_next;
            if (sysi < 0) break;
            if (threadIdx.x == 0) batch_args(ba, ba.sys[sysi], ws, sa);
            __syncthreads();
            if constexpr (CG) cg_body<T, 1, kOpStencil>(sa, s, grp);
            else plcg_body<T, L, 1, kOpStencil, GangGroup<T>, 1, false, T, true>(sa, s, grp);
            if (ld_volatile(grp.abort_flag)) return;
            // every member has read gslot before the leader overwrites it: they
            // all passed the solve's own barriers since reading it
        }
    }
    T *ws = reinterpret_cast<T *>(ba.ws + (size_t)b * ba.ws_stride);
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(ba.ctr_small, 1);
        __syncthreads();
        const int k = s_next;
        __syncthreads();
        if (k >= ba.nsmall) return;
        if (threadIdx.x == 0) batch_args(ba, ba.sys[ba.order_small[k]], ws, sa);
        __syncthreads();
        BlockGroup<T> grp;
        // VW rows per thread need nx % VW == 0 (a vector never straddles two
        // grid lines); the ring vectors (n = nx * ny * nz apart), b and x
        // (16-byte aligned) are then aligned for the vector loads
        if (VW > 1 && sa.st.nx % VW == 0) {
            if constexpr (CG) cg_body<T, VW, kOpStencil, BlockGroup<T>, 1>(sa, s, grp);
            else plcg_body<T, L, VW, kOpStencil, BlockGroup<T>, 1, false, T, true>(sa, s, grp);
        } else {
            if constexpr (CG) cg_body<T, 1, kOpStencil, BlockGroup<T>, RPT>(sa, s, grp);
            else plcg_body<T, L, 1, kOpStencil, BlockGroup<T>, RPT, false, T, true>(sa, s, grp);
        }
    }
}

}  // namespace plcg
