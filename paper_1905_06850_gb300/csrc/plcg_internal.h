// plcg_internal.h -- structures shared by the host side of libplcg.so and its
// kernels.  Not part of the public ABI (include/plcg.h is).
#pragma once

#include <stdint.h>

namespace plcg {

constexpr int kMaxL = 8;                  // largest pipeline length l
constexpr int kMaxDots = 2 * kMaxL + 1;   // dot products per iteration (Algorithm 1, K5)
constexpr int kBlock = 256;               // threads per CTA of the persistent solver
constexpr int kNormSlots = 2;             // doubles per CTA in the norm partials

// Operators: constant-coefficient stencil, CSR, the structured symmetric
// 27-point variable-coefficient stencil (diagonal + 13 forward weights per
// cell); the *Jacobi kinds add the preconditioner M = diag(A) (Sec. 2.2).
enum OpKind : int { kOpStencil = 0, kOpCsr = 1, kOpCsrJacobi = 2, kOpVar27 = 3, kOpVar27Jacobi = 4 };
#ifdef __CUDACC__
#define PLCG_HD __host__ __device__
#else
#define PLCG_HD
#endif
PLCG_HD constexpr bool op_is_csr(int op) { return op == kOpCsr || op == kOpCsrJacobi; }
PLCG_HD constexpr bool op_is_var27(int op) { return op == kOpVar27 || op == kOpVar27Jacobi; }
PLCG_HD constexpr bool op_is_jacobi(int op) { return op == kOpCsrJacobi || op == kOpVar27Jacobi; }

// End reasons of one segment (a run of Algorithm 1 from a residual).
enum SegEnd : int { kSegConverged = 0, kSegMaxit = 1, kSegBreakdown = 2, kSegLucky = 3,
                    kSegNonfinite = 4 };

// Device-side result of one solve; written by CTA 0, thread 0.
struct DevResult {
    int status;              // plcg_status
    int abort;               // set by any CTA whose bounded wait expired
    long long iters;
    long long spmvs;
    long long restarts;
    long long refinements;
    double recursive_relres;
    double true_relres;
    unsigned long long t_end_ns;   // device global timer when the result was written
};

// Division of a 32-bit unsigned x < 2^31 by an invariant d >= 1 with one
// multiply-high, an add and a shift: Granlund & Montgomery, "Division by
// invariant integers using multiplication" (PLDI 1994): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// x / d = (umulhi(x, m) + x) >> l (no overflow since x < 2^31).
struct FastDivU32 {
    uint32_t m;
    uint32_t s;
};

inline FastDivU32 make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
    return FastDivU32{(uint32_t)m, l};
}

// Matrix-free constant-coefficient Dirichlet stencil (5-point 2D / 7-point 3D).
struct StencilDesc {
    int dim;
    int nx, ny, nz;
    double center;   // includes the diagonal shift
    double off;
    FastDivU32 dnx, dny;   // division by nx and by ny
};

// CSR arrays in device memory; val, dinv and diag are float or double (the
// kernel's T).  dinv / diag (1 / a_rr and a_rr) are set for the Jacobi kinds.
// The structured 27-point operator keeps its [14][n] coefficients in val.
struct CsrDesc {
    const int64_t *rowptr;
    const int32_t *col;
    const void *val;
    const void *dinv;
    const void *diag;
    int64_t stride;           // structured 27-point: elements between coefficient arrays
};

// Everything one persistent solve needs (passed by value to the kernel).
template <typename T>
struct SolveArgs {
    int64_t n;
    StencilDesc st;
    CsrDesc csr;
    const double *b;          // FP64 right-hand side
    double *x;                // FP64 iterate (in: x0)
    const double *dinv64;     // kOpCsrJacobi: FP64 1 / a_rr (natural norms, M^{-1} r)
    double *r;                // FP64 residual b - A x
    T *zring;                 // ring storage of the l+1 bases (p(l)-CG) / p ring (CG)
    int64_t vstride;          // elements between consecutive ring vectors
    int depth[kMaxL + 1];     // ring depth of basis k
    FastDivU32 ddiv[kMaxL + 1];   // division by depth[k] (ring slots)
    int64_t base[kMaxL + 1];  // offset (in vectors) of basis k's ring
    T *p;                     // search direction p (p(l)-CG) / q = A p (CG)
    T *rc;                    // CG: the recursive residual in T (FP32 path)
    double *part;             // dot partials [(l+1) slots][P][kMaxDots]
    double *npart;            // norm partials [P][kNormSlots]
    unsigned int *bar;        // grid barrier arrival counter
    DevResult *out;
    // parameters
    int method;               // 0 = p(l)-CG, 1 = CG
    int l;
    double sigma[kMaxL];
    double rtol;
    long long maxit;
    int dots_2l1;
    int max_restarts;
    double inner_floor;       // FP32 path: floor of the inner relative tolerance
    int fp32;                 // 1: T = float with FP64 outer refinement
    unsigned long long poll_limit;
    int force_timeout;
    int lookahead;            // l >= 2: compute the next iteration's scalars during the sweep
    int cluster;              // > 0: the grid is one thread-block cluster of this many CTAs
    unsigned dsmem;           // dynamic shared memory of the launch (CSR / 27-point staging)
    const char *ws_lo, *ws_hi;   // the solve's workspace (bounds for staged copies)
    const char *cf_lo, *cf_hi;   // structured 27-point: the coefficient allocation (same)
    int64_t halo;             // structured 27-point: zero elements before ring vector 0 (and
                              // at least as many after every ring vector)
    int nring;                // ring vectors in zring
    int stage;                // CSR kernels: stage each unit's entries (rows long enough to pay)
    double *trace;            // CG: alpha_k, beta_k of the first segment (spectrum estimates), or null
    int trace_cap;            // pairs trace can hold
};

// Structured 27-point tiles: per sweep unit, shared-memory slots of
// kV27Slot elements -- the diagonal and 13 forward coefficient segments, with
// SB (staged backward) the 13 backward segments (forward array k at rows
// g - d_k), and nine slots' room for z around the unit (the 9 line segments,
// or 3 plane segments) -- and, for l <= 3, v27_vec_slots(l, jacobi) slots of
// the vector operands the steady-state p(l)-CG sweep streams (z^(l)_{i-1},
// the l current and l previous z^(k), p, the iterate and, with Jacobi,
// 1/a_gg; a_gg is the diagonal slot).  Without SB the backward coefficients
// come through L2 (another unit's forward copies bring them there shortly
// before or after) and the smaller tiles leave room for a third buffer.
// v27_bufs(SB) buffers, each with its mbarrier: the unit being computed and
// the next ones in flight.  The dynamic shared memory starts with the
// mbarriers, then (without SB) the 13 base pointers of the backward loads,
// then the buffers.
constexpr int kV27Slot = 256 + 16;
PLCG_HD constexpr int v27_bufs(bool sb) { return sb ? 2 : 3; }
PLCG_HD constexpr int v27_op_slots(bool sb) { return 14 + (sb ? 13 : 0) + 9; }
PLCG_HD constexpr unsigned v27_hdr(bool sb) { return 16u * ((unsigned)(v27_bufs(sb) + 1) / 2u) + (sb ? 0u : 112u); }
// the choice per kernel family (measured on GB300, 128^3 heterogeneous
// operator, Jacobi): fully staged tiles in two buffers for both, p(l)-CG
// (p(1) 13.0 vs 13.6 ms through L2 with three buffers; p(3)'s three buffers
// do not fit two CTAs per SM) and classic CG (19.4 vs 20.6 ms)
constexpr bool kV27StageBwdPlcg = true;
constexpr bool kV27StageBwdCg = true;
// z staged by plane (three copies per unit) where a plane's three lines fit,
// else by line (nine); measured: p(l)-CG 128^3 Jacobi p(1) 13.07 -> 12.55 ms
// by plane, classic CG's SpMV 19.43 (by line) vs 21.56 ms (by plane)
constexpr bool kV27MergeZPlcg = true;
constexpr bool kV27MergeZCg = false;

// The 13 forward offsets (dz, dy, dx) of the structured 27-point operator,
// lexicographic (the order of its coefficient arrays 1..13).
PLCG_HD constexpr int v27_dz(int k) { return k < 4 ? 0 : 1; }
PLCG_HD constexpr int v27_dy(int k) { return k == 0 ? 0 : k < 4 ? 1 : k < 7 ? -1 : k < 10 ? 0 : 1; }
PLCG_HD constexpr int v27_dx(int k) { return k == 0 ? 1 : k < 4 ? k - 2 : (k - 4) % 3 - 1; }

// Zero elements kept before the structured 27-point operator's coefficient
// arrays and its solves' ring vectors, and at least as many after each of
// them: more than the largest offset nx*ny + nx + 1 plus the 16-byte rounding
// of a staged copy, in whole 256-byte groups.  A tile's copies then never
// leave an array and its zero margins.
PLCG_HD constexpr int64_t v27_halo(int64_t nx, int64_t ny) { return (nx * ny + nx + 8 + 63) / 64 * 64; }
constexpr int v27_vec_slots(int l, bool jacobi)
{
    return l <= 3 ? 2 * l + 3 + (jacobi ? 1 : 0) : 0;
}
constexpr unsigned v27_tile_bytes_nv(unsigned value_bytes, int nv, bool sb)
{
    // header, buffers, then one 40-byte copy plan per slot
    return v27_hdr(sb) + (unsigned)v27_bufs(sb) * (unsigned)(v27_op_slots(sb) + nv) * (unsigned)kV27Slot * value_bytes +
           40u * (unsigned)(v27_op_slots(sb) + nv);
}
// dynamic shared memory of the p(l)-CG kernels and of classic CG's
constexpr unsigned v27_tile_bytes(unsigned value_bytes, int l, bool jacobi)
{
    return v27_tile_bytes_nv(value_bytes, v27_vec_slots(l, jacobi), kV27StageBwdPlcg);
}
constexpr unsigned v27_tile_bytes_cg(unsigned value_bytes)
{
    return v27_tile_bytes_nv(value_bytes, 0, kV27StageBwdCg);
}

// CSR entries (column index + value) each warp of a CSR kernel stages in
// shared memory for its 32 rows of a sweep unit; warps whose rows have more
// entries read them from global memory.  Layout of the dynamic shared
// memory: 8 mbarriers (128 bytes), the warps' column indices, their values.
constexpr int kCsrStageWarpCap = 1024;
constexpr unsigned csr_stage_bytes(unsigned value_bytes)
{
    return 128u + 8u * (unsigned)kCsrStageWarpCap * (4u + value_bytes);
}

// One system of a batched solve (stencil operators only).
struct BatchSys {
    int dim;
    int nx, ny, nz;
    FastDivU32 dnx, dny;
    double center;            // includes the diagonal shift
    double off;
    const double *b;
    double *x;
    DevResult *out;
    double sigma[kMaxL];
};

// Arguments of the batched kernel.  proto carries the solve parameters and
// the ring layout; the per-system fields are filled in on the device.
template <typename T>
struct BatchArgs {
    const BatchSys *sys;
    // "large" list: solved by gangs of G CTAs; "small" list: one CTA each
    int nlarge, nsmall;
    const int *order_large;   // system indices, largest estimated work first
    const int *order_small;
    int *ctr_large, *ctr_small;   // next positions in the lists
    int ngangs, G;
    unsigned *gbar;           // [ngangs][32] gang barrier counters (own cache lines)
    int *gabort;              // [ngangs]
    int *gslot;               // [ngangs] system a gang's leader took
    double *gpart;            // [ngangs][kMaxL + 1][G][kMaxDots]
    double *gnpart;           // [ngangs][G][kNormSlots]
    char *gws;                // per-gang workspaces
    size_t gws_stride;
    char *ws;                 // per-CTA workspaces (one-CTA path)
    size_t ws_stride;
    unsigned long long *t0;   // device global timer at the launch's start (block 0)
    SolveArgs<T> proto;
};

}  // namespace plcg
