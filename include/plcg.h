/*
 * plcg.h -- C ABI of libplcg.so: deep pipelined Conjugate Gradients, p(l)-CG,
 * on one NVIDIA GB300 (sm_103a).
 *
 * Method: Cools, Cornelis, Ghysels, Vanroose, "Improving strong scaling of
 * the Conjugate Gradient method for solving large linear systems using global
 * reduction pipelining", EuroMPI'19 (arXiv:1905.06850), Algorithm 1 with
 * M = I or the Jacobi preconditioner M = diag(A) (Sec. 2.2, "Preconditioned
 * p(l)-CG"), and classic Hestenes-Stiefel CG (cited and costed in Sec. 1 and
 * Table 1; preconditioned alike) for comparison.  The problem is A x = b with A sparse symmetric
 * positive definite (Sec. 2.1).
 *
 * Conventions
 *   - Every function returns a plcg_status; nothing throws across the ABI.
 *     On failure plcg_last_error() returns a thread-local message.
 *   - Vectors are contiguous FP64 arrays of length n.  Pointers marked
 *     "device" must be CUDA device (or managed) memory of the current
 *     device; pointers marked "host" are ordinary host memory.  The caller
 *     owns all vectors and keeps them alive until the call returns (or, for
 *     plcg_submit, until plcg_poll reports completion).
 *   - The library copies matrix data into device memory it owns; that memory
 *     and every workspace are released by plcg_destroy.
 *   - A solve runs on the stream given at matrix creation (NULL = the legacy
 *     default stream) and returns after the stream has finished it.
 *   - Every device-side wait in the library is bounded; when a bound expires
 *     the solve returns PLCG_ERR_TIMEOUT and the CUDA context stays usable.
 */
#ifndef PLCG_H
#define PLCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PLCG_OK = 0,
    PLCG_PENDING = 1,           /* plcg_poll: the request is not finished      */
    PLCG_ERR_INVALID = -1,      /* bad argument (checked on the host)          */
    PLCG_ERR_NOMEM = -2,        /* device or host allocation failed            */
    PLCG_ERR_CUDA = -3,         /* a CUDA call failed (message has the reason) */
    PLCG_ERR_BREAKDOWN = -4,    /* square-root breakdowns exceeded max_restarts
                                   (Algorithm 1, K2; Sec. 2.2)                    */
    PLCG_ERR_MAXIT = -5,        /* iteration budget exhausted; x = last iterate */
    PLCG_ERR_NONFINITE = -6,    /* NaN/Inf met in b, x0 or a recurrence         */
    PLCG_ERR_TIMEOUT = -7,      /* a bounded device wait expired                */
    PLCG_ERR_UNIMPL = -8        /* combination not implemented                  */
} plcg_status;

typedef enum {
    PLCG_FP64 = 0,              /* vectors, dots and scalars in FP64            */
    PLCG_FP32_FP64DOT = 1,      /* FP32 vectors and matrix values; FP64 dot
                                   accumulation, scalar recurrences, true
                                   residual and an FP64 outer refinement loop   */
    PLCG_FP32_MATRIX = 2        /* FP32 matrix values (a CSR or structured
                                   27-point matrix created with
                                   PLCG_FP32_FP64DOT) under FP64 vectors, dots
                                   and scalars: the FP64 algorithm on the
                                   FP32-rounded operator, with the matrix
                                   traffic of the FP32 path (stencils:
                                   PLCG_ERR_UNIMPL)                              */
} plcg_precision;

typedef enum {
    PLCG_METHOD_PLCG = 0,       /* p(l)-CG, Algorithm 1                         */
    PLCG_METHOD_CG = 1          /* classic Hestenes-Stiefel CG                  */
} plcg_method;

typedef enum {
    PLCG_PRECOND_NONE = 0,      /* M = I                                         */
    PLCG_PRECOND_JACOBI = 1     /* M = diag(A); every diagonal entry must be
                                   positive.  Tolerances then apply to natural
                                   norms ||v||_{M^{-1}} = sqrt(v^T M^{-1} v)
                                   (Sec. 2.2, "Residual norm in p(l)-CG"), and
                                   shifts / [lmin, lmax] describe the spectrum
                                   of M^{-1} A (inside [0, 2] for a diagonally
                                   dominant A)                                    */
} plcg_precond;

/* Opaque matrix handle: operator + its device data + cached workspaces. */
typedef struct plcg_matrix plcg_matrix;

/* Structured constant-coefficient operator with homogeneous Dirichlet
 * boundaries (a neighbour outside the grid contributes 0).  Unknowns are in
 * lexicographic order, x fastest: index = (z*ny + y)*nx + x.
 *   dim = 2, points = 5:  (A u)_p = (center + diag_shift) u_p + off * sum of the 4 neighbours
 *   dim = 3, points = 7:  same with the 6 neighbours.
 * The 2D Laplacian of Sec. 4 is center = 4, off = -1; the 3D one center = 6. */
typedef struct {
    int dim;                    /* 2 or 3                                        */
    int points;                 /* 5 (dim 2) or 7 (dim 3)                        */
    int64_t nx, ny, nz;         /* grid; nz = 1 when dim = 2; n = nx*ny*nz < 2^31 */
    double center;
    double off;
    double diag_shift;          /* added to the diagonal (0 for the Laplacian)   */
} plcg_stencil_desc;

/* Solve parameters; plcg_params_default() fills the defaults shown. */
typedef struct {
    int method;                 /* plcg_method (PLCG_METHOD_PLCG)                */
    int l;                      /* pipeline length, 1..8 (1)                     */
    const double *shifts;       /* host array of l shifts sigma_0..sigma_{l-1},
                                   or NULL: Chebyshev shifts on [lmin, lmax],
                                   Sec. 2.2 Eq. (chebyshev) (NULL)               */
    double lmin, lmax;          /* spectrum interval for the shifts (0, 8)      */
    double rtol;                /* stop when ||b - A x|| < rtol ||b|| (1e-8);
                                   Jacobi: in the natural norm                   */
    int64_t maxit;              /* budget on the iterate index k, <= 2^30 (100000) */
    int prec;                   /* plcg_precision (PLCG_FP64)                    */
    int dots_2l1;               /* 1: the 2l+1 dot products of Algorithm 1, K5;
                                   0: l+1 dots via the symmetry of G (Sec. 2.2)  (0) */
    int max_restarts;           /* explicit restarts allowed (8)                 */
    double inner_rtol_floor;    /* FP32 path: floor of the inner relative tolerance
                                   of each refinement step (1e-4) */
    int grid_ctas;              /* 0: choose; else the number of CTAs (tuning)   */
    int precond;                /* plcg_precond (PLCG_PRECOND_NONE)              */
} plcg_params;

typedef struct {
    int status;                 /* plcg_status of this solve                     */
    int64_t iters;              /* k of the returned x (summed over segments)    */
    int64_t spmvs;              /* applications of A, residuals included         */
    int64_t restarts;           /* segments started after the first              */
    int64_t refinements;        /* FP64 outer refinement steps (FP32 path)        */
    double recursive_relres;    /* |zeta_k| / ||b|| at the end of the last segment */
    double true_relres;         /* ||b - A x|| / ||b||, FP64, at return (Jacobi:
                                   both in the natural norm)                      */
    double seconds;             /* device time of the solve (CUDA events)        */
    double latency;             /* serving: seconds from plcg_submit to completion;
                                   plcg_solve_batched: seconds from the batch
                                   launch's start to this system's completion
                                   (device timer); other entry points: = seconds */
} plcg_result;

/* Fill *p with the defaults listed in plcg_params. */
void plcg_params_default(plcg_params *p);

/* Create a matrix-free stencil operator.  stream: a cudaStream_t (NULL =
 * default stream) on which every solve of this matrix runs.
 * Errors: PLCG_ERR_INVALID (bad dims/points, n >= 2^31), PLCG_ERR_CUDA. */
plcg_status plcg_create_stencil(const plcg_stencil_desc *desc, void *stream,
                                plcg_matrix **out);

/* Create a CSR operator (A symmetric positive definite; not checked).
 * rowptr[n+1] (int64, rowptr[0] = 0, non-decreasing), col[nnz] (int32, in
 * [0, n)), val[nnz] (FP64).  on_device = 1: the three arrays are device
 * pointers, else host pointers.  prec fixes the stored value type: PLCG_FP64
 * keeps FP64 values; PLCG_FP32_FP64DOT rounds them to FP32 once, and all
 * solves of this matrix (including the FP64 residuals) use those rounded
 * values.  The arrays are copied; the caller may free them on return.  The
 * diagonal (the sum of a row's entries in column r, in FP64 from the stored
 * values) and its inverse are formed here for PLCG_PRECOND_JACOBI solves,
 * which return PLCG_ERR_INVALID if an entry is not positive.
 * Errors: PLCG_ERR_INVALID (n <= 0, n >= 2^31, bad rowptr or col, checked on
 * the host when on_device = 0), PLCG_ERR_NOMEM, PLCG_ERR_CUDA. */
plcg_status plcg_create_csr(int64_t n, int64_t nnz, const int64_t *rowptr,
                            const int32_t *col, const double *val, int on_device,
                            int prec, void *stream, plcg_matrix **out);

/* Create a structured symmetric 27-point operator with per-cell coefficients
 * on an nx x ny x nz grid (lexicographic order, x fastest; n = nx*ny*nz <
 * 2^31), the operator of a variable-coefficient 27-point discretisation
 * stored without column indices.  coef[14][n] (FP64; host, or device when
 * on_device = 1): coef[0][c] = A[c][c]; coef[1+k][c] = A[c][c + d_k] for the
 * 13 "forward" offsets d_k = (dz, dy, dx), in this order:
 *   (0,0,1) (0,1,-1) (0,1,0) (0,1,1) (1,-1,-1) (1,-1,0) (1,-1,1)
 *   (1,0,-1) (1,0,0) (1,0,1) (1,1,-1) (1,1,0) (1,1,1),
 * offset index d = (dz*ny + dy)*nx + dx.  A[c][c - d_k] = A[c - d_k][c] (A is
 * symmetric, so the backward entries are the neighbours' forward ones).
 * Entries towards cells outside the grid are ignored (Dirichlet).  A must be
 * positive definite (not checked).  prec fixes the stored type as for CSR:
 * PLCG_FP32_FP64DOT rounds the coefficients to FP32 once and every solve
 * (the FP64 residuals included) uses the rounded values.  The array is
 * copied; the Jacobi data (1/A[c][c]) is formed here.
 * Errors: PLCG_ERR_INVALID (sizes, NULL, non-finite values when on host),
 * PLCG_ERR_NOMEM, PLCG_ERR_CUDA. */
plcg_status plcg_create_var27(int64_t nx, int64_t ny, int64_t nz, const double *coef,
                              int on_device, int prec, void *stream, plcg_matrix **out);

/* Estimate the spectrum interval the Chebyshev shifts need (Sec. 2.2 suggests
 * estimating the extreme eigenvalues beforehand): `steps` iterations of
 * classic CG on the GPU (prm->prec and prm->precond: the operator is A, or
 * diag(A)^{-1} A with PLCG_PRECOND_JACOBI) from a fixed pseudo-random
 * right-hand side, whose coefficients give the Lanczos tridiagonal matrix;
 * *lmin and *lmax are its smallest and largest eigenvalues (Ritz values:
 * inside the true interval, the largest one close to lambda_max after a few
 * tens of steps).  steps in [2, 1000].  Runs on the matrix's stream and uses
 * its workspace and host-entry staging buffers.
 * Errors: PLCG_ERR_INVALID, PLCG_ERR_NONFINITE, PLCG_ERR_CUDA, PLCG_ERR_NOMEM. */
plcg_status plcg_estimate_interval(plcg_matrix *A, const plcg_params *prm, int steps, double *lmin,
                                   double *lmax);

/* Release the matrix, its device copies and workspaces.  NULL is a no-op. */
void plcg_destroy(plcg_matrix *A);

/* Solve A x = b.  b: device FP64[n]; x: device FP64[n], in: x0, out: the
 * returned iterate (written even when the status is MAXIT or BREAKDOWN).
 * The whole solve (every iteration, restart and refinement step) runs in one
 * persistent kernel launch; the call waits for it.  res may be NULL.
 * Returns the solve status (also in res->status). */
plcg_status plcg_solve(plcg_matrix *A, const double *b, double *x,
                       const plcg_params *prm, plcg_result *res);

/* As plcg_solve, but b and x are HOST arrays: the call copies b and x0 to
 * the device, solves, and copies x back (pinned staging owned by A). */
plcg_status plcg_solve_host(plcg_matrix *A, const double *b, double *x,
                            const plcg_params *prm, plcg_result *res);

/* Solve count independent systems A[i] x[i] = b[i] (device pointers,
 * 16-byte aligned, else PLCG_ERR_INVALID) in one persistent launch; each system gets its own thread block(s), converged
 * systems retire and their blocks take the next system.  prm applies to
 * every system except that shifts == NULL places Chebyshev shifts on each
 * system's own [lmin_i, lmax_i] given in lmin[], lmax[] (may be NULL: then
 * prm->lmin/lmax for all).  Systems of large estimated work are solved by
 * gangs of thread blocks (see plcg_set_batched_schedule), the rest by one
 * thread block each; each results[i].seconds is the whole batch's time.
 * results[count] may be NULL.  Only stencil matrices, l <= 4 and the l + 1
 * dot products (prm->dots_2l1 = 0) are supported (PLCG_ERR_UNIMPL
 * otherwise).
 * Returns PLCG_OK when every system returned PLCG_OK, else the first
 * non-OK status in index order. */
plcg_status plcg_solve_batched(int count, plcg_matrix *const *A,
                               const double *const *b, double *const *x,
                               const double *lmin, const double *lmax,
                               const plcg_params *prm, plcg_result *results);

/* Stencil solve that allocates nothing, for callers that may not allocate
 * device memory while they solve (a fixed memory budget or pre-reserved
 * pool, a real-time loop that must stay out of the allocator, a plugin
 * handed a stream but no allocator).  The paper has no counterpart: this is
 * a deployment variant of plcg_solve for stencil operators.
 *   desc, prm, res: as for plcg_create_stencil / plcg_solve (res may be
 *   NULL; res->seconds is 0).  b, x: device FP64[n], 16-byte aligned, owned
 *   by the caller (x in: x0, out: the solution).  stream: cudaStream_t.
 * The solve runs as plcg_solve runs it for the same operator and parameters
 * (the same checks, shifts, kernel, launch shape and kernel arguments, the
 * debug hooks included), so its iterates and status are those of plcg_solve.
 * The solver's scratch is one fixed __device__ array of 32 MiB inside the
 * library, held by every GPU that loads it until the process exits; a solve
 * whose scratch would not fit (roughly n > 400k for FP64 l = 1) returns
 * PLCG_ERR_INVALID and names both sizes.  The call performs no cudaMalloc,
 * cudaFree or other allocation.  Its first call on a device looks up that
 * array's device address (cudaGetSymbolAddress), so make the first call on
 * each device before any stream capture.  The call is synchronous: it
 * returns after the solve has finished on the stream and its result record
 * has been read back.  All calls share the one array, which keeps the
 * previous call's contents (the parts that must start at zero are cleared
 * by each call); calls whose kernels overlap on the GPU race with each
 * other.  Returns the solve status like plcg_solve. */
plcg_status plcg_solve_stencil_noalloc(const plcg_stencil_desc *desc, const double *b,
                                       double *x, const plcg_params *prm,
                                       plcg_result *res, void *stream);

/* ---- serving (continuous batching) ------------------------------------ */
typedef struct plcg_server plcg_server;

/* Create a solve server on the current device.  A scheduler thread admits
 * submitted requests in FIFO order as soon as (a) their device workspace fits
 * the remaining mem_budget_bytes (0: 80% of the free memory at creation),
 * (b) one of max_inflight stream slots is free (0: 32), and (c) their thread
 * blocks fit on the GPU next to the solves already running; a request that
 * does not fit yet lets later requests that fit start before it for up to
 * 100 ms of its waiting time (backfilling), then admission waits for it.
 * Each admitted request runs as its own persistent launch (Algorithm 1 or
 * CG, as in plcg_solve) on its own stream, so requests of different sizes
 * overlap on the device and new requests start while others are running.
 * A request's grid size depends only on the request (at most half of the
 * GPU's resident thread blocks), so its result is bit-identical whether it
 * runs alone or in a mix.
 * Errors: PLCG_ERR_INVALID, PLCG_ERR_CUDA. */
plcg_status plcg_server_create(size_t mem_budget_bytes, int max_inflight, plcg_server **out);

/* Queue a solve of A x = b (device pointers, 16-byte aligned, kept alive by
 * the caller -- together with A -- until the request completes).  prm is
 * copied.  Returns PLCG_OK and a ticket, PLCG_ERR_INVALID for bad arguments,
 * or PLCG_ERR_NOMEM when the request's workspace exceeds the whole budget. */
plcg_status plcg_submit(plcg_server *S, plcg_matrix *A, const double *b, double *x,
                        const plcg_params *prm, uint64_t *ticket);

/* PLCG_PENDING while the request is queued or running; once it has finished,
 * its final status (the result, with res->latency = submit-to-completion
 * seconds, is written to *res) and the ticket is released.  Unknown or
 * already-collected tickets: PLCG_ERR_INVALID. */
plcg_status plcg_poll(plcg_server *S, uint64_t ticket, plcg_result *res);

/* As plcg_poll, but blocks until the request has finished. */
plcg_status plcg_wait(plcg_server *S, uint64_t ticket, plcg_result *res);

/* Run every queued and running request to completion, then release the
 * server.  Results not collected are discarded.  NULL is a no-op. */
void plcg_server_destroy(plcg_server *S);

/* Schedule of plcg_solve_batched (set by an autotuner; process-wide).  The
 * systems whose estimated work n * sqrt(kappa) exceeds large_work_factor
 * times one CTA's fair share of the batch are solved by gangs of gang_size
 * thread blocks each (at most max_gang_fraction of the launch's blocks form
 * gangs); the others get one thread block each.  gang_size = 0 restores the
 * defaults (8, 1.0, 0.5); gang_size = 1 disables gangs.  Errors:
 * PLCG_ERR_INVALID. */
plcg_status plcg_set_batched_schedule(int gang_size, double large_work_factor,
                                      double max_gang_fraction);

/* Measurement helper (the paper has no counterpart): the FP64 FMA
 * throughput of the current device, in FLOP/s (2 per FMA), from a kernel of
 * independent FMA chains on every resident thread (best of 3 timed launches
 * after a warm-up, CUDA events).  It is the FP64 peak the FP64 sweeps are
 * compared with.  Allocates and frees a small output buffer.
 * Errors: PLCG_ERR_INVALID (NULL), PLCG_ERR_CUDA. */
plcg_status plcg_measure_fp64_fma_rate(double *flops_per_s);

/* Launch shape of plcg_solve_batched's FP32 solves (set by an autotuner;
 * process-wide): the kernel variant whose registers are sized for
 * ctas_per_sm (3 or 4) thread blocks per SM, with rows_per_thread (1, 2 or
 * 4) row groups per thread in the one-block-per-system path
 * (vector_width = 1); or (4, 1, 2): in that path each thread takes pairs of
 * adjacent rows as 2-wide vectors in the systems whose nx is even, one row
 * group in the others.  0, 0, 0 restores each method's default (4 blocks per
 * SM; 2-wide rows for p(1)- and p(2)-CG, 1 row group for l >= 3, 4 for
 * classic CG).  FP64 batched solves always use their defaults (4 row groups
 * for p(1)-CG and classic CG, 1 for l >= 2).  Errors: PLCG_ERR_INVALID. */
plcg_status plcg_set_batched_launch(int ctas_per_sm, int rows_per_thread, int vector_width);

/* Small systems (stencil or CSR operators, M = I or a Jacobi-preconditioned
 * stencil, grid_ctas = 0) are solved by one thread-block cluster of up to 16
 * blocks instead of a grid of blocks: the cluster barrier replaces the grid
 * barrier and each block's partial dot products are read by the others from
 * its shared memory.  This applies to p(l)-CG with 2 <= l <= 4 and classic CG
 * up to max_rows unknowns, and to p(1)-CG up to max_rows / 2.  Process-wide;
 * 0 disables; the default is 12288.  A device that cannot place a cluster
 * falls back to the grid.  Errors: PLCG_ERR_INVALID (max_rows < 0). */
plcg_status plcg_set_cluster_rows(int64_t max_rows);

/* Thread-local message describing the last failure in this thread. */
const char *plcg_last_error(void);

/* Library version string. */
const char *plcg_version(void);

/* ---- test hooks (no effect unless called) ----------------------------- */
/* Bound on the polls of every device-side wait (grid barrier, server
 * mailbox); 0 restores the default (about 2 s at 64 ns per poll). */
void plcg_debug_set_poll_limit(uint64_t polls);
/* 1: every grid barrier of the next solves waits for one arrival more than
 * there are thread blocks, so the first wait runs out and the solve returns
 * PLCG_ERR_TIMEOUT (exercises the bounded-wait path); 0: off. */
void plcg_debug_force_barrier_timeout(int on);

/* Launch shape and flags of the calling thread's last single-system solve
 * launch (plcg_solve, plcg_solve_host, plcg_estimate_interval,
 * plcg_solve_stencil_noalloc), so that tests can check that two entry
 * points launch the same way; all zero before the first launch. */
typedef struct {
    uint64_t kernel;            /* identifies the kernel instantiation          */
    int grid_ctas;              /* thread blocks of the cooperative launch      */
    unsigned dyn_smem;          /* dynamic shared memory bytes per block        */
    int lookahead;              /* 1: each iteration's scalars are computed
                                   during the previous sweep (l >= 2)           */
    int staged;                 /* 1: CSR entries staged in shared memory       */
    uint64_t poll_limit;        /* bound of every device-side wait (polls)      */
    int force_timeout;          /* the plcg_debug_force_barrier_timeout setting */
    int cluster;                /* > 0: the grid is one thread-block cluster of
                                   this many blocks (small systems)             */
} plcg_launch_info;
void plcg_debug_last_launch(plcg_launch_info *out);

/* Test hook (no GPU work): the server's admission pass over a queue of n
 * requests in FIFO order -- request i needs bytes[i] of workspace, occupies
 * share[i] SMs and has waited waited_s[i] seconds -- given mem_free bytes of
 * budget left, sm_used SMs occupied by running solves, num_sms SMs and
 * free_slots stream slots.  Writes the admitted indices, in order, to
 * admitted[] (room for n) and returns their count. */
int plcg_debug_server_admission(int n, const uint64_t *bytes, const double *share,
                                const double *waited_s, uint64_t mem_free, double sm_used,
                                int num_sms, int free_slots, int *admitted);

#ifdef __cplusplus
}
#endif

#endif /* PLCG_H */
