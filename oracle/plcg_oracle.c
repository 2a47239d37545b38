/*
 * plcg_oracle.c -- plain, serial, FP64 CPU oracle for classic CG and for the
 * deep pipelined Conjugate Gradient method p(l)-CG of Cools, Cornelis,
 * Ghysels and Vanroose, "Improving strong scaling of the Conjugate Gradient
 * method for solving large linear systems using global reduction
 * pipelining" (EuroMPI'19, arXiv:1905.06850).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA library: the two meet only through the
 * seeded input arrays that the tests hand to both.
 *
 * What it computes
 *   - orc_apply      : y = A x for a Dirichlet 5-point (2D) / 7-point (3D)
 *                      constant-coefficient stencil, a CSR matrix, or a
 *                      symmetric 27-point variable-coefficient stencil given
 *                      by its diagonal and 13 forward weights per cell.
 *   - orc_cg         : classic Hestenes-Stiefel CG (the paper cites it, Sec. 1,
 *                      and costs it in Table 1, but prints no listing, so the
 *                      textbook recurrence is used).
 *   - orc_plcg       : Algorithm 1, step by step, in the paper's notation,
 *                      with M = I or the Jacobi preconditioner M = diag(A),
 *                      under the kernel names of Sec. 3.1: K1 apply A and
 *                      M^{-1}, K2 finalise a column of G (with the
 *                      square-root breakdown check), K3 add a column to T,
 *                      K4 the l+1 basis recurrences (Eq. all_z_rec2 /
 *                      specific_z_rec), K5 the dot products (Sec. 2.2
 *                      "Number of dot products" for the l+1 variant), K6 the
 *                      D-Lanczos solution update and stop test (Sec. 2.1).
 *   - orc_chebyshev_shifts : the shift formula of Sec. 2.2 (Eq. chebyshev).
 *
 * Readings of points the paper leaves open:
 *   R1  the initialization normalises u_0 together with z_0 (with M = I,
 *       u_i = z^(l)_i for all i, so K1 at i = 0 forms (A - sigma_0 I) z_0 as
 *       Eq. z_rec says).
 *   R2  every index range is clamped at 0; g_{j,i} and z_j with j < 0 are zero;
 *       delta_{-1} = 0 (Sec. 2.1).
 *   R3  stop test |zeta_k| < rtol * ||b|| (strict), ||b|| of the original
 *       system, kept across restarts; the returned iterate is x_k with
 *       k = i - l, and a final FP64 true residual ||b - A x|| decides
 *       convergence (a segment whose true residual is not below
 *       rtol * ||b|| is restarted from x).
 *   R4  square-root breakdown (Sec. 2.2 "Square root breakdowns"): with
 *       arg = g_{c,c} - sum_k g_{k,c}^2 and thr = 64 eps g_{c,c}(raw):
 *         |arg| <= thr  -> lucky breakdown: the Krylov space is invariant,
 *                          gamma_{i-l} is still defined, delta_{i-l} = 0;
 *                          form x_{i-l+1} = x_{i-l} + zeta_{i-l} p_{i-l} and
 *                          end the segment;
 *         arg < -thr    -> breakdown: form x_{i-l} and restart from it.
 *       Restarts are counted; more than max_restarts ends the solve with
 *       ORC_ERR_BREAKDOWN.
 *   R5  dots: dots_2l1 = 1 computes the 2l+1 products of K5 literally;
 *       dots_2l1 = 0 computes only the l+1 products of Sec. 2.2 and fills
 *       rows c-2l .. c-l-1 of column c from the symmetry
 *       g_{j,c} = g_{c-l,j+l} (Eq. symmetry_G) when column c is finalised.
 *   R6  the iteration budget maxit counts the x-index k summed over
 *       segments.
 *   R7  preconditioning (precond = 1): M = diag(A), every diagonal entry
 *       positive (else ORC_ERR_INVALID).  p(l)-CG keeps u_i and z^(l)_i as
 *       separate vectors: K1 forms u_{i+1} and then z^(l)_{i+1} =
 *       M^{-1} u_{i+1}, K4 also runs the u recurrence of Sec. 2.2
 *       (Eq. zhatid3), and the dots of K5 take u_{i+1}.  The
 *       initialization normalises u_0 with z_0 (R1).  The norm of R3 becomes the natural
 *       norm ||v||_{M^{-1}} = sqrt(v^T M^{-1} v) (Sec. 2.2 "Residual norm":
 *       |zeta_k| = sqrt((u_k, r_k)) for the preconditioned method): the stop
 *       test is |zeta_k| < rtol * ||b||_{M^{-1}} and the true residual is
 *       measured as ||b - A x||_{M^{-1}}.  CG becomes the textbook
 *       preconditioned CG with rho = (r, M^{-1} r).
 *
 * Everything is double precision and serial; dot products are summed left
 * to right.  No blocking, fusion or reordering beyond the algorithm's own.
 */
#include <math.h>
#include <float.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK              0
#define ORC_ERR_INVALID    -1
#define ORC_ERR_NOMEM      -2
#define ORC_ERR_BREAKDOWN  -4
#define ORC_ERR_MAXIT      -5
#define ORC_ERR_NONFINITE  -6

#define ORC_STENCIL 0
#define ORC_CSR     1
#define ORC_VAR27   2

/* The operator A.  Stencil: unknowns in lexicographic order, x fastest. */
typedef struct {
    int kind;                 /* ORC_STENCIL, ORC_CSR or ORC_VAR27          */
    int dim;                  /* stencil: 2 (5-point) or 3 (7-point)        */
    int64_t nx, ny, nz;       /* stencil grid (nz = 1 in 2D)                */
    double center, off;       /* stencil: diagonal and off-diagonal weight  */
    int64_t n;                /* number of unknowns                          */
    const int64_t *rowptr;    /* CSR: n+1 offsets                            */
    const int32_t *col;       /* CSR: column indices                         */
    const double *val;        /* CSR: values                                 */
    const double *coef;       /* VAR27: [14][n] diagonal, then the weights to
                                 the 13 forward neighbours (see var27_fwd)   */
} orc_op;

/* Parameters of one solve. */
typedef struct {
    int l;                    /* pipeline length (p(l)-CG only)              */
    const double *sigma;      /* l shifts sigma_0 .. sigma_{l-1}             */
    double rtol;              /* relative tolerance tau                      */
    int64_t maxit;            /* budget on the x-index k (R6)               */
    int dots_2l1;             /* R5                                          */
    int max_restarts;         /* R4                                          */
    int precond;              /* R7: 0 M = I, 1 M = diag(A) (Jacobi)          */
} orc_params;

/* Results and optional traces of one solve.  The traces (all caller-owned,
 * NULL to skip) record the FIRST segment only, which is the whole solve
 * when no restart happens; trace_cap bounds every index. */
typedef struct {
    int status;
    int64_t iters;            /* k of the returned x, summed over segments   */
    int64_t spmvs;            /* every application of A                      */
    int64_t dots;             /* every inner product                         */
    int64_t restarts;
    int64_t segments;
    double recursive_relres;  /* |zeta_k| / ||b|| (CG: ||r_k|| / ||b||)      */
    double true_relres;       /* ||b - A x|| / ||b|| (R7: natural norms)     */
    int64_t trace_cap;
    int64_t trace_len;        /* entries written in the x/zeta traces        */
    double *x_hist;           /* [trace_cap][n]      x_k                     */
    double *zeta_hist;        /* [trace_cap]         zeta_k (CG: ||r_k||)    */
    double *gamma_hist;       /* [trace_cap]         gamma_j (CG: alpha_k)   */
    double *delta_hist;       /* [trace_cap]         delta_j (CG: beta_k)    */
    double *g_hist;           /* [trace_cap][2l+1]   column c, rows c-2l..c  */
    double *z_hist;           /* [l+1][trace_cap][n] z^(k)_j (p(l)-CG)       */
    double *graw_hist;        /* [trace_cap][2l+1]   column c as dotted (K5) */
} orc_result;

/* ------------------------------------------------------------------ */
/* Small vector helpers (plain loops).                                 */
/* ------------------------------------------------------------------ */
static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }

/* ------------------------------------------------------------------ */
/* y = A x                                                              */
/* ------------------------------------------------------------------ */
/* The 13 forward offsets (dz, dy, dx) of the symmetric 27-point operator, in
 * lexicographic order (the layout of coef[1..13]); the entry to c - d is the
 * neighbour's entry to c. */
static const int var27_fwd[13][3] = {
    {0, 0, 1}, {0, 1, -1}, {0, 1, 0}, {0, 1, 1},
    {1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1}, {1, 0, 0}, {1, 0, 1},
    {1, 1, -1}, {1, 1, 0}, {1, 1, 1}};

static int in_grid(const orc_op *A, int64_t i, int64_t j, int64_t k)
{
    return i >= 0 && i < A->nx && j >= 0 && j < A->ny && k >= 0 && k < A->nz;
}

void orc_apply(const orc_op *A, const double *x, double *y)
{
    if (A->kind == ORC_VAR27) {
        const int64_t n = A->n;
        for (int64_t k = 0; k < A->nz; ++k)
            for (int64_t j = 0; j < A->ny; ++j)
                for (int64_t i = 0; i < A->nx; ++i) {
                    const int64_t c = (k * A->ny + j) * A->nx + i;
                    double s = A->coef[c] * x[c];
                    for (int d = 0; d < 13; ++d) {
                        const int dz = var27_fwd[d][0], dy = var27_fwd[d][1], dx = var27_fwd[d][2];
                        const int64_t off = (dz * A->ny + dy) * A->nx + dx;
                        if (in_grid(A, i + dx, j + dy, k + dz))
                            s += A->coef[(1 + d) * n + c] * x[c + off];
                        if (in_grid(A, i - dx, j - dy, k - dz))
                            s += A->coef[(1 + d) * n + c - off] * x[c - off];
                    }
                    y[c] = s;
                }
        return;
    }
    if (A->kind == ORC_CSR) {
        for (int64_t r = 0; r < A->n; ++r) {
            double s = 0.0;
            for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e)
                s += A->val[e] * x[A->col[e]];
            y[r] = s;
        }
        return;
    }
    /* Dirichlet stencil: a neighbour outside the grid contributes 0. */
    const int64_t nx = A->nx, ny = A->ny, nz = (A->dim == 3) ? A->nz : 1;
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t id = (k * ny + j) * nx + i;
                double nb = 0.0;
                if (i > 0)      nb += x[id - 1];
                if (i < nx - 1) nb += x[id + 1];
                if (j > 0)      nb += x[id - nx];
                if (j < ny - 1) nb += x[id + nx];
                if (A->dim == 3) {
                    if (k > 0)      nb += x[id - nx * ny];
                    if (k < nz - 1) nb += x[id + nx * ny];
                }
                y[id] = A->center * x[id] + A->off * nb;
            }
}

/* ||v|| (minv == NULL) or the natural norm sqrt(v^T M^{-1} v) (R7). */
static double mnorm(int64_t n, const double *v, const double *minv)
{
    if (!minv) return nrm2(n, v);
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += v[i] * minv[i] * v[i];
    return sqrt(s);
}

/* r = b - A x; returns ||r|| (R7: ||r||_{M^{-1}}). */
static double residual(const orc_op *A, const double *b, const double *x,
                       double *r, const double *minv, orc_result *res)
{
    orc_apply(A, x, r);
    res->spmvs++;
    for (int64_t i = 0; i < A->n; ++i) r[i] = b[i] - r[i];
    res->dots++;
    return mnorm(A->n, r, minv);
}

/* R7: M^{-1} = diag(A)^{-1}.  Returns 0, or -1 if a diagonal entry is not
 * positive (M would not be SPD) or a CSR row has none. */
static int jacobi_minv(const orc_op *A, double *minv)
{
    for (int64_t r = 0; r < A->n; ++r) {
        double d = 0.0;
        if (A->kind == ORC_CSR) {
            for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e)
                if (A->col[e] == r) d += A->val[e];
        } else if (A->kind == ORC_VAR27) {
            d = A->coef[r];
        } else {
            d = A->center;
        }
        if (!(d > 0.0) || !isfinite(d)) return -1;
        minv[r] = 1.0 / d;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Chebyshev shifts, Sec. 2.2 Eq. (chebyshev):                          */
/*   sigma_i = (lmax+lmin)/2 + (lmax-lmin)/2 cos((2i+1) pi / (2l)).     */
/* ------------------------------------------------------------------ */
void orc_chebyshev_shifts(int l, double lmin, double lmax, double *sigma)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < l; ++i)
        sigma[i] = 0.5 * (lmax + lmin)
                 + 0.5 * (lmax - lmin) * cos((2.0 * i + 1.0) * pi / (2.0 * l));
}

/* ------------------------------------------------------------------ */
/* Classic CG (Hestenes-Stiefel), one segment from the residual r.     */
/*   alpha = (r,r)/(p,Ap); x += alpha p; r -= alpha Ap;                */
/*   beta = (r',r')/(r,r); p = r' + beta p.                            */
/* With M (R7), the textbook preconditioned form: z = M^{-1} r,        */
/*   rho = (r,z), alpha = rho/(p,Ap), beta = rho'/rho, p = z' + beta p. */
/* ------------------------------------------------------------------ */
typedef struct { int64_t k; int end; } seg_out;
enum { SEG_CONVERGED = 0, SEG_MAXIT = 1, SEG_BREAKDOWN = 2, SEG_LUCKY = 3, SEG_NONFINITE = 4 };

static int cg_segment(const orc_op *A, double *x, double *r, const double *minv,
                      double tau_abs, int64_t budget, double *work, orc_result *res,
                      int trace, seg_out *so)
{
    const int64_t n = A->n;
    double *p = work, *q = work + n, *z = work + 2 * n;
    for (int64_t i = 0; i < n; ++i) z[i] = minv ? minv[i] * r[i] : r[i];
    memcpy(p, z, (size_t)n * sizeof(double));
    double rr = dot(n, r, z);
    res->dots++;
    int64_t k = 0;
    for (;;) {
        const double rn = sqrt(rr);
        if (trace && res->zeta_hist && k < res->trace_cap) res->zeta_hist[k] = rn;
        if (trace && res->x_hist && k < res->trace_cap)
            memcpy(res->x_hist + k * n, x, (size_t)n * sizeof(double));
        if (trace) res->trace_len = k + 1;
        res->recursive_relres = rn;
        if (!isfinite(rn)) { so->k = k; so->end = SEG_NONFINITE; return 0; }
        if (rn < tau_abs) { so->k = k; so->end = SEG_CONVERGED; return 0; }
        if (k >= budget) { so->k = k; so->end = SEG_MAXIT; return 0; }
        orc_apply(A, p, q);
        res->spmvs++;
        const double pq = dot(n, p, q);
        res->dots++;
        if (!(pq > 0.0)) {   /* A not SPD along p, or NaN */
            so->k = k;
            so->end = isfinite(pq) ? SEG_BREAKDOWN : SEG_NONFINITE;
            return 0;
        }
        const double alpha = rr / pq;
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
        for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
        for (int64_t i = 0; i < n; ++i) z[i] = minv ? minv[i] * r[i] : r[i];
        const double rr_new = dot(n, r, z);
        res->dots++;
        const double beta = rr_new / rr;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        if (trace && res->gamma_hist && k < res->trace_cap) res->gamma_hist[k] = alpha;
        if (trace && res->delta_hist && k < res->trace_cap) res->delta_hist[k] = beta;
        rr = rr_new;
        ++k;
    }
}

/* ------------------------------------------------------------------ */
/* p(l)-CG, one segment of Algorithm 1 started from the residual r    */
/* with rn = sqrt((r, M^{-1} r)) (M = I: ||r||).  x is updated in place. */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int l, R, W;              /* R: ring depth per basis, W = 2l+1 rows     */
    double *zbuf;             /* (l+1) rings of R vectors                   */
    double *ubuf;             /* R7: ring of R vectors u_j (NULL: u = z^(l)) */
    double *gband;            /* column c: rows c-2l .. c                    */
    double *gamma, *delta, *eta, *zeta;
    int64_t ncols;
} plcg_ws;

/* z^(k)_j, stored in slot j mod R of basis k (j >= 0). */
static double *Z(plcg_ws *w, int k, int64_t j)
{
    return w->zbuf + ((int64_t)k * w->R + (j % w->R)) * w->n;
}

/* u_j: its own ring with a preconditioner (R7), else z^(l)_j (M = I). */
static double *U(plcg_ws *w, int64_t j)
{
    return w->ubuf ? w->ubuf + (j % w->R) * w->n : Z(w, w->l, j);
}

/* g_{j,c} for c-2l <= j <= c, j >= 0 (the band of G, Sec. 2.1). */
static double *Gp(plcg_ws *w, int64_t j, int64_t c)
{
    return w->gband + c * w->W + (j - c + 2 * w->l);
}

static double gget(plcg_ws *w, int64_t j, int64_t c)
{
    if (j < 0 || j < c - 2 * w->l || j > c) return 0.0;
    return *Gp(w, j, c);
}

static int plcg_segment(const orc_op *A, double *x, const double *r, double rn,
                        const double *minv, const orc_params *P, double tau_abs,
                        int64_t budget,
                        plcg_ws *w, double *p, orc_result *res, int trace,
                        seg_out *so)
{
    const int64_t n = A->n;
    const int l = P->l;
    const double *sigma = P->sigma;
    const double eps = DBL_EPSILON;

    memset(w->gband, 0, (size_t)(w->ncols * w->W) * sizeof(double));

    /* Algorithm 1, initialization (R1): u_0 := b - A x_0 (= r), r_0 := M^{-1} u_0,
     * z^(k)_0 := r_0 / sqrt((u_0, r_0)), u_0 normalised alike; g_00 := 1. */
    for (int k = 0; k <= l; ++k)
        for (int64_t t = 0; t < n; ++t) Z(w, k, 0)[t] = (minv ? minv[t] * r[t] : r[t]) / rn;
    if (w->ubuf)
        for (int64_t t = 0; t < n; ++t) U(w, 0)[t] = r[t] / rn;
    *Gp(w, 0, 0) = 1.0;
    if (trace && res->g_hist && res->trace_cap > 0) {
        for (int q = 0; q < w->W; ++q) res->g_hist[q] = 0.0;
        res->g_hist[2 * l] = 1.0;
    }
    if (trace && res->x_hist && res->trace_cap > 0)
        memcpy(res->x_hist, x, (size_t)n * sizeof(double));
    if (trace && res->z_hist && res->trace_cap > 0)
        for (int k = 0; k <= l; ++k)
            memcpy(res->z_hist + ((int64_t)k * res->trace_cap) * n, Z(w, k, 0),
                   (size_t)n * sizeof(double));
    if (trace) res->trace_len = 1;

    for (int64_t i = 0;; ++i) {
        if (i + 2 >= w->ncols) { so->k = (i > l) ? i - l : 0; so->end = SEG_MAXIT; return 0; }
        /* ---- K1: u_{i+1} = A z^(l)_i (- sigma_i u_i), then
         * z^(l)_{i+1} := M^{-1} u_{i+1} (M = I: the same vector), and in the
         * fill phase the auxiliary copies z^(k)_{i+1} := z^(l)_{i+1}. */
        double *zl_new = Z(w, l, i + 1);
        double *u_new = U(w, i + 1);
        orc_apply(A, Z(w, l, i), u_new);
        res->spmvs++;
        if (i < l)
            for (int64_t t = 0; t < n; ++t) u_new[t] -= sigma[i] * U(w, i)[t];
        if (minv)
            for (int64_t t = 0; t < n; ++t) zl_new[t] = minv[t] * u_new[t];
        if (i < l - 1)
            for (int k = (int)i + 1; k <= l - 1; ++k)
                memcpy(Z(w, k, i + 1), zl_new, (size_t)n * sizeof(double));

        if (i >= l) {
            const int64_t c = i - l + 1;   /* column of G finalised now       */
            const int64_t m = i - l;       /* column of T added now           */
            const int64_t lo = (c - 2 * l > 0) ? c - 2 * l : 0;   /* = max(0, i-3l+1) */
            /* R5: the l+1 variant fills rows c-2l .. c-l-1 from symmetry. */
            if (!P->dots_2l1)
                for (int64_t j = lo; j <= c - l - 1; ++j)
                    *Gp(w, j, c) = gget(w, c - l, j + l);
            /* ---- K2: correct rows c-l+1 .. c-1, then the diagonal. */
            for (int64_t j = (c - l + 1 > 0 ? c - l + 1 : 0); j <= c - 1; ++j) {
                double s = *Gp(w, j, c);
                for (int64_t k = lo; k <= j - 1; ++k) s -= gget(w, k, j) * gget(w, k, c);
                *Gp(w, j, c) = s / gget(w, j, j);
            }
            const double graw = *Gp(w, c, c);
            double arg = graw;
            for (int64_t k = lo; k <= c - 1; ++k) arg -= gget(w, k, c) * gget(w, k, c);

            /* ---- K3, gamma part: it does not use g_{c,c}. */
            const double gmm = gget(w, m, m);
            double gam;
            if (i < 2 * l)
                gam = (gget(w, m, c) + sigma[m] * gmm
                       - (m >= 1 ? gget(w, m - 1, m) * w->delta[m - 1] : 0.0)) / gmm;
            else
                gam = (gmm * w->gamma[m - l] + gget(w, m, c) * w->delta[m - l]
                       - gget(w, m - 1, m) * w->delta[m - 1]) / gmm;
            w->gamma[m] = gam;

            /* ---- K2: square-root breakdown check (R4). */
            const double thr = 64.0 * eps * fabs(graw);
            if (!isfinite(arg) || !isfinite(gam)) { so->k = m; so->end = SEG_NONFINITE; return 0; }
            if (arg <= thr) {
                if (arg >= -thr) {
                    /* Lucky breakdown: T_{m+1} is the whole (square) tridiagonal
                     * matrix; x_{m+1} is the exact solution in this space. */
                    if (m == 0) {
                        w->eta[0] = gam;
                        w->zeta[0] = rn;
                        for (int64_t t = 0; t < n; ++t) p[t] = Z(w, 0, 0)[t] / w->eta[0];
                    } else {
                        const double lam = w->delta[m - 1] / w->eta[m - 1];
                        w->eta[m] = gam - lam * w->delta[m - 1];
                        w->zeta[m] = -lam * w->zeta[m - 1];
                        for (int64_t t = 0; t < n; ++t) x[t] += w->zeta[m - 1] * p[t];
                        for (int64_t t = 0; t < n; ++t)
                            p[t] = (Z(w, 0, m)[t] - w->delta[m - 1] * p[t]) / w->eta[m];
                    }
                    for (int64_t t = 0; t < n; ++t) x[t] += w->zeta[m] * p[t];
                    res->recursive_relres = 0.0;
                    so->k = m + 1;
                    so->end = SEG_LUCKY;
                    return 0;
                }
                /* Breakdown: keep x_m = x_{m-1} + zeta_{m-1} p_{m-1} and restart. */
                if (m >= 1)
                    for (int64_t t = 0; t < n; ++t) x[t] += w->zeta[m - 1] * p[t];
                so->k = m;
                so->end = SEG_BREAKDOWN;
                return 0;
            }
            *Gp(w, c, c) = sqrt(arg);

            /* ---- K3, delta part. */
            if (i < 2 * l) w->delta[m] = *Gp(w, c, c) / gmm;
            else           w->delta[m] = *Gp(w, c, c) * w->delta[m - l] / gmm;
            const double dm = w->delta[m];
            const double dm1 = (m >= 1) ? w->delta[m - 1] : 0.0;   /* delta_{-1} = 0 */

            /* ---- K4: one new vector per basis.                            */
            /* z^(k)_{m+k+1} = (z^(k+1)_{m+k+1} + (sigma_k - gamma_m) z^(k)_{m+k}
             *                  - delta_{m-1} z^(k)_{m+k-1}) / delta_m,  k < l    */
            for (int k = 0; k < l; ++k) {
                double *zn = Z(w, k, m + k + 1);
                const double *zup = Z(w, k + 1, m + k + 1);
                const double *zc = Z(w, k, m + k);
                const double *zp = (m + k - 1 >= 0) ? Z(w, k, m + k - 1) : NULL;
                for (int64_t t = 0; t < n; ++t)
                    zn[t] = (zup[t] + (sigma[k] - gam) * zc[t]
                             - (zp ? dm1 * zp[t] : 0.0)) / dm;
            }
            /* z^(l)_{i+1} = (M^{-1} A z^(l)_i - gamma_m z^(l)_i
             *                        - delta_{m-1} z^(l)_{i-1}) / delta_m */
            {
                const double *zc = Z(w, l, i);
                const double *zp = (i - 1 >= 0) ? Z(w, l, i - 1) : NULL;
                for (int64_t t = 0; t < n; ++t)
                    zl_new[t] = (zl_new[t] - gam * zc[t] - (zp ? dm1 * zp[t] : 0.0)) / dm;
            }
            /* Eq. zhatid3: u_{i+1} = (A z^(l)_i - gamma_m u_i
             *                                   - delta_{m-1} u_{i-1}) / delta_m */
            if (w->ubuf) {
                const double *uc = U(w, i);
                const double *up = (i - 1 >= 0) ? U(w, i - 1) : NULL;
                for (int64_t t = 0; t < n; ++t)
                    u_new[t] = (u_new[t] - gam * uc[t] - (up ? dm1 * up[t] : 0.0)) / dm;
            }
            if (trace && res->gamma_hist && m < res->trace_cap) res->gamma_hist[m] = gam;
            if (trace && res->delta_hist && m < res->trace_cap) res->delta_hist[m] = dm;
            if (trace && res->g_hist && c < res->trace_cap)
                for (int q = 0; q < w->W; ++q) res->g_hist[c * w->W + q] = w->gband[c * w->W + q];
        }

        /* ---- K5: g_{j,i+1} = (u_{i+1}, z^(0)_j) / (u_{i+1}, z^(l)_j). */
        {
            const int64_t c1 = i + 1;
            const int64_t j0 = P->dots_2l1 ? ((i - 2 * l + 1 > 0) ? i - 2 * l + 1 : 0) : i - l + 1;
            for (int64_t j = (j0 > 0 ? j0 : 0); j <= i - l + 1; ++j) {
                *Gp(w, j, c1) = dot(n, u_new, Z(w, 0, j));
                res->dots++;
            }
            for (int64_t j = (i - l + 2 > 0 ? i - l + 2 : 0); j <= i + 1; ++j) {
                *Gp(w, j, c1) = dot(n, u_new, Z(w, l, j));
                res->dots++;
            }
            if (trace && res->graw_hist && c1 < res->trace_cap)
                for (int q = 0; q < w->W; ++q) res->graw_hist[c1 * w->W + q] = w->gband[c1 * w->W + q];
        }
        if (trace && res->z_hist) {
            /* the vectors this iteration produced */
            const int64_t cap = res->trace_cap;
            if (i + 1 < cap)
                memcpy(res->z_hist + ((int64_t)l * cap + i + 1) * n, zl_new, (size_t)n * sizeof(double));
            if (i < l - 1)
                for (int k = (int)i + 1; k <= l - 1; ++k)
                    if (i + 1 < cap)
                        memcpy(res->z_hist + ((int64_t)k * cap + i + 1) * n, Z(w, k, i + 1),
                               (size_t)n * sizeof(double));
            if (i >= l)
                for (int k = 0; k < l; ++k) {
                    const int64_t j = i - l + k + 1;
                    if (j < cap)
                        memcpy(res->z_hist + ((int64_t)k * cap + j) * n, Z(w, k, j),
                               (size_t)n * sizeof(double));
                }
        }

        /* ---- K6: D-Lanczos update, Sec. 2.1. */
        if (i == l) {
            w->eta[0] = w->gamma[0];
            w->zeta[0] = rn;
            for (int64_t t = 0; t < n; ++t) p[t] = Z(w, 0, 0)[t] / w->eta[0];
            if (trace && res->zeta_hist && res->trace_cap > 0) res->zeta_hist[0] = rn;
        } else if (i >= l + 1) {
            const int64_t m = i - l;
            const double lam = w->delta[m - 1] / w->eta[m - 1];
            w->eta[m] = w->gamma[m] - lam * w->delta[m - 1];
            w->zeta[m] = -lam * w->zeta[m - 1];
            /* x_m = x_{m-1} + zeta_{m-1} p_{m-1}, then p_m from v_m = z^(0)_m. */
            for (int64_t t = 0; t < n; ++t) x[t] += w->zeta[m - 1] * p[t];
            for (int64_t t = 0; t < n; ++t)
                p[t] = (Z(w, 0, m)[t] - w->delta[m - 1] * p[t]) / w->eta[m];
            res->recursive_relres = fabs(w->zeta[m]);
            if (trace && res->x_hist && m < res->trace_cap)
                memcpy(res->x_hist + m * n, x, (size_t)n * sizeof(double));
            if (trace && res->zeta_hist && m < res->trace_cap) res->zeta_hist[m] = w->zeta[m];
            if (trace && m + 1 > res->trace_len) res->trace_len = m + 1;
            if (!isfinite(w->zeta[m])) { so->k = m; so->end = SEG_NONFINITE; return 0; }
            if (fabs(w->zeta[m]) < tau_abs) { so->k = m; so->end = SEG_CONVERGED; return 0; }
            if (m >= budget) { so->k = m; so->end = SEG_MAXIT; return 0; }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Driver shared by both methods: residual -> segment -> true residual */
/* -> restart (R3, R4).                                                 */
/* ------------------------------------------------------------------ */
static int solve(int method, const orc_op *A, const double *b, double *x,
                 const orc_params *P, orc_result *res)
{
    const int64_t n = A->n;
    const int l = P->l;
    if (n <= 0 || !(P->rtol > 0.0) || P->maxit < 0) return ORC_ERR_INVALID;
    if (method == 1 && (l < 1 || l > 64 || P->sigma == NULL)) return ORC_ERR_INVALID;

    res->iters = res->spmvs = res->dots = res->restarts = res->segments = 0;
    res->trace_len = 0;
    res->recursive_relres = res->true_relres = 0.0;

    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *work = (double *)malloc((size_t)(3 * n) * sizeof(double));
    double *minv = P->precond ? (double *)malloc((size_t)n * sizeof(double)) : NULL;
    plcg_ws w;
    memset(&w, 0, sizeof(w));
    if (method == 1) {
        w.n = n; w.l = l; w.R = l + 2; w.W = 2 * l + 1;
        w.ncols = P->maxit + 2 * (int64_t)l + 4;
        w.zbuf = (double *)malloc((size_t)((l + 1) * w.R) * (size_t)n * sizeof(double));
        if (P->precond) w.ubuf = (double *)malloc((size_t)w.R * (size_t)n * sizeof(double));
        w.gband = (double *)malloc((size_t)(w.ncols * w.W) * sizeof(double));
        w.gamma = (double *)calloc((size_t)w.ncols, sizeof(double));
        w.delta = (double *)calloc((size_t)w.ncols, sizeof(double));
        w.eta = (double *)calloc((size_t)w.ncols, sizeof(double));
        w.zeta = (double *)calloc((size_t)w.ncols, sizeof(double));
    }
    int status = ORC_OK;
    if (!r || !work || (P->precond && !minv) ||
        (method == 1 && (!w.zbuf || !w.gband || !w.gamma || !w.delta || !w.eta || !w.zeta ||
                         (P->precond && !w.ubuf)))) {
        status = ORC_ERR_NOMEM;
        goto done;
    }
    if (P->precond && jacobi_minv(A, minv) != 0) { status = ORC_ERR_INVALID; goto done; }

    const double normb = mnorm(n, b, minv);   /* R7: the natural norm */
    if (normb == 0.0) {
        memset(x, 0, (size_t)n * sizeof(double));
        res->status = ORC_OK;
        goto done;
    }
    if (!isfinite(normb)) { status = ORC_ERR_NONFINITE; goto done; }
    const double tau_abs = P->rtol * normb;
    int last_end = SEG_CONVERGED;
    for (;;) {
        const double rn = residual(A, b, x, r, minv, res);
        res->true_relres = rn / normb;
        if (!isfinite(rn)) { status = ORC_ERR_NONFINITE; break; }
        if (rn < tau_abs) { status = ORC_OK; break; }
        if (res->iters >= P->maxit) { status = ORC_ERR_MAXIT; break; }
        if (res->segments > 0) {
            if (res->restarts >= P->max_restarts) {
                status = (last_end == SEG_MAXIT) ? ORC_ERR_MAXIT : ORC_ERR_BREAKDOWN;
                break;
            }
            res->restarts++;
        }
        seg_out so;
        const int trace = (res->segments == 0);
        const int64_t budget = P->maxit - res->iters;
        if (method == 0) cg_segment(A, x, r, minv, tau_abs, budget, work, res, trace, &so);
        else plcg_segment(A, x, r, rn, minv, P, tau_abs, budget, &w, work, res, trace, &so);
        res->segments++;
        res->iters += so.k;
        last_end = so.end;
        if (so.end == SEG_NONFINITE) { status = ORC_ERR_NONFINITE; break; }
        if (so.end == SEG_MAXIT && res->iters >= P->maxit) {
            const double rn2 = residual(A, b, x, r, minv, res);
            res->true_relres = rn2 / normb;
            status = (rn2 < tau_abs) ? ORC_OK : ORC_ERR_MAXIT;
            break;
        }
    }
    res->recursive_relres /= normb;

done:
    res->status = status;
    free(r); free(work); free(minv); free(w.ubuf);
    free(w.zbuf); free(w.gband); free(w.gamma); free(w.delta); free(w.eta); free(w.zeta);
    return status;
}

int orc_cg(const orc_op *A, const double *b, double *x, const orc_params *P, orc_result *res)
{
    return solve(0, A, b, x, P, res);
}

int orc_plcg(const orc_op *A, const double *b, double *x, const orc_params *P, orc_result *res)
{
    return solve(1, A, b, x, P, res);
}

/* Sizes of the structs, so the ctypes wrapper can check its layout. */
int orc_sizeof_op(void) { return (int)sizeof(orc_op); }
int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
int orc_sizeof_result(void) { return (int)sizeof(orc_result); }
