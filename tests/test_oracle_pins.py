"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a dense
Cholesky solve, textbook CG in 60-digit arithmetic, closed forms
(Chebyshev shifts, Laplacian spectra, the Lanczos-CG relation), invariants
(the symmetry of G, the basis relations of Sec. 2.2, A-norm monotonicity)
and the orthogonal invariance behind the paper's diagonal toy problem.
"""
import math

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

from oracle import hiprec as H
from oracle import oracle as O
from paper_1905_06850_gb300 import workloads as W


def dense(op):
    return W.to_scipy(op).toarray()


def shifts(l, op):
    return O.chebyshev_shifts(l, *W.shift_interval(op))


SMALL_OPS = [
    W.stencil2d(12, 12),
    W.stencil2d(17, 9, shift=0.37),
    W.stencil3d(6, 5, 7),
    W.hetero27_csr(5, 5, 5, seed=11),
    W.random_spd_csr(300, seed=12),
]
SMALL_IDS = ["2d12", "2d17x9shift", "3d6x5x7", "h27_5", "rand300"]


# ---------------------------------------------------------------- P1 ------
@pytest.mark.parametrize("op", SMALL_OPS, ids=SMALL_IDS)
def test_p1_final_x_vs_dense_cholesky(op):
    """Both solvers' final x against scipy's dense Cholesky solve:
    ||x - x_chol|| / ||x_chol|| <= kappa * rtol (residual bound)."""
    A = dense(op)
    n = A.shape[0]
    b = np.random.default_rng(5).standard_normal(n)
    x_chol = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), b)
    ev = np.linalg.eigvalsh(A)
    kappa = ev[-1] / ev[0]
    rtol = 1e-10
    bound = 1.01 * kappa * rtol + 1e-13
    r = O.cg(op, b, rtol=rtol)
    assert r.status == O.ORC_OK
    assert np.linalg.norm(r.x - x_chol) / np.linalg.norm(x_chol) <= bound
    for l in range(1, 6):
        for d in (True, False):
            r = O.plcg(op, b, l=l, sigma=shifts(l, op), rtol=rtol, dots_2l1=d)
            assert r.status == O.ORC_OK, (l, d, r.status)
            assert r.true_relres < rtol
            assert np.linalg.norm(r.x - x_chol) / np.linalg.norm(x_chol) <= bound, (l, d)


# ---------------------------------------------------------------- P2 ------
TINY = [W.stencil2d(5, 5), W.stencil2d(3, 4), W.stencil3d(3, 3, 3)]


@pytest.mark.parametrize("op", TINY, ids=["2d5", "2d3x4", "3d3"])
@pytest.mark.parametrize("l", [1, 2, 3, 5])
def test_p2_plcg_is_cg_iterate_for_iterate(op, l):
    """Sec. 2.1: p(l)-CG is a reformulation of CG.  In 60-digit arithmetic
    the Algorithm 1 iterates equal textbook CG's (the identity pins the
    readings R1/R2); the FP64 oracle's early iterates match them to
    rounding."""
    A = dense(op)
    n = A.shape[0]
    b = np.random.default_rng(7).standard_normal(n)
    sig = shifts(l, op)
    xs_cg, _, _, _ = H.cg_decimal(A.tolist(), b, 40)
    hp = H.plcg_decimal(A.tolist(), b, l, sig, 40)
    K = min(len(xs_cg), len(hp["xs"]))
    assert K >= 4
    for k in range(K):
        d = max(abs(float(a - c)) for a, c in zip(hp["xs"][k], xs_cg[k]))
        assert d < 1e-40, (k, d)
    r = O.plcg(op, b, l=l, sigma=sig, rtol=1e-14, trace_cap=60)
    for k in range(1, min(7, K, r.trace["len"])):
        ref = np.array([float(v) for v in xs_cg[k]])
        assert np.linalg.norm(r.trace["x"][k] - ref) <= 1e-10 * np.linalg.norm(ref), k
    rc = O.cg(op, b, rtol=1e-14, trace_cap=60)
    for k in range(1, min(10, K, rc.trace["len"])):
        ref = np.array([float(v) for v in xs_cg[k]])
        assert np.linalg.norm(rc.trace["x"][k] - ref) <= 1e-12 * np.linalg.norm(ref), k


# ---------------------------------------------------------------- P3 ------
@pytest.mark.parametrize("l", [1, 2, 3, 4])
@pytest.mark.parametrize("dots_2l1", [True, False])
def test_p3_tridiagonal_T_matches_lanczos_cg_relation(l, dots_2l1):
    """gamma_j = 1/alpha_j + beta_{j-1}/alpha_{j-1}, delta_j = sqrt(beta_j)/alpha_j
    (the textbook Lanczos-CG relation, Saad Sec. 6.7.3), from exact CG."""
    op = W.stencil2d(6, 7)
    A = dense(op)
    b = np.random.default_rng(8).standard_normal(A.shape[0])
    _, al, be, _ = H.cg_decimal(A.tolist(), b, 30)
    al = [float(a) for a in al]
    be = [float(x) for x in be]
    r = O.plcg(op, b, l=l, sigma=shifts(l, op), rtol=1e-14, dots_2l1=dots_2l1, trace_cap=60)
    K = 8
    for j in range(K):
        g_ref = 1 / al[j] + (be[j - 1] / al[j - 1] if j > 0 else 0.0)
        d_ref = math.sqrt(be[j]) / al[j]
        assert abs(r.trace["gamma"][j] - g_ref) <= 1e-9 * abs(g_ref), j
        assert abs(r.trace["delta"][j] - d_ref) <= 1e-9 * abs(d_ref), j


# ---------------------------------------------------------------- P4 ------
@pytest.mark.parametrize("l", [1, 2, 3])
def test_p4_zeta_is_residual_norm(l):
    """Sec. 2.2: |zeta_j| = ||b - A x_j||."""
    op = W.stencil2d(9, 8, shift=0.1)
    A = dense(op)
    b = np.random.default_rng(9).standard_normal(A.shape[0])
    r = O.plcg(op, b, l=l, sigma=shifts(l, op), rtol=1e-12, trace_cap=200)
    L = r.trace["len"]
    assert L > 10
    for k in range(L):
        true = np.linalg.norm(b - A @ r.trace["x"][k])
        if true < 1e-8 * np.linalg.norm(b):
            break
        assert abs(abs(r.trace["zeta"][k]) - true) <= 1e-8 * true, k


# ---------------------------------------------------------------- P5 ------
@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_p5_symmetry_of_G(l):
    """Eq. (symmetry_G): g_{j,c} = g_{c-l,j+l}.  With all 2l+1 dot products,
    rows c-2l..c-l of column c are direct dots (z_c, v_j) and their partners
    are entries of earlier columns finalised by the K2 forward substitution."""
    op = W.stencil2d(10, 10)
    b = np.random.default_rng(10).standard_normal(100)
    r = O.plcg(op, b, l=l, sigma=shifts(l, op), rtol=1e-12, dots_2l1=True, trace_cap=80)
    g = r.trace["g"]
    W_ = 2 * l + 1
    checked = 0
    for c in range(2 * l, 2 * l + 12):
        for j in range(c - 2 * l, c - l):
            direct = g[c][j - (c - 2 * l)]
            partner = g[j + l][(c - l) - (j + l - 2 * l)]
            assert abs(direct - partner) <= 1e-11 * max(1.0, abs(partner)), (c, j)
            checked += 1
    assert checked > 0 and W_ == g.shape[1]


# ---------------------------------------------------------------- P6 ------
@pytest.mark.parametrize("l", [1, 2, 3])
def test_p6_auxiliary_bases(l):
    """Eq. (def_zjk): z^(k)_j = P_j(A) v_0 for j <= k and P_k(A) v_{j-k} for
    j > k, with P_k(t) = prod_{i<k} (t - sigma_i) (Eq. poly); V = Z^(0) is
    orthonormal and satisfies the Lanczos relation A V_j = V_{j+1} T_{j+1,j}."""
    op = W.stencil2d(8, 9)
    A = dense(op)
    n = A.shape[0]
    b = np.random.default_rng(11).standard_normal(n)
    sig = shifts(l, op)
    r = O.plcg(op, b, l=l, sigma=sig, rtol=1e-12, trace_cap=40)
    Z = r.trace["z"]
    V = Z[0]

    def P(k):
        M = np.eye(n)
        for i in range(k):
            M = M @ (A - sig[i] * np.eye(n))
        return M

    J = 8
    for k in range(l + 1):
        for j in range(J):
            ref = P(j) @ V[0] if j <= k else P(k) @ V[j - k]
            assert np.linalg.norm(Z[k][j] - ref) <= 1e-9 * np.linalg.norm(ref), (k, j)
    Vj = V[:J].T
    assert np.abs(Vj.T @ Vj - np.eye(J)).max() < 1e-10
    gam, dl = r.trace["gamma"], r.trace["delta"]
    for j in range(J - 1):
        lhs = A @ V[j]
        rhs = gam[j] * V[j] + dl[j] * V[j + 1] + (dl[j - 1] * V[j - 1] if j > 0 else 0)
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(lhs), j


# ---------------------------------------------------------------- P7 ------
def test_p7_finite_termination_in_high_precision():
    """CG (and so p(l)-CG) ends in at most as many steps as A has distinct
    eigenvalues: the 4x4 2D Laplacian has 9."""
    op = W.stencil2d(4, 4)
    A = dense(op)
    assert len(np.unique(np.round(np.linalg.eigvalsh(A), 9))) == 9
    b = np.random.default_rng(12).standard_normal(16)
    xs, _, _, rn = H.cg_decimal(A.tolist(), b, 40)
    assert len(xs) - 1 <= 9
    assert float(rn[-1]) <= 1e-40 * float(rn[0])
    for l in (1, 2, 3):
        hp = H.plcg_decimal(A.tolist(), b, l, shifts(l, op), 40)
        assert len(hp["xs"]) - 1 <= 9


@pytest.mark.parametrize("nx,ny", [(3, 3), (3, 5), (4, 4), (5, 5), (6, 4), (6, 6)])
@pytest.mark.parametrize("l", [1, 2, 3, 4, 5])
def test_p7_lucky_breakdown_terminates_in_fp64(nx, ny, l):
    """Near exact termination the square-root argument of K2 (Algorithm 1) goes
    to zero; the oracle's breakdown handling (R4) must still deliver the
    solution to rtol 1e-12."""
    op = W.stencil2d(nx, ny)
    b = np.random.default_rng(nx * 10 + ny).standard_normal(nx * ny)
    r = O.plcg(op, b, l=l, sigma=shifts(l, op), rtol=1e-12)
    assert r.status == O.ORC_OK
    assert r.true_relres < 1e-12
    assert r.iters <= 3 * nx * ny


# ---------------------------------------------------------------- P8 ------
@pytest.mark.parametrize("l", [1, 2, 3, 4, 5, 8])
def test_p8_chebyshev_shifts(l):
    """Eq. (chebyshev): the shifts are the zeros of T_l mapped to [a, b]; the
    monic polynomial prod (t - sigma_i) has sup-norm 2 ((b-a)/4)^l there."""
    a, bb = 0.3, 11.0
    s = O.chebyshev_shifts(l, a, bb)
    t = (2 * s - (a + bb)) / (bb - a)
    coef = np.zeros(l + 1)
    coef[l] = 1
    assert np.abs(np.polynomial.chebyshev.chebval(t, coef)).max() < 1e-12
    grid = np.linspace(a, bb, 20001)
    Pl = np.prod(grid[:, None] - s[None, :], axis=1)
    assert abs(np.abs(Pl).max() - 2 * ((bb - a) / 4) ** l) <= 1e-9 * 2 * ((bb - a) / 4) ** l
    if l == 1:
        assert abs(s[0] - (a + bb) / 2) < 1e-14


# ---------------------------------------------------------------- P9 ------
@pytest.mark.parametrize("op", [W.stencil2d(11, 11), W.stencil2d(7, 13), W.stencil3d(5, 6, 4),
                                W.stencil2d(9, 9, shift=0.5)], ids=["2d11", "2d7x13", "3d", "2dshift"])
def test_p9_spectrum_closed_form_and_operator(op):
    """Extreme eigenvalues of the Dirichlet stencils in closed form, and the
    oracle's matrix-free apply equals scipy's Kronecker-sum matrix."""
    A = dense(op)
    ev = np.linalg.eigvalsh(A)
    lo, hi = W.stencil_spectrum_bounds(op)
    assert abs(ev[0] - lo) < 1e-12 and abs(ev[-1] - hi) < 1e-12
    x = np.random.default_rng(13).standard_normal(A.shape[0])
    assert np.abs(O.apply(op, x) - A @ x).max() < 1e-12


def test_p9_known_extremes_2d_100():
    """4 -+ 4 cos(pi/101) for the 100x100 2D Laplacian (values in
    tests/golden/spectrum_2d_100.txt)."""
    vals = {}
    with open("tests/golden/spectrum_2d_100.txt") as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    lo, hi = W.stencil_spectrum_bounds(W.stencil2d(100, 100))
    assert abs(lo - vals["lambda_min"]) < 1e-11 and abs(hi - vals["lambda_max"]) < 1e-11


def test_p9_csr_apply_matches_scipy():
    for op in (W.hetero27_csr(6, 5, 4, seed=2), W.random_spd_csr(500, seed=3)):
        M = W.to_scipy(op)
        x = np.random.default_rng(14).standard_normal(op["n"])
        assert np.abs(O.apply(op, x) - M @ x).max() < 1e-12 * np.abs(M @ x).max()
        assert abs(M - M.T).max() == 0.0


# ---------------------------------------------------------------- P10 -----
@pytest.mark.parametrize("method", ["cg", "plcg1", "plcg2", "plcg3"])
def test_p10_orthogonal_invariance_diagonal_toy(method):
    """Sec. 4's communication-bound toy: a diagonal matrix with the 2D
    Laplacian's eigenvalues and the rotated right-hand side Q^T b has the
    same residual history (Q = DST-I eigenvectors, via scipy.fft)."""
    N = 24
    op = W.stencil2d(N, N)
    b = np.random.default_rng(15).standard_normal(N * N)
    j = np.arange(1, N + 1)
    lam1 = 2 - 2 * np.cos(j * np.pi / (N + 1))
    lam = (lam1[None, :] + lam1[:, None]).ravel()          # (y, x) order
    bt = scipy.fft.dstn(b.reshape(N, N), type=1, norm="ortho").ravel()
    diag_op = {"kind": "csr", "n": N * N, "rowptr": np.arange(N * N + 1, dtype=np.int64),
               "col": np.arange(N * N, dtype=np.int32), "val": lam}
    assert np.allclose(W.to_scipy(op) @ scipy.fft.idstn(bt.reshape(N, N), type=1, norm="ortho").ravel(),
                       scipy.fft.idstn((lam * bt).reshape(N, N), type=1, norm="ortho").ravel())
    if method == "cg":
        ra = O.cg(op, b, rtol=1e-9, trace_cap=400)
        rb = O.cg(diag_op, bt, rtol=1e-9, trace_cap=400)
    else:
        l = int(method[-1])
        s = O.chebyshev_shifts(l, 0, 8)
        ra = O.plcg(op, b, l=l, sigma=s, rtol=1e-9, trace_cap=400)
        rb = O.plcg(diag_op, bt, l=l, sigma=s, rtol=1e-9, trace_cap=400)
    assert ra.iters == rb.iters
    za, zb = np.abs(ra.trace["zeta"][:ra.trace["len"]]), np.abs(rb.trace["zeta"][:rb.trace["len"]])
    assert np.allclose(za, zb, rtol=1e-7, atol=1e-12 * za[0])


# ---------------------------------------------------------------- P11 -----
@pytest.mark.parametrize("method", ["cg", "plcg1", "plcg3"])
def test_p11_a_norm_error_monotone_and_bounded(method):
    op = W.stencil2d(15, 15, shift=0.05)
    A = dense(op)
    b = np.random.default_rng(16).standard_normal(A.shape[0])
    xstar = np.linalg.solve(A, b)
    if method == "cg":
        r = O.cg(op, b, rtol=1e-10, trace_cap=500)
    else:
        l = int(method[-1])
        r = O.plcg(op, b, l=l, sigma=shifts(l, op), rtol=1e-10, trace_cap=500)
    ev = np.linalg.eigvalsh(A)
    sk = math.sqrt(ev[-1] / ev[0])
    rho = (sk - 1) / (sk + 1)
    errs = []
    for k in range(r.trace["len"]):
        e = xstar - r.trace["x"][k]
        errs.append(math.sqrt(e @ A @ e))
    e0 = errs[0]
    for k in range(1, len(errs)):
        if errs[k] < 1e-9 * e0:
            break
        assert errs[k] < errs[k - 1], k
        assert errs[k] <= 2 * rho ** k * e0 * (1 + 1e-9), k


# ---------------------------------------------------------------- P12 -----
@pytest.mark.parametrize("l", [1, 2, 4])
def test_p12_first_step_is_steepest_descent(l):
    """p_0 = v_0 / eta_0 and zeta_0 = ||r_0|| give x_1 = x_0 + (r'r / r'Ar) r."""
    op = W.stencil3d(5, 4, 6)
    A = dense(op)
    b = np.random.default_rng(17).standard_normal(A.shape[0])
    x0 = np.random.default_rng(18).standard_normal(A.shape[0])
    r = O.plcg(op, b, x0=x0, l=l, sigma=shifts(l, op), rtol=1e-12, trace_cap=10)
    r0 = b - A @ x0
    x1 = x0 + (r0 @ r0) / (r0 @ A @ r0) * r0
    assert np.linalg.norm(r.trace["x"][1] - x1) <= 1e-13 * np.linalg.norm(x1)


# ---------------------------------------------------------------- P13 -----
@pytest.mark.parametrize("l", [1, 2, 3, 5])
def test_p13_one_spmv_per_iteration(l):
    """Table 1: one SPMV per iteration.  A single-segment solve applies A
    k + l + 1 times in the loop (i = 0 .. k + l) plus the initial and final
    residual; the l+1-dot variant computes l+1 dots per iteration (Sec. 2.2)."""
    c = W.config_2d()
    for d in (True, False):
        r = O.plcg(c["op"], c["b"], l=l, sigma=O.chebyshev_shifts(l, 0, 8), rtol=1e-6, dots_2l1=d)
        assert r.status == O.ORC_OK and r.restarts == 0
        assert r.spmvs == r.iters + l + 1 + 2
        i_end = r.iters + l
        if not d:
            # l+1 per iteration once i >= l-1 (fewer while j ranges are clamped), + 2 residual norms
            assert r.dots <= (l + 1) * (i_end + 1) + 2
            assert r.dots >= (l + 1) * (i_end + 1 - l) + 2
    rc = O.cg(c["op"], c["b"], rtol=1e-6)
    assert rc.spmvs == rc.iters + 2


# ---------------------------------------------------- behaviour pins ------
def test_config1_iteration_counts_equal_cg():
    """The 2D 100x100 problem: p(l)-CG for l = 1..5 stops at the same k as CG
    (values in tests/golden/config2d_iters.txt, written by
    tests/golden/make_golden.py from the oracle)."""
    table = {}
    with open("tests/golden/config2d_iters.txt") as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                method, rtol, k = line.split()
                table[(method, float(rtol))] = int(k)
    c = W.config_2d()
    for rtol in (1e-6, 1e-8):
        kcg = O.cg(c["op"], c["b"], rtol=rtol).iters
        assert kcg == table[("cg", rtol)]
        for l in range(1, 6):
            r = O.plcg(c["op"], c["b"], l=l, sigma=O.chebyshev_shifts(l, 0, 8), rtol=rtol)
            assert r.iters == table[(f"plcg{l}", rtol)] == kcg


@pytest.mark.parametrize("l", [2, 3])
def test_breakdown_restart_with_poor_shifts(l):
    """Sec. 2.2: shifts on [0, 2] do not cover the 2D Laplacian's spectrum;
    square-root breakdowns occur and explicit restarts still converge, at a
    higher iteration count than CG.  With no restarts allowed the solve
    reports the breakdown."""
    c = W.config_2d()
    s = O.chebyshev_shifts(l, 0, 2)
    r = O.plcg(c["op"], c["b"], l=l, sigma=s, rtol=1e-6, max_restarts=60)
    assert r.status == O.ORC_OK and r.restarts > 0 and r.true_relres < 1e-6
    assert r.iters > O.cg(c["op"], c["b"], rtol=1e-6).iters
    r0 = O.plcg(c["op"], c["b"], l=l, sigma=s, rtol=1e-6, max_restarts=0)
    assert r0.status == O.ORC_ERR_BREAKDOWN


def test_maxit_and_degenerate_inputs():
    c = W.config_2d()
    r = O.plcg(c["op"], c["b"], l=2, sigma=O.chebyshev_shifts(2, 0, 8), rtol=1e-8, maxit=17)
    assert r.status == O.ORC_ERR_MAXIT and r.iters == 17
    assert r.true_relres > 1e-8
    # b = 0 -> x = 0 immediately
    r = O.plcg(c["op"], np.zeros(10000), l=1, sigma=[4.0], rtol=1e-8)
    assert r.status == O.ORC_OK and r.iters == 0 and not r.x.any()
    # x0 already the solution
    r = O.plcg(c["op"], c["b"], x0=c["xstar"], l=1, sigma=[4.0], rtol=1e-8)
    assert r.status == O.ORC_OK and r.iters == 0
    # non-finite rhs
    bad = c["b"].copy()
    bad[5] = np.nan
    assert O.plcg(c["op"], bad, l=1, sigma=[4.0]).status == O.ORC_ERR_NONFINITE
    # a 1x1 system
    one = W.stencil2d(1, 1)
    r = O.plcg(one, np.array([3.0]), l=2, sigma=O.chebyshev_shifts(2, 0, 8), rtol=1e-12)
    assert r.status == O.ORC_OK and abs(r.x[0] - 0.75) < 1e-15


def test_dot_variants_agree():
    """The l+1-dot variant (symmetry of G) and the 2l+1 dots of K5 (Algorithm 1) give
    the same iteration counts and nearly the same x."""
    c = W.config_2d()
    for l in (1, 2, 3, 4):
        s = O.chebyshev_shifts(l, 0, 8)
        a = O.plcg(c["op"], c["b"], l=l, sigma=s, rtol=1e-8, dots_2l1=True)
        b = O.plcg(c["op"], c["b"], l=l, sigma=s, rtol=1e-8, dots_2l1=False)
        assert a.iters == b.iters
        assert np.linalg.norm(a.x - b.x) <= 1e-10 * np.linalg.norm(a.x)


# ------------------------------------------------- Jacobi preconditioning --
# Sec. 2.2 "Preconditioned p(l)-CG": Algorithm 1 with M = diag(A), u_i and
# z^(l)_i kept apart, dots taken with u, the stop test in the natural norm.

def _jacobi_scaled(op):
    """S A S and S = diag(A)^{-1/2}, formed with scipy.sparse (library)."""
    import scipy.sparse as sp
    A = W.to_scipy(op).tocsr()
    s = 1.0 / np.sqrt(A.diagonal())
    Ah = (sp.diags(s) @ A @ sp.diags(s)).tocsr()
    Ah.sort_indices()
    return {"kind": "csr", "n": A.shape[0], "rowptr": Ah.indptr.astype(np.int64),
            "col": Ah.indices.astype(np.int32), "val": Ah.data.astype(np.float64)}, s


def _jacobi_interval(op):
    A = W.to_scipy(op).tocsr()
    return 0.0, float((np.asarray(abs(A).sum(axis=1)).ravel() / A.diagonal()).max())


@pytest.mark.parametrize("op", [W.hetero27_csr(5, 5, 5, seed=11), W.random_spd_csr(300, seed=12)],
                         ids=["h27_5", "rand300"])
@pytest.mark.parametrize("method", ["cg", "plcg1", "plcg2", "plcg3"])
def test_j1_jacobi_is_cg_on_the_symmetrically_scaled_system(op, method):
    """With M = diag(A) = S^{-2}, preconditioned CG / p(l)-CG on (A, b) is
    the unpreconditioned method on (S A S, S b) with x = S x_hat: the same
    iteration count, iterates x_k = S x_hat_k and |zeta_k| (the natural norm
    of the residual equals ||S r||).  The unpreconditioned path is pinned by
    P1-P13; a dropped M^{-1}, a u/z mix-up in K1, K4 or K5, or a 2-norm stop
    test breaks this identity."""
    n = op["n"]
    b = np.random.default_rng(5).standard_normal(n)
    oph, s = _jacobi_scaled(op)
    if method == "cg":
        r1 = O.cg(op, b, rtol=1e-10, trace_cap=400, precond="jacobi")
        r2 = O.cg(oph, s * b, rtol=1e-10, trace_cap=400)
        tol_x = 1e-10
    else:
        l = int(method[-1])
        sig = O.chebyshev_shifts(l, *_jacobi_interval(op))
        r1 = O.plcg(op, b, l=l, sigma=sig, rtol=1e-10, trace_cap=400, precond="jacobi")
        r2 = O.plcg(oph, s * b, l=l, sigma=sig, rtol=1e-10, trace_cap=400)
        tol_x = 1e-6 if l >= 2 else 1e-10
    assert r1.status == O.ORC_OK and r2.status == O.ORC_OK
    # near termination a rounding-level difference can turn a lucky breakdown
    # into a restart; the first segments are compared iterate by iterate
    assert abs(r1.iters - r2.iters) <= 2
    xs = np.linalg.norm(r1.x)
    k = min(r1.trace["len"], r2.trace["len"])
    assert k >= 10
    for j in range(k):
        assert np.linalg.norm(r1.trace["x"][j] - s * r2.trace["x"][j]) <= tol_x * xs, j
    z1, z2 = np.abs(r1.trace["zeta"][:k]), np.abs(r2.trace["zeta"][:k])
    # rounding grows along the p(l)-CG recurrences (Sec. 2.2); it is bounded
    # relative to the initial residual, not to each small late |zeta_k|
    assert np.all(np.abs(z1 - z2) <= 1e-6 * z1 + 10 * tol_x * z1[0])
    # both converged to 1e-10 in the same natural norm
    assert np.linalg.norm(r1.x - s * r2.x) <= 1e-7 * xs


@pytest.mark.parametrize("l", [1, 2, 3])
def test_j2_zeta_is_the_natural_residual_norm(l):
    """Sec. 2.2 "Residual norm": with a preconditioner, |zeta_j| is
    sqrt(r_j^T M^{-1} r_j) of the true residual r_j = b - A x_j."""
    op = W.hetero27_csr(5, 5, 5, seed=21)
    A = W.to_scipy(op)
    minv = 1.0 / A.diagonal()
    b = np.random.default_rng(22).standard_normal(op["n"])
    sig = O.chebyshev_shifts(l, *_jacobi_interval(op))
    r = O.plcg(op, b, l=l, sigma=sig, rtol=1e-10, trace_cap=400, precond="jacobi")
    assert r.status == O.ORC_OK
    # early iterates: with l >= 2 rounding errors grow along the recurrences
    # (on this operator by ~8x per iteration for l = 3)
    for j in range(0, 5):
        rj = b - A @ r.trace["x"][j]
        nat = math.sqrt(rj @ (minv * rj))
        assert abs(abs(r.trace["zeta"][j]) - nat) <= 1e-8 * nat + 1e-10 * abs(r.trace["zeta"][0]), j
        # and it is not the 2-norm (the operator's diagonal varies)
        assert abs(nat - np.linalg.norm(rj)) > 1e-3 * nat


def test_j3_finite_termination_counts_eigenvalues_of_minv_a():
    """A = T L T (T diagonal, L the 4x4-grid Laplacian) has distinct
    eigenvalues, but diag(A)^{-1} A = T^{-1} (L / 4) T has L's 9: the
    preconditioned methods end in about 9 steps, the plain ones need far
    more (Saad, Sec. 9.2: PCG minimises over the Krylov space of M^{-1}A)."""
    import scipy.sparse as sp
    N = 4
    Lm = dense(W.stencil2d(N, N))
    t = np.exp(np.random.default_rng(3).standard_normal(N * N))
    A = sp.csr_matrix(np.diag(t) @ Lm @ np.diag(t))
    A.sort_indices()
    op = {"kind": "csr", "n": N * N, "rowptr": A.indptr.astype(np.int64),
          "col": A.indices.astype(np.int32), "val": A.data}
    ev = np.linalg.eigvals(np.diag(1.0 / A.diagonal()) @ A.toarray()).real
    assert len(np.unique(np.round(ev, 8))) == 9
    b = np.random.default_rng(4).standard_normal(N * N)
    rc = O.cg(op, b, rtol=1e-12, precond="jacobi")
    assert rc.status == O.ORC_OK and rc.iters <= 9
    assert O.cg(op, b, rtol=1e-12).iters >= 16
    for l in (1, 2):
        r = O.plcg(op, b, l=l, sigma=O.chebyshev_shifts(l, 0.0, 2.0), rtol=1e-12, precond="jacobi")
        assert r.status == O.ORC_OK and r.iters <= 10 and r.true_relres < 1e-12, l
        ru = O.plcg(op, b, l=l, sigma=O.chebyshev_shifts(l, *W.shift_interval(op)), rtol=1e-12)
        assert ru.iters >= 16


@pytest.mark.parametrize("l", [1, 2, 3])
def test_j4_diagonal_matrix_is_solved_exactly(l):
    """M = A for a diagonal A: M^{-1}A = I, the Krylov space has dimension 1
    and the preconditioned methods return b / diag(A) at once."""
    n = 50
    d = np.random.default_rng(9).uniform(0.5, 3.0, n)
    op = {"kind": "csr", "n": n, "rowptr": np.arange(n + 1, dtype=np.int64),
          "col": np.arange(n, dtype=np.int32), "val": d}
    b = np.random.default_rng(10).standard_normal(n)
    r = O.plcg(op, b, l=l, sigma=O.chebyshev_shifts(l, 0.0, 2.0), rtol=1e-12, precond="jacobi")
    assert r.status == O.ORC_OK and r.iters <= 2
    assert np.abs(r.x - b / d).max() <= 1e-14 * np.abs(b / d).max()
    rc = O.cg(op, b, rtol=1e-12, precond="jacobi")
    assert rc.status == O.ORC_OK and rc.iters == 1
    assert np.abs(rc.x - b / d).max() <= 1e-14 * np.abs(b / d).max()


@pytest.mark.parametrize("op", [W.hetero27_csr(5, 5, 5, seed=11), W.random_spd_csr(300, seed=12)],
                         ids=["h27_5", "rand300"])
def test_j5_jacobi_final_x_vs_dense_cholesky(op):
    """Final x against scipy's Cholesky solve.  A natural-norm relative
    residual rho bounds the 2-norm one by sqrt(max d / min d) rho, hence
    ||x - x*|| / ||x*|| <= kappa sqrt(max d / min d) rho."""
    A = dense(op)
    d = np.diag(A)
    b = np.random.default_rng(5).standard_normal(op["n"])
    x_chol = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), b)
    ev = np.linalg.eigvalsh(A)
    rtol = 1e-10
    bound = 1.01 * (ev[-1] / ev[0]) * math.sqrt(d.max() / d.min()) * rtol + 1e-13
    rc = O.cg(op, b, rtol=rtol, precond="jacobi")
    assert rc.status == O.ORC_OK
    assert np.linalg.norm(rc.x - x_chol) / np.linalg.norm(x_chol) <= bound
    for l in range(1, 5):
        r = O.plcg(op, b, l=l, sigma=O.chebyshev_shifts(l, *_jacobi_interval(op)), rtol=rtol,
                   precond="jacobi")
        assert r.status == O.ORC_OK and r.true_relres < rtol, l
        assert np.linalg.norm(r.x - x_chol) / np.linalg.norm(x_chol) <= bound, l


@pytest.mark.parametrize("l", [1, 3])
def test_j6_constant_diagonal_changes_nothing(l):
    """For a constant-coefficient stencil M = c I: every scalar of
    Algorithm 1 and every iterate equal the unpreconditioned ones."""
    op = W.stencil2d(15, 11)
    b = np.random.default_rng(23).standard_normal(op["nx"] * op["ny"])
    sig = shifts(l, op)
    r0 = O.plcg(op, b, l=l, sigma=sig, rtol=1e-9)
    # the spectrum of M^{-1} A is the operator's divided by c = 4
    r1 = O.plcg(op, b, l=l, sigma=sig / 4.0, rtol=1e-9, precond="jacobi")
    assert r0.iters == r1.iters
    assert np.linalg.norm(r0.x - r1.x) <= 1e-11 * np.linalg.norm(r0.x)


def test_j7_jacobi_rejects_a_nonpositive_diagonal():
    op = {"kind": "csr", "n": 2, "rowptr": np.array([0, 1, 2], dtype=np.int64),
          "col": np.array([0, 1], dtype=np.int32), "val": np.array([1.0, -2.0])}
    assert O.cg(op, np.ones(2), precond="jacobi").status == O.ORC_ERR_INVALID
    assert O.plcg(op, np.ones(2), l=1, sigma=[0.5], precond="jacobi").status == O.ORC_ERR_INVALID


@pytest.mark.parametrize("l", [0, 1, 2])
def test_p10_e3_workload_generator(l):
    """The diagonal-toy workload generator builds what P10 pins: the oracle on
    it has the 2D Laplacian's iteration count, and rotating its x back
    (inverse DST-I) gives the Laplacian solve's x."""
    N = 30
    e = W.e3_diagonal(N)
    lap = W.config_2d(nx=N)
    if l == 0:
        a, b = O.cg(e["op"], e["b"], rtol=1e-8), O.cg(lap["op"], lap["b"], rtol=1e-8)
    else:
        s = O.chebyshev_shifts(l, *e["interval"])
        a = O.plcg(e["op"], e["b"], l=l, sigma=s, rtol=1e-8)
        b = O.plcg(lap["op"], lap["b"], l=l, sigma=s, rtol=1e-8)
    assert a.status == b.status == O.ORC_OK and a.iters == b.iters
    xa = scipy.fft.idstn(a.x.reshape(N, N), type=1, norm="ortho").ravel()
    assert np.linalg.norm(xa - b.x) <= 1e-12 * np.linalg.norm(b.x)
    assert np.array_equal(e["b_laplacian"], lap["b"])


# ------------------------------------------- structured 27-point operator --
@pytest.mark.parametrize("dims", [(5, 5, 5), (7, 4, 6), (1, 3, 2), (9, 8, 7)])
def test_var27_apply_matches_the_csr_operator(dims):
    """The oracle's structured 27-point apply (diagonal + 13 forward weights,
    backward weights from the neighbours) equals scipy's product with the CSR
    matrix the generator builds independently from the same coefficients."""
    v = W.hetero27_var27(*dims, seed=11)
    c = W.hetero27_csr(*dims, seed=11)
    x = np.random.default_rng(1).standard_normal(c["n"])
    y = O.apply(v, x)
    ref = W.to_scipy(c) @ x
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_var27_solves_vs_dense_cholesky():
    """CG, p(l)-CG and their Jacobi forms on the structured operator reach
    the Cholesky solution of the same matrix (P1 / J5 bounds)."""
    v = W.hetero27_var27(6, 5, 7, seed=12)
    A = dense(W.hetero27_csr(6, 5, 7, seed=12))
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    x_chol = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), b)
    ev = np.linalg.eigvalsh(A)
    d = np.diag(A)
    rtol = 1e-10
    bound = 1.01 * (ev[-1] / ev[0]) * math.sqrt(d.max() / d.min()) * rtol + 1e-13
    runs = [O.cg(v, b, rtol=rtol), O.cg(v, b, rtol=rtol, precond="jacobi")]
    for l in (1, 2, 3):
        runs.append(O.plcg(v, b, l=l, sigma=O.chebyshev_shifts(l, *W.shift_interval(v)), rtol=rtol))
        runs.append(O.plcg(v, b, l=l, sigma=O.chebyshev_shifts(l, *W.jacobi_shift_interval(v)),
                           rtol=rtol, precond="jacobi"))
    for r in runs:
        assert r.status == O.ORC_OK and r.true_relres < rtol
        assert np.linalg.norm(r.x - x_chol) / np.linalg.norm(x_chol) <= bound


# ------------------------------------------------------------ refinement loop
def test_refined_loop_reduces_to_one_solve_and_matches_cholesky():
    """O.refined (the FP32 path's outer loop in FP64): with a floor below
    rtol it is one plain solve to rtol / 2, the inner target (same
    iterations, same x); with the default
    floor 1e-4 and rtol 1e-8 it takes at least two inner solves, and its x
    satisfies the Cholesky bound like a plain solve."""
    import scipy.linalg as sla
    op = W.stencil2d(12, 11, shift=0.02)
    b = np.random.default_rng(5).standard_normal(W.op_size(op))
    for method, l in (("plcg", 1), ("plcg", 2), ("cg", 1)):
        sig = O.chebyshev_shifts(l, *W.shift_interval(op)) if method == "plcg" else None
        plain = (O.plcg(op, b, l=l, sigma=sig, rtol=0.5e-8, dots_2l1=False) if method == "plcg"
                 else O.cg(op, b, rtol=0.5e-8))
        one = O.refined(op, b, method=method, l=l, sigma=sig, rtol=1e-8, floor=1e-12)
        assert one.segments == 1 and one.iters == plain.iters
        assert np.array_equal(one.x, plain.x)
        two = O.refined(op, b, method=method, l=l, sigma=sig, rtol=1e-8, floor=1e-4)
        assert two.status == O.ORC_OK and two.segments >= 2
        A = W.to_scipy(op).toarray()
        xc = sla.cho_solve(sla.cho_factor(A), b)
        lo, hi = W.stencil_spectrum_bounds(op)
        assert np.linalg.norm(two.x - xc) / np.linalg.norm(xc) <= (hi / lo) * 1e-8
        assert np.linalg.norm(b - A @ two.x) / np.linalg.norm(b) < 1e-8
