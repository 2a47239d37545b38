"""GPU parity of the Jacobi-preconditioned solvers (M = diag(A); Sec. 2.2,
"Preconditioned p(l)-CG") against the FP64 CPU oracle, through the C ABI.

Tolerances as for the unpreconditioned path: FP64 solution relative error
<= max(1e-10, 4x the oracle's own rounding-order sensitivity); FP32 path
<= 1e-5 against the FP64 oracle on the FP32-rounded operator; natural-norm
true relative residual < rtol (checked again on the host); iteration counts
within 10% (FP32: a wider window, its inner solves restart)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_06850_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    from paper_1905_06850_gb300 import build as B
    from paper_1905_06850_gb300 import plcg
    B.build()
    plcg.load()
    torch.cuda.set_device(0)
    return plcg


def gpu_solve(P, op, b, prec="fp64", x0=None, **kw):
    import torch
    A = P.Matrix(op, prec=prec)
    bt = torch.tensor(b, dtype=torch.float64, device="cuda")
    xt = torch.zeros_like(bt) if x0 is None else torch.tensor(x0, dtype=torch.float64, device="cuda")
    res = A.solve(bt, xt, check=False, prec=prec, **kw)
    A.close()
    return xt.cpu().numpy(), res


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def natural_relres(op, b, x):
    """||b - A x||_{M^{-1}} / ||b||_{M^{-1}}, M = diag(A), via scipy."""
    A = W.to_scipy(op)
    minv = 1.0 / A.diagonal()
    r = b - A @ x
    return np.sqrt(r @ (minv * r)) / np.sqrt(b @ (minv * b))


def permuted(op, perm):
    import scipy.sparse as sp
    A = W.to_scipy(op)
    Ap = sp.csr_matrix(A[perm][:, perm])
    Ap.sort_indices()
    return {"kind": "csr", "n": op["n"], "rowptr": Ap.indptr.astype(np.int64),
            "col": Ap.indices.astype(np.int32), "val": Ap.data}


def self_sensitivity(op, b, method, l, sig, rtol):
    """The oracle against itself under a permutation of the unknowns (only the
    rounding order changes): relative x difference and iteration spread."""
    perm = np.random.default_rng(0).permutation(op["n"])
    opp = permuted(op, perm)
    if method == "cg":
        a = O.cg(op, b, rtol=rtol, precond="jacobi")
        c = O.cg(opp, b[perm], rtol=rtol, precond="jacobi")
    else:
        a = O.plcg(op, b, l=l, sigma=sig, rtol=rtol, dots_2l1=False, precond="jacobi")
        c = O.plcg(opp, b[perm], l=l, sigma=sig, rtol=rtol, dots_2l1=False, precond="jacobi")
    xc = np.empty_like(c.x)
    xc[perm] = c.x
    return rel(xc, a.x), abs(a.iters - c.iters) / max(a.iters, 1)


def check_jacobi(P, op, b, method, l, rtol, prec="fp64", iter_slack=None, max_restarts=8):
    oop = W.fp32_rounded(op) if prec == "fp32" else op
    interval = W.jacobi_shift_interval(oop)
    sig = O.chebyshev_shifts(l, *interval) if method == "plcg" else None
    if method == "cg":
        ref = O.cg(oop, b, rtol=rtol, precond="jacobi")
    else:
        ref = O.plcg(oop, b, l=l, sigma=sig, rtol=rtol, dots_2l1=False, precond="jacobi",
                     max_restarts=max_restarts)
    assert ref.status == O.ORC_OK
    if prec == "fp64":
        sx, sk = self_sensitivity(oop, b, method, l, sig, rtol)
        tol, slack = max(1e-10, 4 * sx), max(0.1, 2 * sk)
    else:
        tol, slack = 1e-5, 0.5
    if iter_slack is not None:
        slack = iter_slack
    x, res = gpu_solve(P, op, b, prec=prec, method=method, l=l, interval=interval, rtol=rtol,
                       precond="jacobi", max_restarts=max_restarts)
    assert res.status == P.PLCG_OK, (res, P.last_error())
    assert res.true_relres < rtol
    assert natural_relres(oop, b, x) < rtol * 1.000001
    assert rel(x, ref.x) <= tol, (rel(x, ref.x), tol, res.iters, ref.iters)
    assert abs(res.iters - ref.iters) <= max(1, int(slack * ref.iters)), (res.iters, ref.iters)
    return res, ref


H27 = W.hetero27_csr(14, 12, 10, seed=3)
H27_B = W.rhs(H27, np.random.default_rng(4).standard_normal(H27["n"]))
RAND = W.random_spd_csr(7000, seed=9)
RAND_B = np.random.default_rng(10).standard_normal(RAND["n"])


@pytest.mark.parametrize("l", [1, 2, 3])
def test_jacobi_hetero27_fp64(P, l):
    check_jacobi(P, H27, H27_B, "plcg", l, 1e-8)


@pytest.mark.parametrize("l", [1, 2, 3])
def test_jacobi_hetero27_fp32(P, l):
    res, ref = check_jacobi(P, H27, H27_B, "plcg", l, 1e-8, prec="fp32", max_restarts=64)
    assert res.refinements + res.restarts >= 1   # FP64 correction steps ran


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_jacobi_cg_hetero27(P, prec):
    check_jacobi(P, H27, H27_B, "cg", 1, 1e-8, prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_jacobi_random_spd(P, prec):
    for l in (1, 2):
        check_jacobi(P, RAND, RAND_B, "plcg", l, 1e-8, prec=prec, max_restarts=64)
    check_jacobi(P, RAND, RAND_B, "cg", 1, 1e-8, prec=prec)


def test_jacobi_preconditioning_pays_on_hetero27(P):
    """Jacobi removes the coefficient contrast: fewer iterations than M = I."""
    x0, r0 = gpu_solve(P, H27, H27_B, l=1, interval=W.shift_interval(H27), rtol=1e-8)
    x1, r1 = gpu_solve(P, H27, H27_B, l=1, interval=W.jacobi_shift_interval(H27), rtol=1e-8,
                       precond="jacobi")
    assert r0.ok and r1.ok and r1.iters < r0.iters


def test_jacobi_early_iterates_elementwise(P):
    """Iterates 1..6 of p(2)-CG with M = diag(A) against the oracle's, before
    rounding differences grow."""
    sig = O.chebyshev_shifts(2, *W.jacobi_shift_interval(H27))
    for k in (1, 3, 6):
        ref = O.plcg(H27, H27_B, l=2, sigma=sig, rtol=1e-8, maxit=k, dots_2l1=False,
                     precond="jacobi")
        x, res = gpu_solve(P, H27, H27_B, l=2, interval=W.jacobi_shift_interval(H27), rtol=1e-8,
                           maxit=k, precond="jacobi")
        assert res.status == P.PLCG_ERR_MAXIT and res.iters == k
        assert rel(x, ref.x) <= 1e-10, k


@pytest.mark.parametrize("l", [1, 2, 3])
def test_jacobi_on_stencils_matches_oracle(P, l):
    """Constant-coefficient stencils: M = c I; the library runs the
    unpreconditioned recurrences with the shifts scaled by c."""
    for c in (W.config_2d(), W.config_3d(nx=32)):
        op, b = c["op"], c["b"]
        interval = W.jacobi_shift_interval(op)
        sig = O.chebyshev_shifts(l, *interval)
        ref = O.plcg(op, b, l=l, sigma=sig, rtol=1e-8, dots_2l1=False, precond="jacobi")
        x, res = gpu_solve(P, op, b, l=l, interval=interval, rtol=1e-8, precond="jacobi")
        assert res.ok and res.true_relres < 1e-8
        assert rel(x, ref.x) <= 1e-10 and abs(res.iters - ref.iters) <= 1
    refc = O.cg(op, b, rtol=1e-8, precond="jacobi")
    xc, rc = gpu_solve(P, op, b, method="cg", rtol=1e-8, precond="jacobi")
    assert rc.ok and rel(xc, refc.x) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_jacobi_diagonal_matrix_exact(P, prec):
    """M = A: M^{-1} A = I, the answer b / diag(A) comes at once."""
    n = 5000
    d = np.random.default_rng(9).uniform(0.5, 3.0, n)
    op = {"kind": "csr", "n": n, "rowptr": np.arange(n + 1, dtype=np.int64),
          "col": np.arange(n, dtype=np.int32), "val": d}
    b = np.random.default_rng(10).standard_normal(n)
    dd = W.fp32_rounded(op)["val"] if prec == "fp32" else d
    for l in (1, 2, 3):
        x, res = gpu_solve(P, op, b, prec=prec, l=l, interval=(0.0, 2.0), rtol=1e-12,
                           precond="jacobi")
        assert res.ok and res.iters <= 2, (l, res)
        assert rel(x, b / dd) <= 1e-13
    x, res = gpu_solve(P, op, b, prec=prec, method="cg", rtol=1e-12, precond="jacobi")
    assert res.ok and res.iters <= 2 and rel(x, b / dd) <= 1e-13


def test_jacobi_rejects_nonpositive_diagonal(P):
    import torch
    n = 3
    op = {"kind": "csr", "n": n, "rowptr": np.array([0, 1, 2, 3], dtype=np.int64),
          "col": np.array([0, 1, 2], dtype=np.int32), "val": np.array([1.0, -2.0, 3.0])}
    A = P.Matrix(op)
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(P.PlcgError) as e:
        A.solve(b, x, precond="jacobi")
    assert e.value.status == P.PLCG_ERR_INVALID and "diagonal" in P.last_error()
    A.close()
    A = P.Matrix(W.stencil2d(4, 4, center=-4.0, off=1.0))
    b = torch.ones(16, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(P.PlcgError) as e:
        A.solve(b, x, precond="jacobi")
    assert e.value.status == P.PLCG_ERR_INVALID
    A.close()


def test_jacobi_batched_stencils(P):
    """Batched shifted 2D systems with Jacobi: each system's shifts are given
    on M^{-1} A's spectrum; the result equals the unpreconditioned batched solve
    on the unscaled interval (M = c_i I per system)."""
    import torch
    systems = W.batched_systems(count=24, s_lo=8, s_hi=40, seed=7)
    mats = [P.Matrix(s["op"]) for s in systems]
    bs = [torch.tensor(s["b"], device="cuda") for s in systems]
    x0 = [torch.zeros_like(t) for t in bs]
    x1 = [torch.zeros_like(t) for t in bs]
    lo = [s["interval"][0] for s in systems]
    hi = [s["interval"][1] for s in systems]
    cen = [s["op"]["center"] for s in systems]
    st0, r0 = P.solve_batched(mats, bs, x0, lo, hi, l=2, rtol=1e-8, prec="fp32")
    st1, r1 = P.solve_batched(mats, bs, x1, [a / c for a, c in zip(lo, cen)],
                              [a / c for a, c in zip(hi, cen)], l=2, rtol=1e-8, prec="fp32",
                              precond="jacobi")
    assert st0 == P.PLCG_OK and st1 == P.PLCG_OK
    for s, a, c, ra, rc in zip(systems, x0, x1, r0, r1):
        assert abs(ra.iters - rc.iters) <= 1
        assert rel(c.cpu().numpy(), a.cpu().numpy()) <= 1e-6
        assert natural_relres(W.fp32_rounded(s["op"]), s["b"], c.cpu().numpy()) < 1e-8 * 1.000001
    for m in mats:
        m.close()


def test_jacobi_serving_request(P):
    """A Jacobi CSR request through the server equals the direct solve."""
    import torch
    op = W.random_spd_csr(3000, seed=31)
    b = np.random.default_rng(32).standard_normal(op["n"])
    interval = W.jacobi_shift_interval(op)
    xd, rd = gpu_solve(P, op, b, l=2, interval=interval, rtol=1e-8, precond="jacobi")
    A = P.Matrix(op)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    S = P.Server(mem_budget_bytes=1 << 30)
    t = S.submit(A, bt, xt, l=2, interval=interval, rtol=1e-8, precond="jacobi")
    res = S.wait(t)
    S.close()
    A.close()
    assert res.ok and rd.ok and res.iters == rd.iters
    assert np.array_equal(xt.cpu().numpy(), xd)


def test_jacobi_hetero27_full_size(P):
    """The 128^3 27-point heterogeneous CSR workload with Jacobi in the
    benchmark's launch configuration: iterate 6 element-wise against the
    oracle on the FP64 path (same operator values), iterate 1 on the FP32
    path (later FP32 iterates carry FP32 rounding, ~1e-5 by k = 6), then full
    FP32 solves for l = 1, 2, 3 and CG to the natural-norm rtol, checked on
    the host."""
    c = W.config_hetero27()
    op, b = c["op"], c["b"]
    op32 = W.fp32_rounded(op)
    interval = W.jacobi_shift_interval(op32)
    sig = O.chebyshev_shifts(2, *interval)
    for prec, k, tol in (("fp64", 6, 1e-10), ("fp32", 1, 1e-6)):
        ref = O.plcg(op32, b, l=2, sigma=sig, rtol=1e-8, maxit=k, dots_2l1=False,
                     precond="jacobi")
        x, res = gpu_solve(P, op32, b, prec=prec, l=2, interval=interval, rtol=1e-8, maxit=k,
                           precond="jacobi")
        assert res.status == P.PLCG_ERR_MAXIT and res.iters == k
        assert rel(x, ref.x) <= tol, (prec, rel(x, ref.x))
        idx = np.random.default_rng(0).integers(0, op["n"], 1000)
        assert np.max(np.abs(x[idx] - ref.x[idx])) <= 10 * tol * np.max(np.abs(ref.x))
    for l in (1, 2, 3):
        x, res = gpu_solve(P, op, b, prec="fp32", l=l, interval=interval, rtol=1e-8,
                           precond="jacobi", max_restarts=64)
        assert res.ok, (l, res, P.last_error())
        assert natural_relres(op32, b, x) < 1e-8 * 1.000001
    x, res = gpu_solve(P, op, b, prec="fp32", method="cg", rtol=1e-8, precond="jacobi")
    assert res.ok and natural_relres(op32, b, x) < 1e-8 * 1.000001


# ------------------------------------------------------------ shift interval
@pytest.mark.parametrize("precond", [None, "jacobi"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_estimate_interval_brackets_the_spectrum(P, precond, prec):
    """plcg_estimate_interval returns Ritz values of the (preconditioned)
    operator: inside [lambda_min, lambda_max] (scipy's eigenvalues of the same
    matrix), the largest within 3% of lambda_max after 40 CG steps."""
    import scipy.sparse.linalg as sla
    op = W.hetero27_csr(16, 14, 12, seed=3)
    opr = W.fp32_rounded(op) if prec == "fp32" else op
    A = W.to_scipy(opr).tocsr()
    if precond:
        import scipy.sparse as sp
        s = 1.0 / np.sqrt(A.diagonal())
        A = (sp.diags(s) @ A @ sp.diags(s)).tocsr()   # similar to diag(A)^{-1} A
    lmax = sla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = sla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    M = P.Matrix(op, prec=prec)
    lo, hi = M.estimate_interval(steps=40, prec=prec, precond=precond)
    M.close()
    slack = 1e-6 if prec == "fp64" else 1e-4
    assert lmin * (1 - slack) <= lo <= hi <= lmax * (1 + slack), (lo, hi, lmin, lmax)
    assert hi >= 0.97 * lmax


def test_estimated_interval_removes_fp32_breakdowns(P):
    """Chebyshev shifts on the estimated interval [0, 1.02 lambda_max] instead
    of the Gershgorin bound [0, 2]: the FP32 p(2)-CG with Jacobi runs without
    square-root breakdowns and matches the oracle on that interval."""
    M = P.Matrix(H27, prec="fp32")
    lo, hi = M.estimate_interval(steps=40, prec="fp32", precond="jacobi")
    M.close()
    interval = (0.0, 1.02 * hi)
    oop = W.fp32_rounded(H27)
    sig = O.chebyshev_shifts(2, *interval)
    ref = O.plcg(oop, H27_B, l=2, sigma=sig, rtol=1e-8, dots_2l1=False, precond="jacobi")
    x, res = gpu_solve(P, H27, H27_B, prec="fp32", l=2, interval=interval, rtol=1e-8, precond="jacobi")
    assert res.ok and res.restarts == 0
    assert rel(x, ref.x) <= 1e-5
    assert abs(res.iters - ref.iters) <= max(1, int(0.1 * ref.iters))
