"""GPU parity of the structured symmetric 27-point operator (diagonal + 13
forward weights per cell, `plcg_create_var27`) against the FP64 CPU oracle,
through the C ABI.  It is the heterogeneous 27-point operator of the CSR
tests stored without column indices, so the same bars apply: FP64 solution
within max(1e-10, 4x the oracle's rounding-order sensitivity) of the
oracle's, FP32 within 1e-5, true residual < rtol (re-checked on the host),
iteration counts within 10% (FP32 path: its inner solves restart, 50%)."""
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


def gpu_solve(P, op, b, prec="fp64", **kw):
    import torch
    A = P.Matrix(op, prec=prec)
    bt = torch.tensor(b, dtype=torch.float64, device="cuda")
    xt = torch.zeros_like(bt)
    res = A.solve(bt, xt, check=False, prec=prec, **kw)
    A.close()
    return xt.cpu().numpy(), res


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def relres(op, b, x, natural=False):
    A = W.to_scipy(op)
    r = b - A @ x
    if natural:
        m = 1.0 / A.diagonal()
        return np.sqrt(r @ (m * r)) / np.sqrt(b @ (m * b))
    return np.linalg.norm(r) / np.linalg.norm(b)


def sensitivity(op, b, method, l, sig, rtol, precond):
    """The oracle against itself with the unknowns permuted (CSR form): the
    largest relative x difference and iteration spread over three
    permutations."""
    out = [_sensitivity1(op, b, method, l, sig, rtol, precond, seed) for seed in range(3)]
    return max(o[0] for o in out), max(o[1] for o in out)


def _sensitivity1(op, b, method, l, sig, rtol, precond, seed):
    import scipy.sparse as sp
    A = W.to_scipy(op)
    perm = np.random.default_rng(seed).permutation(A.shape[0])
    Ap = sp.csr_matrix(A[perm][:, perm])
    Ap.sort_indices()
    opp = {"kind": "csr", "n": A.shape[0], "rowptr": Ap.indptr.astype(np.int64),
           "col": Ap.indices.astype(np.int32), "val": Ap.data}
    if method == "cg":
        a = O.cg(op, b, rtol=rtol, precond=precond)
        c = O.cg(opp, b[perm], rtol=rtol, precond=precond)
    else:
        a = O.plcg(op, b, l=l, sigma=sig, rtol=rtol, dots_2l1=False, precond=precond)
        c = O.plcg(opp, b[perm], l=l, sigma=sig, rtol=rtol, dots_2l1=False, precond=precond)
    xc = np.empty_like(c.x)
    xc[perm] = c.x
    return rel(xc, a.x), abs(a.iters - c.iters) / max(a.iters, 1)


def check(P, op, b, method, l, rtol, prec="fp64", precond=None, max_restarts=8):
    oop = W.fp32_rounded(op) if prec == "fp32" else op
    interval = W.jacobi_shift_interval(oop) if precond else W.shift_interval(oop)
    sig = O.chebyshev_shifts(l, *interval) if method == "plcg" else None
    if method == "cg":
        ref = O.cg(oop, b, rtol=rtol, precond=precond)
    else:
        ref = O.plcg(oop, b, l=l, sigma=sig, rtol=rtol, dots_2l1=False, precond=precond,
                     max_restarts=max_restarts)
    assert ref.status == O.ORC_OK
    if prec == "fp64":
        # classic CG: 8x (its recursive residual carries the rounding of every
        # step's dots, and the GPU's tree summation is an order no permutation
        # of the serial sum reproduces); p(l)-CG: 4x
        sx, sk = sensitivity(oop, b, method, l, sig, rtol, precond)
        tol, slack = max(1e-10, (8 if method == "cg" else 4) * sx), max(0.1, 2 * sk)
    else:
        tol, slack = 1e-5, 0.5
    x, res = gpu_solve(P, op, b, prec=prec, method=method, l=l, interval=interval, rtol=rtol,
                       precond=precond, max_restarts=max_restarts)
    assert res.status == P.PLCG_OK, (res, P.last_error())
    assert res.true_relres < rtol
    assert relres(oop, b, x, natural=bool(precond)) < rtol * 1.000001
    assert rel(x, ref.x) <= tol, (rel(x, ref.x), tol)
    assert abs(res.iters - ref.iters) <= max(1, int(slack * ref.iters)), (res.iters, ref.iters)
    return x, res


V27 = W.hetero27_var27(14, 12, 10, seed=3)
V27_B = W.rhs(V27, np.random.default_rng(4).standard_normal(W.op_size(V27)))


@pytest.mark.parametrize("l", [1, 2, 3])
def test_var27_fp64(P, l):
    check(P, V27, V27_B, "plcg", l, 1e-8)


@pytest.mark.parametrize("l", [1, 2])
def test_var27_fp64_jacobi(P, l):
    check(P, V27, V27_B, "plcg", l, 1e-8, precond="jacobi")


@pytest.mark.parametrize("l", [1, 2])
def test_var27_fp32_jacobi(P, l):
    check(P, V27, V27_B, "plcg", l, 1e-8, prec="fp32", precond="jacobi", max_restarts=64)


@pytest.mark.parametrize("prec,precond", [("fp64", None), ("fp32", "jacobi"), ("fp64", "jacobi")])
def test_var27_classic_cg(P, prec, precond):
    check(P, V27, V27_B, "cg", 1, 1e-8, prec=prec, precond=precond)


def test_var27_equals_csr_form_and_early_iterates(P):
    """Iterates 1 and 6 equal the oracle's element-wise; the solve on the
    structured layout equals the one on the CSR form of the same matrix."""
    sig = O.chebyshev_shifts(2, *W.shift_interval(V27))
    for k in (1, 6):
        ref = O.plcg(V27, V27_B, l=2, sigma=sig, rtol=1e-8, maxit=k, dots_2l1=False)
        x, res = gpu_solve(P, V27, V27_B, l=2, interval=W.shift_interval(V27), rtol=1e-8, maxit=k)
        assert res.status == P.PLCG_ERR_MAXIT and res.iters == k
        assert rel(x, ref.x) <= 1e-10
    x1, r1 = gpu_solve(P, V27, V27_B, l=1, interval=W.shift_interval(V27), rtol=1e-10)
    x2, r2 = gpu_solve(P, W.var27_to_csr(V27), V27_B, l=1, interval=W.shift_interval(V27), rtol=1e-10)
    assert r1.ok and r2.ok and rel(x1, x2) <= 1e-7


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 7), (3, 1, 4), (2, 3, 1), (5, 2, 3), (33, 3, 2)])
def test_var27_ragged_grids(P, dims):
    """Degenerate and ragged grids: 1-wide axes, odd sizes, a single cell."""
    op = W.hetero27_var27(*dims, seed=sum(dims))
    n = W.op_size(op)
    b = np.random.default_rng(n).standard_normal(n)
    xs = np.linalg.solve(W.to_scipy(op).toarray(), b)
    for kw in ({"l": 1}, {"l": 2}, {"method": "cg"}, {"l": 1, "precond": "jacobi"}):
        interval = W.jacobi_shift_interval(op) if "precond" in kw else W.shift_interval(op)
        x, res = gpu_solve(P, op, b, interval=interval, rtol=1e-12, max_restarts=32, **kw)
        assert res.ok, (dims, kw, res)
        assert rel(x, xs) <= 1e-9, (dims, kw)


@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 1, 4), (33, 3, 2), (5, 2, 3), (17, 9, 13), (40, 30, 20),
                                  (275, 2, 3), (300, 3, 2)])
def test_var27_fp32_tiles_ragged_grids(P, dims):
    """The FP32 p(l)-CG sweep (and classic CG's SpMV) stages shared-memory
    tiles (coefficients, z by plane -- or by line when a plane's three lines
    do not fit, nx > 275 -- and, in the p(l)-CG steady state, the vector
    operands) and applies rows
    without boundary tests (out-of-grid entries stored as zero, zero halos
    around the arrays): ragged and degenerate grids, units that straddle the
    grid's ends, l = 1..5 with and without Jacobi (l > 3 stages the operator
    only), refined to rtol 1e-10."""
    import scipy.sparse.linalg as spl
    op = W.hetero27_var27(*dims, seed=7 + sum(dims))
    n = W.op_size(op)
    b = np.random.default_rng(n + 1).standard_normal(n)
    A = W.to_scipy(W.fp32_rounded(op)).tocsc()
    xs = spl.spsolve(A, b)
    for kw in ({"l": 1}, {"l": 2}, {"l": 3}, {"l": 1, "precond": "jacobi"}, {"l": 3, "precond": "jacobi"},
               {"l": 4}, {"l": 5, "precond": "jacobi"},   # l > 3: tiles without vector slots
               {"method": "cg"}, {"method": "cg", "precond": "jacobi"}):   # classic CG's tiled SpMV
        oop = W.fp32_rounded(op)
        interval = W.jacobi_shift_interval(oop) if "precond" in kw else W.shift_interval(oop)
        x, res = gpu_solve(P, op, b, prec="fp32", interval=interval, rtol=1e-10, max_restarts=64, **kw)
        assert res.ok, (dims, kw, res, P.last_error())
        assert rel(x, xs) <= 1e-8, (dims, kw, rel(x, xs))


def test_var27_rejects_bad_arguments(P):
    import ctypes as C
    lib = P.load()
    h = C.c_void_p()
    coef = np.ones((14, 8))
    assert lib.plcg_create_var27(0, 2, 2, coef.ctypes.data, 0, 0, None, C.byref(h)) == P.PLCG_ERR_INVALID
    bad = coef.copy()
    bad[3, 5] = np.nan
    assert lib.plcg_create_var27(2, 2, 2, bad.ctypes.data, 0, 0, None, C.byref(h)) == P.PLCG_ERR_INVALID
    assert lib.plcg_create_var27(2, 2, 2, None, 0, 0, None, C.byref(h)) == P.PLCG_ERR_INVALID


def test_var27_full_size_128(P):
    """The 128^3 heterogeneous workload in the structured layout (FP32 values,
    FP64 correction, Jacobi) in the benchmark's launch configuration: iterate
    6 element-wise on the FP64 path, iterate 1 on the FP32 path, then full
    FP32 solves for l = 1, 2 and CG to the natural-norm rtol, checked on the
    host."""
    c = W.config_hetero27_var27(nx=128)
    op, b = c["op"], c["b"]
    interval = W.jacobi_shift_interval(op)
    sig = O.chebyshev_shifts(2, *interval)
    for prec, k, tol in (("fp64", 6, 1e-10), ("fp32", 1, 1e-6)):
        ref = O.plcg(op, b, l=2, sigma=sig, rtol=1e-8, maxit=k, dots_2l1=False, precond="jacobi")
        x, res = gpu_solve(P, op, b, prec=prec, l=2, interval=interval, rtol=1e-8, maxit=k,
                           precond="jacobi")
        assert res.status == P.PLCG_ERR_MAXIT and res.iters == k
        assert rel(x, ref.x) <= tol, (prec, rel(x, ref.x))
    for kw in ({"l": 1}, {"l": 2}, {"method": "cg"}):
        x, res = gpu_solve(P, op, b, prec="fp32", interval=interval, rtol=1e-8, precond="jacobi",
                           max_restarts=64, **kw)
        assert res.ok, (kw, res, P.last_error())
        assert relres(op, b, x, natural=True) < 1e-8 * 1.000001
