"""GPU parity of FP64 p(l)-CG on systems of at least 2^19 rows, where the
kernel keeps its bases scaled (Z_j = z^(l)_j / s_j, W^(k)_j = z^(k)_j /
t^(k)_j, phat_m / t^(0)_m, the K5 dots multiplied back by their scales in the
scalar step; l <= 5 on the stencils, l = 1 on CSR and the structured
27-point operator) and rescales by a power of two when a scale leaves
[2^-256, 2^256] (about every 160 iterations on the 3D Laplacian at l = 1).  Against the FP64 oracle,
through the C ABI: iterates before and after a rescale element-wise, whole
solves, and the CSR and structured 27-point operators with Jacobi."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_06850_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NX = 82   # 82^3 = 551,368 rows >= 2^19


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


@pytest.fixture(scope="module")
def lap3d():
    c = W.config_3d(nx=NX)
    assert W.op_size(c["op"]) >= 1 << 19
    return c


@pytest.mark.parametrize("k,dots_2l1", [(1, False), (2, False), (20, False), (170, False), (330, False),
                                        (170, True)])
def test_3d_iterates_across_rescales(P, lap3d, k, dots_2l1):
    """x_k element-wise: before the first rescale (k < 160) and after one
    and two (k = 170, 330); with 2l+1 dots the third dot's scale too."""
    c = lap3d
    sig = O.chebyshev_shifts(1, *c["interval"])
    ref = O.plcg(c["op"], c["b"], l=1, sigma=sig, rtol=1e-14, maxit=k, dots_2l1=dots_2l1)
    x, res = gpu_solve(P, c["op"], c["b"], l=1, rtol=1e-14, maxit=k, interval=c["interval"],
                       dots_2l1=dots_2l1)
    assert res.status == P.PLCG_ERR_MAXIT and res.iters == k
    assert rel(x, ref.x) <= 1e-11, (k, rel(x, ref.x))


def test_3d_whole_solve(P, lap3d):
    c = lap3d
    sig = O.chebyshev_shifts(1, *c["interval"])
    ref = O.plcg(c["op"], c["b"], l=1, sigma=sig, rtol=1e-10, dots_2l1=False)
    x, res = gpu_solve(P, c["op"], c["b"], l=1, rtol=1e-10, interval=c["interval"])
    assert res.ok and res.true_relres < 1e-10
    assert abs(res.iters - ref.iters) <= 1, (res.iters, ref.iters)
    assert rel(x, ref.x) <= 1e-11
    assert rel(x, c["xstar"]) <= 1e-7


@pytest.mark.parametrize("kind", ["csr", "var27"])
def test_jacobi_early_iterates(P, kind):
    """The heterogeneous 27-point operator (CSR and structured layouts) with
    M = diag(A): iterate 6 element-wise (its iterates are rounding-order
    sensitive further on), then a whole solve to the natural-norm rtol."""
    c = W.config_hetero27(nx=NX) if kind == "csr" else W.config_hetero27_var27(nx=NX)
    op, b = c["op"], c["b"]
    interval = W.jacobi_shift_interval(op if kind == "csr" else W.var27_to_csr(op))
    sig = O.chebyshev_shifts(1, *interval)
    ref = O.plcg(op, b, l=1, sigma=sig, rtol=1e-8, maxit=6, dots_2l1=False, precond="jacobi")
    x, res = gpu_solve(P, op, b, l=1, interval=interval, rtol=1e-8, maxit=6, precond="jacobi")
    assert res.status == P.PLCG_ERR_MAXIT and res.iters == 6
    assert rel(x, ref.x) <= 1e-10, rel(x, ref.x)
    x, res = gpu_solve(P, op, b, l=1, interval=interval, rtol=1e-8, precond="jacobi",
                       max_restarts=16)
    assert res.ok and res.true_relres < 1e-8, (res, P.last_error())


@pytest.mark.parametrize("l", [2, 3, 4, 5])
@pytest.mark.parametrize("k", [1, 3, 40, 170, 330])
def test_3d_scaled_l_iterates_across_rescales(P, lap3d, l, k):
    """l >= 2 (every basis recurrence with a unit coefficient): x_k
    element-wise at 1e-11 before and after rescales of the l + 1 scale
    chains, and the launch is the scaled-basis kernel."""
    c = lap3d
    sig = O.chebyshev_shifts(l, *c["interval"])
    ref = O.plcg(c["op"], c["b"], l=l, sigma=sig, rtol=1e-14, maxit=k, dots_2l1=False)
    x, res = gpu_solve(P, c["op"], c["b"], l=l, rtol=1e-14, maxit=k, interval=c["interval"])
    assert res.status == P.PLCG_ERR_MAXIT and res.iters == k
    assert rel(x, ref.x) <= 1e-11, (l, k, rel(x, ref.x))


@pytest.mark.parametrize("l", [2, 3])
def test_3d_scaled_l_whole_solve_and_2l1_dots(P, lap3d, l):
    c = lap3d
    sig = O.chebyshev_shifts(l, *c["interval"])
    ref = O.plcg(c["op"], c["b"], l=l, sigma=sig, rtol=1e-10, dots_2l1=False)
    x, res = gpu_solve(P, c["op"], c["b"], l=l, rtol=1e-10, interval=c["interval"])
    assert res.ok and res.true_relres < 1e-10
    assert abs(res.iters - ref.iters) <= 1, (res.iters, ref.iters)
    assert rel(x, ref.x) <= 1e-11
    ref = O.plcg(c["op"], c["b"], l=l, sigma=sig, rtol=1e-14, maxit=200, dots_2l1=True)
    x, res = gpu_solve(P, c["op"], c["b"], l=l, rtol=1e-14, maxit=200, interval=c["interval"], dots_2l1=True)
    assert res.status == P.PLCG_ERR_MAXIT and rel(x, ref.x) <= 1e-11, rel(x, ref.x)

