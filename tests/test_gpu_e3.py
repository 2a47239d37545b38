"""GPU parity on the paper's communication-bound toy (Sec. 4, Fig. "lapl",
right): a diagonal operator with the 2D Laplacian's eigenvalues and the
rotated right-hand side.  Its SpMV is one multiply per row, so an iteration
is dominated by the reduction and the grid barrier -- the regime where the
paper sees p(2)-CG overtake p(1)-CG.  Tolerances: FP64 x <= 1e-10 against the
oracle; the residual history (hence the iteration count) equals that of the
Laplacian with the unrotated b (orthogonal invariance)."""
import numpy as np
import pytest
import scipy.fft

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


def gpu_solve(P, op, b, **kw):
    import torch
    A = P.Matrix(op)
    bt = torch.tensor(b, dtype=torch.float64, device="cuda")
    xt = torch.zeros_like(bt)
    res = A.solve(bt, xt, check=False, **kw)
    A.close()
    return xt.cpu().numpy(), res


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_e3_diagonal_100(P, l):
    e = W.e3_diagonal(100)
    lap = W.config_2d(100)
    kw = {"method": "cg"} if l == 0 else {"l": l, "interval": e["interval"]}
    if l == 0:
        ref = O.cg(e["op"], e["b"], rtol=e["rtol"])
    else:
        ref = O.plcg(e["op"], e["b"], l=l, sigma=O.chebyshev_shifts(l, *e["interval"]),
                     rtol=e["rtol"], dots_2l1=False)
    x, res = gpu_solve(P, e["op"], e["b"], rtol=e["rtol"], **kw)
    assert res.ok and res.true_relres < e["rtol"]
    assert rel(x, ref.x) <= 1e-10 and res.iters == ref.iters
    xl, rl = gpu_solve(P, lap["op"], lap["b"], rtol=e["rtol"], **kw)
    assert rl.ok and rl.iters == res.iters
    xr = scipy.fft.idstn(x.reshape(100, 100), type=1, norm="ortho").ravel()
    assert rel(xr, xl) <= 1e-9


def test_e3_diagonal_2000_full_size(P):
    """The paper's size, 4M unknowns (2000^2 eigenvalues): the first 20
    iterates against the oracle element-wise, then full solves for l = 1, 2
    and CG with the true residual checked on the host."""
    e = W.e3_diagonal(2000)
    op, b = e["op"], e["b"]
    lam = op["val"]
    sig = O.chebyshev_shifts(2, *e["interval"])
    ref = O.plcg(op, b, l=2, sigma=sig, rtol=e["rtol"], maxit=20, dots_2l1=False)
    x, res = gpu_solve(P, op, b, l=2, interval=e["interval"], rtol=e["rtol"], maxit=20)
    assert res.status == P.PLCG_ERR_MAXIT and res.iters == 20
    assert rel(x, ref.x) <= 1e-10
    idx = np.random.default_rng(0).integers(0, op["n"], 1000)
    assert np.max(np.abs(x[idx] - ref.x[idx])) <= 1e-9 * np.max(np.abs(ref.x))
    for kw in ({"l": 1, "interval": e["interval"]}, {"l": 2, "interval": e["interval"]},
               {"method": "cg"}):
        x, res = gpu_solve(P, op, b, rtol=e["rtol"], **kw)
        assert res.ok, (kw, res)
        assert np.linalg.norm(b - lam * x) / np.linalg.norm(b) < e["rtol"]
