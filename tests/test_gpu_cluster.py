"""The cluster-resident path for small systems (the grid is one thread-block
cluster of up to 16 CTAs: cluster barrier, dot partials read through
distributed shared memory) against the FP64 oracle, with the same bars as
the grid path: FP64 1e-10 and the oracle's iteration count, FP32 1e-5; and
against the grid path on the same systems."""
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
    yield plcg
    plcg.set_cluster_rows()


def _solve(P, op, b, rows, **kw):
    import torch
    P.set_cluster_rows(rows)
    A = P.Matrix(op, prec=kw.get("prec", "fp64"))
    bt = torch.tensor(b, device="cuda")
    x = torch.zeros_like(bt)
    r = A.solve(bt, x, check=False, **kw)
    info = P.last_launch()
    A.close()
    return x.cpu().numpy(), r, info


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [("2d100", lambda: W.config_2d()), ("2d45", lambda: W.config_2d(nx=45)),
         ("3d24", lambda: W.config_3d(nx=24)), ("e3_100", lambda: W.e3_diagonal(100))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("method,l", [("plcg", 1), ("plcg", 2), ("plcg", 3), ("plcg", 4), ("cg", 1)])
def test_cluster_path_matches_the_oracle(P, name, make, method, l):
    c = make()
    op, b = c["op"], c["b"]
    rtol = c.get("rtol", 1e-8)
    if method == "cg":
        ref = O.cg(op, b, rtol=rtol)
    else:
        ref = O.plcg(op, b, l=l, sigma=O.chebyshev_shifts(l, *c["interval"]), rtol=rtol, dots_2l1=False)
    x, r, info = _solve(P, op, b, 1 << 20, method=method, l=l, interval=c["interval"], rtol=rtol)
    assert info["cluster"] > 0, info
    assert r.ok and r.true_relres < rtol, (r, P.last_error())
    assert _rel(x, ref.x) <= 1e-10, (_rel(x, ref.x), r.iters, ref.iters)
    assert r.iters == ref.iters, (r.iters, ref.iters)
    xg, rg, ig = _solve(P, op, b, 0, method=method, l=l, interval=c["interval"], rtol=rtol)
    assert ig["cluster"] == 0 and rg.iters == r.iters and _rel(x, xg) <= 1e-10


@pytest.mark.parametrize("l", [1, 2])
def test_cluster_path_fp32_and_jacobi_stencil(P, l):
    c = W.config_3d(nx=20)
    op, b = c["op"], c["b"]
    ref = O.plcg(W.fp32_rounded(op), b, l=l, sigma=O.chebyshev_shifts(l, *c["interval"]), rtol=1e-8,
                 dots_2l1=False)
    x, r, info = _solve(P, op, b, 1 << 20, l=l, interval=c["interval"], rtol=1e-8, prec="fp32")
    assert info["cluster"] > 0 and r.ok and r.refinements >= 1
    assert _rel(x, ref.x) <= 1e-5
    refj = O.plcg(op, b, l=l, sigma=O.chebyshev_shifts(l, *W.jacobi_shift_interval(op)), rtol=1e-8,
                  dots_2l1=False, precond="jacobi")
    x, r, info = _solve(P, op, b, 1 << 20, l=l, interval=W.jacobi_shift_interval(op), rtol=1e-8,
                        precond="jacobi")
    assert info["cluster"] > 0 and r.ok and _rel(x, refj.x) <= 1e-10 and r.iters == refj.iters


@pytest.mark.parametrize("n", [1, 2, 7, 300])
def test_cluster_path_tiny_and_edge_cases(P, n):
    op = W.stencil2d(n, 1)
    b = np.arange(1, n + 1, dtype=np.float64)
    for l in (1, 3):
        x, r, info = _solve(P, op, b, 1 << 20, l=l, rtol=1e-12)
        assert info["cluster"] > 0 and r.ok
        assert _rel(x, np.linalg.solve(W.to_scipy(op).toarray(), b)) < 1e-11
    x, r, info = _solve(P, op, np.zeros(n), 1 << 20, l=2)
    assert r.ok and r.iters == 0 and not x.any()
    # the restart path: poor shifts, breakdowns and restarts on one cluster
    if n == 300:
        c = W.config_2d(nx=40)
        x, r, info = _solve(P, c["op"], c["b"], 1 << 20, l=2, interval=(0, 1), rtol=1e-8, max_restarts=100)
        assert info["cluster"] > 0 and r.ok and r.restarts > 0 and r.true_relres < 1e-8


def test_cluster_path_repeatable(P):
    c = W.config_2d()
    x1, r1, _ = _solve(P, c["op"], c["b"], 1 << 20, l=2, interval=c["interval"], rtol=1e-8)
    x2, r2, _ = _solve(P, c["op"], c["b"], 1 << 20, l=2, interval=c["interval"], rtol=1e-8)
    assert r1.iters == r2.iters and np.array_equal(x1, x2)
