"""GPU tests of the serving path (plcg_server_create / plcg_submit / plcg_poll /
plcg_wait): continuous batching of mixed solves."""
import time

import numpy as np
import pytest
from test_gpu_solver import oracle_sensitivity

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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def mix(seed=21):
    """Requests of mixed type, size, precision and method."""
    rng = np.random.default_rng(seed)
    reqs = []
    kinds = ["2d", "3d", "csr"]
    for i in range(18):
        kind = kinds[i % 3]
        if kind == "2d":
            s = int(rng.integers(20, 160))
            op = W.stencil2d(s, s, shift=float(rng.uniform(0, 0.5)))
        elif kind == "3d":
            s = int(rng.integers(10, 48))
            op = W.stencil3d(s, s, s)
        else:
            op = W.random_spd_csr(int(rng.integers(500, 30000)), seed=int(rng.integers(1 << 30)))
        prec = "fp32" if i % 2 else "fp64"
        if kind == "csr":
            op_used = W.fp32_rounded(op) if prec == "fp32" else op
        else:
            op_used = W.fp32_rounded(op) if prec == "fp32" else op
        kw = {"rtol": 1e-8, "prec": prec, "interval": W.shift_interval(op)}
        if i % 5 == 4:
            kw["method"] = "cg"
        else:
            kw["l"] = 1 + (i % 3)
        b = np.random.default_rng([seed, i]).standard_normal(W.op_size(op))
        reqs.append({"op": op, "op_used": op_used, "b": b, "kw": kw})
    return reqs


def submit_all(P, S, reqs):
    import torch
    out = []
    for r in reqs:
        A = P.Matrix(r["op"], prec=r["kw"]["prec"])
        b = torch.tensor(r["b"], device="cuda")
        x = torch.zeros_like(b)
        t = S.submit(A, b, x, **r["kw"])
        out.append((A, b, x, t))
    return out


def test_serving_mix_matches_oracle_and_alone(P):
    reqs = mix()
    S = P.Server()
    handles = submit_all(P, S, reqs)
    results = [S.wait(t) for (_, _, _, t) in handles]
    xs_mix = [x.cpu().numpy() for (_, _, x, _) in handles]
    for r, res, x in zip(reqs, results, xs_mix):
        assert res.ok, res
        assert res.true_relres < 1e-8
        opu = r["op_used"]
        kw = r["kw"]
        if kw.get("method") == "cg":
            ref = O.cg(opu, r["b"], rtol=1e-8)
        else:
            l = kw["l"]
            ref = O.plcg(opu, r["b"], l=l, sigma=O.chebyshev_shifts(l, *kw["interval"]), rtol=1e-8,
                         dots_2l1=False, max_restarts=64)
        # FP64 stencil requests: the single-solve bar, 1e-10; FP64 random-CSR
        # requests: max(1e-10, 4x the oracle's own rounding-order sensitivity
        # on that operator, measured here); FP32 path: 1e-5
        if kw["prec"] != "fp64":
            tol = 1e-5
        elif opu["kind"] == "csr":
            sens_x, _ = oracle_sensitivity(opu, r["b"], kw.get("l", 0),
                                           None if kw.get("method") == "cg"
                                           else O.chebyshev_shifts(kw["l"], *kw["interval"]), 1e-8, False,
                                           method=kw.get("method", "plcg"))
            tol = max(1e-10, 4 * sens_x)
        else:
            tol = 1e-10
        assert rel(x, ref.x) <= tol, (opu["kind"], kw, rel(x, ref.x), tol)
        assert np.linalg.norm(r["b"] - W.rhs(opu, x)) / np.linalg.norm(r["b"]) < 1e-8 * 1.0000001
    # each request alone through the same server: bit-identical x
    for r, x_mix in zip(reqs, xs_mix):
        (A, b, x, t), = submit_all(P, S, [r])
        res = S.wait(t)
        assert res.ok
        assert np.array_equal(x.cpu().numpy(), x_mix)
    S.close()


def test_admission_by_memory_budget(P):
    """A budget that holds only a couple of workspaces: requests queue and
    are admitted as memory frees up; all complete."""
    import torch
    op = W.stencil3d(64, 64, 64)
    S = P.Server(mem_budget_bytes=2 * 64 ** 3 * 8 * 14, max_inflight=8)
    A = P.Matrix(op)
    bufs = []
    tickets = []
    for i in range(6):
        b = torch.tensor(np.random.default_rng(i).standard_normal(64 ** 3), device="cuda")
        x = torch.zeros_like(b)
        bufs.append((b, x))
        tickets.append(S.submit(A, b, x, l=1, interval=(0, 12), rtol=1e-8))
    res = [S.wait(t) for t in tickets]
    assert all(r.ok for r in res)
    # a request larger than the whole budget is refused at submission
    big = P.Matrix(W.stencil3d(128, 128, 128))
    b = torch.ones(128 ** 3, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(P.PlcgError) as e:
        S.submit(big, b, x, l=1, interval=(0, 12))
    assert e.value.status == P.PLCG_ERR_NOMEM
    S.close()


def test_requests_overlap_on_the_device(P):
    """Continuous batching, not a queue: a short request submitted after a
    long one is admitted while the long one runs and finishes first."""
    import torch
    S = P.Server()
    big = P.Matrix(W.stencil2d(1024, 1024))
    bb = torch.tensor(np.random.default_rng(1).standard_normal(1024 ** 2), device="cuda")
    xb = torch.zeros_like(bb)
    small = P.Matrix(W.stencil2d(32, 32))
    bs = torch.tensor(np.random.default_rng(2).standard_normal(32 ** 2), device="cuda")
    xs = torch.zeros_like(bs)
    t_big = S.submit(big, bb, xb, l=1, interval=(0, 8), rtol=1e-8)
    time.sleep(0.002)
    t_small = S.submit(small, bs, xs, l=1, interval=(0, 8), rtol=1e-8)
    order = []
    pending = {t_big, t_small}
    deadline = time.time() + 60
    while pending and time.time() < deadline:
        for t in list(pending):
            r = S.poll(t)
            if r is not None:
                assert r.ok
                order.append(t)
                pending.discard(t)
    assert order == [t_small, t_big]
    S.close()


def test_poll_semantics_and_errors(P):
    import torch
    S = P.Server()
    A = P.Matrix(W.stencil2d(200, 200))
    b = torch.tensor(np.random.default_rng(3).standard_normal(200 ** 2), device="cuda")
    x = torch.zeros_like(b)
    t = S.submit(A, b, x, l=2, interval=(0, 8), rtol=1e-10)
    r = S.wait(t)
    assert r.ok and r.latency >= r.seconds > 0
    with pytest.raises(P.PlcgError):      # already collected
        S.poll(t)
    with pytest.raises(P.PlcgError):
        S.poll(123456789)
    # a request that exhausts its budget reports MAXIT through poll
    x.zero_()
    t = S.submit(A, b, x, l=1, interval=(0, 8), rtol=1e-10, maxit=5)
    r = S.wait(t)
    assert r.status == P.PLCG_ERR_MAXIT and r.iters == 5
    # destroy with requests still queued or running: they complete first
    xs = [torch.zeros_like(b) for _ in range(4)]
    ts = [S.submit(A, b, xx, l=1, interval=(0, 8), rtol=1e-8) for xx in xs]
    S.close()
    for xx in xs:
        assert np.linalg.norm(b.cpu().numpy() - W.rhs(W.stencil2d(200, 200), xx.cpu().numpy())) \
            < 1e-8 * np.linalg.norm(b.cpu().numpy()) * 1.0000001
