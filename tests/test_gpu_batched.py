"""GPU parity of plcg_solve_batched (one system per CTA, one persistent launch)
against the FP64 oracle, system by system, on a mixed batch of shifted 2D
Poisson systems (odd and even sides, the batched workload's shapes) and a few
3D ones."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make_batch(count=40, seed=11):
    rng = np.random.default_rng(seed)
    systems = []
    for i in range(count):
        if i % 8 == 7:
            s = int(rng.integers(6, 20))
            op = W.stencil3d(s, s + 1, s - 1, shift=float(rng.uniform(0, 1)))
            iv = (op["center"] - 6.0, op["center"] + 6.0)
        else:
            s = int(rng.integers(16, 97))
            c = float(rng.uniform(0, 1))
            op = W.stencil2d(s, s, shift=c)
            iv = (c, 8.0 + c)
        b = np.random.default_rng([seed, i]).standard_normal(W.op_size(op))
        systems.append((op, b, iv))
    return systems


def run(P, systems, prec, **kw):
    import torch
    mats = [P.Matrix(op) for op, _, _ in systems]
    bs = [torch.tensor(b, device="cuda") for _, b, _ in systems]
    xs = [torch.zeros_like(b) for b in bs]
    st, res = P.solve_batched(mats, bs, xs, lmins=[iv[0] for _, _, iv in systems],
                              lmaxs=[iv[1] for _, _, iv in systems], check=False, prec=prec, **kw)
    out = [x.cpu().numpy() for x in xs]
    for m in mats:
        m.close()
    return st, res, out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("l", [1, 2, 3])
def test_batched_plcg_matches_oracle(P, prec, l):
    systems = make_batch()
    st, res, xs = run(P, systems, prec, l=l, rtol=1e-8)
    assert st == P.PLCG_OK, P.last_error()
    for (op, b, iv), r, x in zip(systems, res, xs):
        oop = W.fp32_rounded(op) if prec == "fp32" else op
        sig = O.chebyshev_shifts(l, *iv)
        ref = O.plcg(oop, b, l=l, sigma=sig, rtol=1e-8, dots_2l1=False)
        assert r.ok and r.true_relres < 1e-8
        assert np.linalg.norm(b - W.rhs(oop, x)) / np.linalg.norm(b) < 1e-8 * 1.0000001
        assert rel(x, ref.x) <= (1e-10 if prec == "fp64" else 1e-5), (op["nx"], rel(x, ref.x))
        # FP32: against the FP64 oracle run with the same refinement segments
        kref = ref.iters if prec == "fp64" else O.refined(oop, b, l=l, sigma=sig, rtol=1e-8).iters
        assert abs(r.iters - kref) <= max(2, int(0.1 * kref)), (op["nx"], r.iters, kref, ref.iters)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_cg_matches_oracle(P, prec):
    systems = make_batch(count=24, seed=5)
    st, res, xs = run(P, systems, prec, method="cg", rtol=1e-8)
    assert st == P.PLCG_OK, P.last_error()
    for (op, b, iv), r, x in zip(systems, res, xs):
        oop = W.fp32_rounded(op) if prec == "fp32" else op
        ref = O.cg(oop, b, rtol=1e-8)
        assert r.ok and r.true_relres < 1e-8
        assert rel(x, ref.x) <= (1e-10 if prec == "fp64" else 1e-5)


def test_batched_equals_single_solves(P):
    """A system gives the same answer alone (plcg_solve, whole grid) and in a
    batch (one CTA) within the FP64 tolerance, and the same iteration count."""
    import torch
    systems = make_batch(count=12, seed=3)
    st, res, xs = run(P, systems, "fp64", l=2, rtol=1e-9)
    assert st == P.PLCG_OK
    for (op, b, iv), r, x in zip(systems, res, xs):
        A = P.Matrix(op)
        bt = torch.tensor(b, device="cuda")
        xt = torch.zeros_like(bt)
        r1 = A.solve(bt, xt, l=2, interval=iv, rtol=1e-9)
        A.close()
        assert r1.iters == r.iters
        assert rel(xt.cpu().numpy(), x) <= 1e-10


def test_batched_edge_cases(P):
    import torch
    systems = make_batch(count=5, seed=8)
    # empty batch
    st, res = P.solve_batched([], [], [], prec="fp32")
    assert st == P.PLCG_OK and res == []
    # one zero right-hand side among others, and l = 5 is rejected
    systems[2] = (systems[2][0], np.zeros_like(systems[2][1]), systems[2][2])
    st, res, xs = run(P, systems, "fp64", l=1, rtol=1e-8)
    assert st == P.PLCG_OK and res[2].iters == 0 and not xs[2].any()
    st, res, xs = run(P, systems, "fp64", l=5, rtol=1e-8)
    assert st == P.PLCG_ERR_UNIMPL
    # the batched kernel computes the l + 1 dot products only
    st, res, xs = run(P, systems, "fp32", l=2, rtol=1e-8, dots_2l1=True)
    assert st == P.PLCG_ERR_UNIMPL and "dots_2l1" in P.last_error()
    # a CSR matrix in the batch is rejected
    csr = P.Matrix(W.random_spd_csr(100, seed=1))
    b = torch.ones(100, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, _ = P.solve_batched([csr], [b], [x], check=False)
    assert st == P.PLCG_ERR_UNIMPL
    csr.close()


@pytest.mark.parametrize("schedule", [(4, 0.01, 1.0), (8, 1.0, 0.5), (1, 1.0, 0.0)],
                         ids=["all-gangs", "default", "no-gangs"])
def test_batched_gang_schedules(P, schedule):
    """The gang path (several thread blocks per system, own barrier and
    partials) and the one-block path both match the oracle."""
    from paper_1905_06850_gb300 import autotune
    systems = make_batch(count=30, seed=17)
    # a few large systems so that gangs have work under the default schedule
    for i, s_ in enumerate((180, 200, 160)):
        op = W.stencil2d(s_, s_, shift=0.002 * (i + 1))
        systems.append((op, np.random.default_rng(100 + i).standard_normal(s_ * s_),
                        (op["center"] - 4.0, op["center"] + 4.0)))
    try:
        autotune.set_schedule(*schedule)
        for prec, l in (("fp64", 1), ("fp32", 2)):
            st, res, xs = run(P, systems, prec, l=l, rtol=1e-8)
            assert st == P.PLCG_OK, P.last_error()
            for (op, b, iv), r, x in zip(systems, res, xs):
                oop = W.fp32_rounded(op) if prec == "fp32" else op
                ref = O.plcg(oop, b, l=l, sigma=O.chebyshev_shifts(l, *iv), rtol=1e-8, dots_2l1=False)
                assert r.ok and r.true_relres < 1e-8
                assert rel(x, ref.x) <= (1e-10 if prec == "fp64" else 1e-5), (op["nx"], schedule)
        st, res, xs = run(P, systems, "fp32", method="cg", rtol=1e-8)
        assert st == P.PLCG_OK and all(r.true_relres < 1e-8 for r in res)
    finally:
        autotune.set_schedule(0)


@pytest.mark.parametrize("shape", [(4, 1, 1), (4, 2, 1), (3, 4, 1), (4, 1, 2)])
def test_batched_launch_shapes(P, shape):
    """Every FP32 launch shape the autotuner chooses among (blocks per SM,
    row groups per thread, vector width; the batch mixes odd and even nx, so
    the 2-wide shape runs both of its paths) solves the batch like the
    oracle, and the tuner installs one of the timed candidates; each
    system's completion time is inside the batch's."""
    from paper_1905_06850_gb300 import autotune
    systems = make_batch(count=24, seed=23)
    try:
        autotune.set_launch(*shape)
        for kw in ({"l": 1}, {"l": 3}, {"method": "cg"}):
            st, res, xs = run(P, systems, "fp32", rtol=1e-8, **kw)
            assert st == P.PLCG_OK, P.last_error()
            for (op, b, iv), r, x in zip(systems, res, xs):
                oop = W.fp32_rounded(op)
                ref = (O.cg(oop, b, rtol=1e-8) if "method" in kw else
                       O.plcg(oop, b, l=kw["l"], sigma=O.chebyshev_shifts(kw["l"], *iv), rtol=1e-8,
                              dots_2l1=False))
                assert r.ok and rel(x, ref.x) <= 1e-5, (shape, kw, op["nx"])
                assert 0.0 < r.latency <= r.seconds * 1.001 + 1e-5, (r.latency, r.seconds)
    finally:
        autotune.set_launch(0, 0)
    mats = [P.Matrix(op) for op, _, _ in systems]
    import torch
    bs = [torch.tensor(b, device="cuda") for _, b, _ in systems]
    sched, shp, times = autotune.tune_batched(mats, bs, [iv[0] for *_, iv in systems],
                                              [iv[1] for *_, iv in systems], prec="fp32", rtol=1e-8, l=1)
    autotune.set_schedule(0)
    autotune.set_launch(0, 0)
    for m in mats:
        m.close()
    assert ("shape", shp) in times and ("schedule", sched) in times
    assert times[("shape", shp)] == min(t for k, t in times.items() if k[0] == "shape")



def test_batched_rejects_unaligned_vectors(P):
    """b and x are read as 16-byte vectors: a system whose b or x is not
    16-byte aligned is rejected before anything runs."""
    import torch
    op = W.stencil2d(16, 16, shift=0.5)
    A = P.Matrix(op)
    buf = torch.zeros(W.op_size(op) + 1, dtype=torch.float64, device="cuda")
    good = torch.ones(W.op_size(op), dtype=torch.float64, device="cuda")
    try:
        for b, x in ((buf[1:], torch.zeros_like(good)), (good, buf[1:])):
            st, _ = P.solve_batched([A], [b], [x], lmins=[0.5], lmaxs=[8.5], check=False, l=1,
                                    prec="fp32")
            assert st == P.PLCG_ERR_INVALID and "16-byte" in P.last_error()
    finally:
        A.close()
