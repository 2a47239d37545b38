"""plcg_solve_stencil_noalloc: the stencil solve that allocates nothing.

Callers under a fixed device-memory budget, in allocator-free real-time
loops or plugins that get a stream but no allocator cannot let the solver
cudaMalloc its workspace; this entry point keeps it in a fixed array inside
the library and otherwise runs the solve as plcg_solve does.  Its results
must equal those of plcg_solve (same kernel, same launch shape and flags),
on two calls in a row (the shared array keeps the previous call's contents,
so the second call checks that what must start at zero is cleared), after a
larger solve has left other contents in the array, with the Jacobi
preconditioner and a diagonal shift, and its bounded waits must honour the
timeout test hooks.  This file is collected last so that a failure here
stops a ``-x`` run only after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _env():
    import torch
    from paper_1905_06850_gb300 import build as B
    from paper_1905_06850_gb300 import plcg

    B.build()
    lib = plcg.load()
    torch.cuda.set_device(0)
    return torch, plcg, lib


def _desc(plcg, op, diag_shift=0.0):
    return plcg.plcg_stencil_desc(dim=op["dim"], points=5 if op["dim"] == 2 else 7,
                                  nx=op["nx"], ny=op["ny"], nz=op["nz"] if op["dim"] == 3 else 1,
                                  center=op["center"], off=op["off"], diag_shift=diag_shift)


def _reference(torch, plcg, lib, d, bt, **kw):
    """plcg_solve on a matrix created from the same description: x, result, launch info."""
    h = C.c_void_p()
    assert lib.plcg_create_stencil(C.byref(d), C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                   C.byref(h)) == plcg.PLCG_OK, plcg.last_error()
    x = torch.zeros_like(bt)
    p, keep = plcg.make_params(**kw)
    r = plcg.plcg_result()
    st = lib.plcg_solve(h, bt.data_ptr(), x.data_ptr(), C.byref(p), C.byref(r))
    info = plcg.last_launch()
    lib.plcg_destroy(h)
    del keep
    assert st == plcg.PLCG_OK, plcg.last_error()
    return x.cpu().numpy(), r, info


def _noalloc(torch, plcg, lib, d, bt, **kw):
    x = torch.zeros_like(bt)
    p, keep = plcg.make_params(**kw)
    r = plcg.plcg_result()
    st = lib.plcg_solve_stencil_noalloc(C.byref(d), bt.data_ptr(), x.data_ptr(), C.byref(p),
                                        C.byref(r), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    info = plcg.last_launch()
    del keep
    return st, x.cpu().numpy(), r, info


def test_noalloc_matches_plcg_solve_on_two_calls():
    """Two calls in a row per case, each against plcg_solve: iterate counts,
    solutions (1e-10 FP64, 1e-5 FP32) and the launch (kernel, grid,
    lookahead, poll limit).  The l = 2 FP64 case runs right after an l = 3
    case, so the shared array holds another solve's ring contents; the 2D
    FP32 case uses the Jacobi preconditioner with a diagonal shift."""
    torch, plcg, lib = _env()
    from paper_1905_06850_gb300 import workloads as W

    cases = [(W.config_3d(nx=40), 0.0, dict(method="plcg", l=3, prec="fp64")),
             (W.config_3d(nx=40), 0.0, dict(method="plcg", l=2, prec="fp64")),
             (W.config_2d(nx=100), 0.0, dict(method="plcg", l=1, prec="fp32")),
             (W.config_2d(nx=96), 0.75, dict(method="plcg", l=2, prec="fp32", precond="jacobi")),
             (W.config_2d(nx=64), 0.0, dict(method="cg", l=1, prec="fp64"))]
    for c, shift, kw in cases:
        op = c["op"]
        d = _desc(plcg, op, shift)
        bt = torch.tensor(c["b"], device="cuda")
        lo, hi = c["interval"]
        if kw.get("precond") == "jacobi":   # spectrum of M^{-1} A for the shifted stencil
            cen = op["center"] + shift
            lo, hi = (lo + shift) / cen, (hi + shift) / cen
        kw = dict(kw, interval=(lo, hi), rtol=1e-8)
        x_ref, r_ref, info_ref = _reference(torch, plcg, lib, d, bt, **kw)
        assert r_ref.status == plcg.PLCG_OK
        if kw.get("l") == 2 and kw["prec"] == "fp64":
            assert info_ref["lookahead"] == 1   # the overlap l >= 2 solves of this size use
        tol = 1e-10 if kw["prec"] == "fp64" else 1e-5
        for _ in range(2):
            st, x, r, info = _noalloc(torch, plcg, lib, d, bt, **kw)
            assert st == plcg.PLCG_OK, plcg.last_error()
            assert r.status == plcg.PLCG_OK and r.iters == r_ref.iters, (kw, r.iters, r_ref.iters)
            assert r.true_relres < 1e-8
            assert _rel(x, x_ref) <= tol, (kw, _rel(x, x_ref))
            for key in ("kernel", "grid_ctas", "dyn_smem", "lookahead", "staged", "poll_limit",
                        "force_timeout", "cluster"):
                assert info[key] == info_ref[key], (kw, key, info[key], info_ref[key])


def test_noalloc_bounded_wait_timeout_then_recover():
    """With the test hooks (a short poll bound and a barrier target one
    arrival too high) the solve's first grid barrier runs out: the call
    returns PLCG_ERR_TIMEOUT naming the expired wait, and the next call on
    the same array succeeds."""
    torch, plcg, lib = _env()
    from paper_1905_06850_gb300 import workloads as W

    c = W.config_2d(nx=64)
    d = _desc(plcg, c["op"])
    bt = torch.tensor(c["b"], device="cuda")
    try:
        plcg.set_cluster_rows(0)   # the grid path: the cluster barrier has no bound to expire
        lib.plcg_debug_set_poll_limit(20000)
        lib.plcg_debug_force_barrier_timeout(1)
        st, _, r, info = _noalloc(torch, plcg, lib, d, bt, l=1, interval=c["interval"], rtol=1e-8)
        assert st == plcg.PLCG_ERR_TIMEOUT and r.status == plcg.PLCG_ERR_TIMEOUT
        assert "wait" in plcg.last_error()
        assert info["poll_limit"] == 20000 and info["force_timeout"] == 1
    finally:
        lib.plcg_debug_force_barrier_timeout(0)
        lib.plcg_debug_set_poll_limit(0)
        plcg.set_cluster_rows()
    st, x, r, _ = _noalloc(torch, plcg, lib, d, bt, l=1, interval=c["interval"], rtol=1e-8)
    assert st == plcg.PLCG_OK and r.true_relres < 1e-8


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, plcg, lib = _env()
    n = 256 ** 3
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    d = plcg.plcg_stencil_desc(dim=3, points=7, nx=256, ny=256, nz=256, center=6.0, off=-1.0,
                               diag_shift=0.0)
    p, keep = plcg.make_params(l=1, interval=(0, 12))
    r = plcg.plcg_result()
    st = lib.plcg_solve_stencil_noalloc(C.byref(d), b.data_ptr(), x.data_ptr(), C.byref(p),
                                        C.byref(r), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == plcg.PLCG_ERR_INVALID
    msg = plcg.last_error()
    assert "scratch" in msg and str(32 << 20) in msg
    assert not x.any()
