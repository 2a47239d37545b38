"""plcg_solve_stencil_noalloc: the stencil solve that allocates nothing.

Callers under a fixed device-memory budget, in allocator-free real-time
loops or plugins that get a stream but no allocator cannot let the solver
cudaMalloc its workspace; this entry point keeps it in a fixed array inside
the library.  Its results must equal those of plcg_solve (same kernels, same
launch shape), on two calls in a row (the shared array keeps the previous
call's contents, so the second call checks that what must start at zero is
cleared).  This file is collected last so that a failure here stops a
``-x`` run only after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_plcg_solve_on_two_calls():
    import torch
    from paper_1905_06850_gb300 import build as B
    from paper_1905_06850_gb300 import plcg
    from paper_1905_06850_gb300 import workloads as W

    B.build()
    lib = plcg.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(W.config_3d(nx=40), "fp64", 2, "plcg"), (W.config_2d(nx=100), "fp32", 1, "plcg"),
             (W.config_2d(nx=64), "fp64", 1, "cg")]
    for c, prec, l, method in cases:
        op, b = c["op"], c["b"]
        bt = torch.tensor(b, device="cuda")
        A = plcg.Matrix(op)
        x_ref = torch.zeros_like(bt)
        r_ref = A.solve(bt, x_ref, method=method, l=l, interval=c["interval"], rtol=1e-8, prec=prec)
        A.close()
        d = plcg.plcg_stencil_desc(dim=op["dim"], points=5 if op["dim"] == 2 else 7,
                                   nx=op["nx"], ny=op["ny"], nz=op["nz"] if op["dim"] == 3 else 1,
                                   center=op["center"], off=op["off"], diag_shift=0.0)
        p, keep = plcg.make_params(method=method, l=l, interval=c["interval"], rtol=1e-8, prec=prec)
        xr = x_ref.cpu().numpy()
        tol = 1e-10 if prec == "fp64" else 1e-5
        for _ in range(2):
            x = torch.zeros_like(bt)
            r = plcg.plcg_result()
            st = lib.plcg_solve_stencil_noalloc(C.byref(d), bt.data_ptr(), x.data_ptr(), C.byref(p),
                                                C.byref(r), C.c_void_p(stream))
            assert st == plcg.PLCG_OK, plcg.last_error()
            assert r.status == plcg.PLCG_OK and r.iters == r_ref.iters
            assert r.true_relres < 1e-8
            assert _rel(x.cpu().numpy(), xr) <= tol
        del keep


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1905_06850_gb300 import plcg

    lib = plcg.load()
    torch.cuda.set_device(0)
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
