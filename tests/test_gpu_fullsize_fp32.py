"""The FP32 path at full size, element-wise against the FP64 oracle's solution.

FP32 vectors and matrix values with FP64 dots, scalars and outer refinement
must match the FP64 oracle (on the FP32-rounded operator) to 1e-5 in
||x - x_oracle|| / ||x_oracle||, with iteration counts within 10%, on the
workloads and launch configurations the benchmark times: the 256^3 7-point
Laplacian (p(1)-CG and p(2)-CG, rtol 1e-8) and the 128^3 heterogeneous
27-point CSR with the Jacobi preconditioner (p(2)-CG and p(3)-CG on the
shift interval plcg_estimate_interval returns).  The oracle's serial solves
run in a spawn process pool while the GPU works.
"""
import numpy as np
import pytest

from oracle import jobs
from paper_1905_06850_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_fp32_full_size_against_the_oracle():
    import torch
    from paper_1905_06850_gb300 import build as B
    from paper_1905_06850_gb300 import plcg

    pool = jobs.pool()
    try:
        fut = {}
        for l in (1, 2):
            fut[("3d", l)] = pool.submit(jobs.run, {"key": f"3d{l}", "workload": {"kind": "3d", "nx": 256},
                                                    "l": l, "interval": (0.0, 12.0), "rtol": 1e-8})
        B.build()
        plcg.load()
        torch.cuda.set_device(0)
        c = W.config_hetero27(nx=128)
        A = plcg.Matrix(c["op"], prec="fp32")
        _, hi = A.estimate_interval(steps=30, prec="fp32", precond="jacobi")
        iv = (0.0, 1.02 * hi)
        for l in (2, 3):
            fut[("h27", l)] = pool.submit(jobs.run, {"key": f"h27{l}", "workload": {"kind": "h27", "nx": 128},
                                                     "l": l, "interval": iv, "rtol": 1e-8,
                                                     "precond": "jacobi", "max_restarts": 64})
        got = {}
        b = torch.tensor(c["b"], device="cuda")
        for l in (2, 3):
            x = torch.zeros_like(b)
            r = A.solve(b, x, l=l, interval=iv, rtol=1e-8, prec="fp32", precond="jacobi", max_restarts=64)
            got[("h27", l)] = (x.cpu().numpy(), r)
        A.close()
        c3 = W.config_3d(nx=256)
        A = plcg.Matrix(c3["op"])
        b = torch.tensor(c3["b"], device="cuda")
        for l in (1, 2):
            x = torch.zeros_like(b)
            r = A.solve(b, x, l=l, interval=c3["interval"], rtol=1e-8, prec="fp32")
            got[("3d", l)] = (x.cpu().numpy(), r)
        A.close()
        for key, (x, r) in got.items():
            _, xo, it, _, _ = fut[key].result()
            err = _rel(x, xo)
            print(f"{key}: err_vs_oracle {err:.3e}, iterations {r.iters} vs oracle {it}")
            assert r.ok and err <= 1e-5, (key, err)
            assert abs(r.iters - it) <= max(1, int(0.1 * it)), (key, r.iters, it)
    finally:
        pool.shutdown(cancel_futures=True)
