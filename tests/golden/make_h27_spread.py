"""Writes h27_128_oracle_spread.json: how far the FP64 oracle's iteration
and restart counts move on the 27-point heterogeneous CSR 128^3 workload
(M = I, rtol 1e-8) when the Chebyshev interval [0, lmax] moves by a few parts
in 10^9 -- square-root breakdowns (Sec. 2.2) are rounding events, so the
restart points, and with them the counts, are chaotic on this operator.
The base lmax is 1.02 times the largest Ritz value of 30 CG steps (the
interval the benchmark uses).  Calls only the oracle.

    python tests/golden/make_h27_spread.py [processes]
"""
import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

LMAX = 566.606447
PERTURB = (-2e-9, -1e-9, 0.0, 1e-9, 2e-9)


def one(args):
    l, d = args
    from oracle import jobs
    job = {"key": f"{l}:{d}", "workload": {"kind": "h27", "nx": 128}, "method": "cg" if l == 0 else "plcg",
           "l": max(l, 1), "interval": (0.0, LMAX * (1.0 + d)), "rtol": 1e-8, "max_restarts": 1000}
    _, _, iters, restarts, secs = jobs.run(job)
    return l, d, iters, restarts, secs


if __name__ == "__main__":
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    work = [(0, 0.0)] + [(l, d) for l in (1, 2, 3) for d in PERTURB]
    with ProcessPoolExecutor(procs) as ex:
        rows = list(ex.map(one, work))
    out = {"workload": "27-point heterogeneous CSR 128^3 (FP32-rounded values), M = I, rtol 1e-8, "
                       "x0 = 0, l+1 dots, max_restarts 1000",
           "interval": [0.0, LMAX], "relative_perturbations": list(PERTURB), "runs": {}}
    for l, d, iters, restarts, _ in rows:
        key = "classic_cg" if l == 0 else f"plcg_l{l}"
        out["runs"].setdefault(key, []).append({"perturbation": d, "iters": iters, "restarts": restarts})
    for key, runs in out["runs"].items():
        its = [r["iters"] for r in runs]
        out["runs"][key] = {"runs": runs, "iters_min": min(its), "iters_max": max(its)}
    with open(os.path.join(HERE, "h27_128_oracle_spread.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: (v["iters_min"], v["iters_max"]) for k, v in out["runs"].items()}))
