"""Run one workload through the library a few times: the fixed command that
profiler captures (ncu) of a single solver kernel are taken on.

    python -m paper_1905_06850_gb300.profile_case --workload h27 --nx 96 \\
        --prec fp32 --l 2 --precond jacobi --maxit 30 --warmup 2

Workloads (the seeded generators of ``workloads.py``): ``3d`` (7-point
Laplacian nx^3), ``2d`` (5-point nx^2), ``h27`` (27-point heterogeneous CSR
nx^3, FP32-rounded values), ``e3`` (the diagonal toy with the nx^2 2D
Laplacian eigenvalues), ``batched`` (``--count`` shifted 2D systems, one
persistent launch).  Each run prints one line per solve: status, iterations
and the device time of the launch.
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=["3d", "2d", "h27", "h27v", "e3", "batched"], default="3d")
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--prec", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--method", choices=["plcg", "cg"], default="plcg")
    ap.add_argument("--l", type=int, default=1)
    ap.add_argument("--precond", choices=["none", "jacobi"], default="none")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=0)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--runs", type=int, default=1)
    args = ap.parse_args(argv)

    import torch
    from . import plcg
    from . import workloads as W

    plcg.load()
    dev = torch.device("cuda", 0)
    kw = {"method": args.method, "l": args.l, "rtol": args.rtol, "prec": args.prec,
          "precond": None if args.precond == "none" else args.precond, "check": False}
    if args.maxit:
        kw["maxit"] = args.maxit
    if args.workload == "batched":
        systems = W.batched_systems(args.count)
        mats = [plcg.Matrix(s["op"]) for s in systems]
        bs = [torch.tensor(s["b"], device=dev) for s in systems]
        lo = [s["interval"][0] for s in systems]
        hi = [s["interval"][1] for s in systems]
        for r in range(args.warmup + args.runs):
            xs = [torch.zeros_like(b) for b in bs]
            st, res = plcg.solve_batched(mats, bs, xs, lmins=lo, lmaxs=hi, **kw)
            its = [x.iters for x in res]
            print(f"run {r}: status {st} systems {len(res)} iters max {max(its)} "
                  f"seconds {res[0].seconds:.6f}", flush=True)
        for m in mats:
            m.close()
        return
    if args.workload == "3d":
        c = W.config_3d(nx=args.nx)
    elif args.workload == "2d":
        c = W.config_2d(nx=args.nx)
    elif args.workload == "h27":
        c = W.config_hetero27(nx=args.nx)
    elif args.workload == "h27v":
        c = W.config_hetero27_var27(nx=args.nx)
        c["interval"] = W.shift_interval(c["op"])
    else:
        c = W.e3_diagonal(args.nx)
    op = c["op"]
    interval = W.jacobi_shift_interval(op) if args.precond == "jacobi" else c["interval"]
    A = plcg.Matrix(op, prec=args.prec if op["kind"] != "stencil" else "fp64")
    b = torch.tensor(c["b"], device=dev)
    for r in range(args.warmup + args.runs):
        x = torch.zeros_like(b)
        res = A.solve(b, x, interval=interval, **kw)
        print(f"run {r}: status {res.status} iters {res.iters} restarts {res.restarts} "
              f"seconds {res.seconds:.6f}", flush=True)
    A.close()


if __name__ == "__main__":
    main()
