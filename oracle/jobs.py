"""Oracle solves described by plain dicts, for running in worker processes.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: the tests and
``bench.py`` (its CPU-baseline leg and the statement of each FP32 result's
error against the FP64 oracle, outside every timed region) run these in a
process pool started with the spawn method, so that the oracle's serial FP64
solves of the large workloads overlap the GPU work.

A job is ``{"key", "workload": {...}, "method": "plcg"|"cg", "l", "interval",
"rtol", "precond", "max_restarts"}``; ``workload`` names one of the seeded
input generators (the same ones the GPU side is fed from).
"""
from __future__ import annotations

import os
import time


def workload(w: dict):
    """(operator, b) of a workload description: "3d" (7-point Laplacian, nx),
    "h27" (the FP32-rounded 27-point heterogeneous CSR, nx), "batched" (one
    system of the shifted 2D batch: index, count), "2d" (5-point Laplacian,
    nx)."""
    from paper_1905_06850_gb300 import workloads as W
    if w["kind"] == "3d":
        c = W.config_3d(nx=w["nx"], seed=2)
        return c["op"], c["b"]   # the Laplacian's coefficients are exact in FP32
    if w["kind"] == "h27":
        c = W.config_hetero27(nx=w["nx"])
        return c["op"], c["b"]
    if w["kind"] == "batched":
        s = W.batched_system(w["index"], count=w["count"])
        return s["op"], s["b"]   # FP32-rounded coefficients
    if w["kind"] == "2d":
        c = W.config_2d(nx=w["nx"])
        return c["op"], c["b"]
    raise ValueError(f"unknown workload {w['kind']!r}")


def warm(_=None):
    """Loads the oracle in a worker (so that a timed batch of run() calls
    does not include the workers' start-up); returns the worker's pid."""
    from oracle import oracle as O   # noqa: F401  (builds nothing: imports and loads the library)
    from paper_1905_06850_gb300 import workloads as W   # noqa: F401
    return os.getpid()


def run(job: dict):
    """One FP64 oracle solve (the worker lowers its own priority): returns
    (key, x, iterations, restarts, seconds)."""
    try:
        os.nice(10)
    except OSError:
        pass
    from oracle import oracle as O
    op, b = workload(job["workload"])
    t0 = time.perf_counter()
    if job.get("method", "plcg") == "cg":
        r = O.cg(op, b, rtol=job["rtol"], precond=job.get("precond"), max_restarts=job.get("max_restarts", 8))
    else:
        sig = O.chebyshev_shifts(job["l"], *job["interval"])
        r = O.plcg(op, b, l=job["l"], sigma=sig, rtol=job["rtol"], dots_2l1=False,
                   max_restarts=job.get("max_restarts", 8), precond=job.get("precond"))
    return job["key"], r.x, int(r.iters), int(getattr(r, "restarts", 0)), time.perf_counter() - t0


def pool(max_workers: int | None = None):
    """A process pool for run() (spawn start method: safe after CUDA is up)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = max_workers or max(1, min(12, (os.cpu_count() or 4) - 2))
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
