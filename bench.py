"""Benchmark: p(l)-CG on the 3D 7-point Laplacian 256^3 (n = 16.8M), FP64, rtol 1e-8.

One step = one full solve of A x = b from x0 = 0 (every iteration, the true
residual check and any restart run in one persistent kernel launch).  The JSON
line reports p(l)-CG iterations/s (the headline), the solve's algorithmic HBM
GB/s, classic CG on the same system and GPU, the FP32-with-FP64-correction
path, an l sweep, an end-to-end number through the host-pointer C entry point,
the dominant kernel's roofline and the FP64 CPU oracle timed on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own copy of the system
(independent replicas, weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "p(l)-CG iterations/s, 3D 7-point Laplacian 256^3 FP64, rtol 1e-8"
UNIT = "iter/s"
NX = 256
RTOL = 1e-8
L_HEAD = 1


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_over_ranks(t_local: float, units_local: float, world: int, device=None):
    """Whole-job figures of a timed region: the slowest rank's time (MAX) and
    the units all ranks processed (SUM); one process: the local values."""
    if world <= 1:
        return float(t_local), float(units_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1905_06850_gb300", "csrc"))):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(ROOT, "paper_1905_06850_gb300", "csrc", f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_record(name: str):
    """A committed ncu summary (profiles/*.json), or None when it is missing
    or its kernel-source hash no longer matches the current sources."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d


def passes_per_iter(l: int, method: str) -> int:
    """Streaming passes over length-n vectors per iteration (fused sweep,
    l+1 dots): 3 per basis (read 2, write 1) + 4 for p and x + extra dot
    operands z^(l)_j for l >= 4; classic CG: 10."""
    if method == "cg":
        return 10
    return 3 * (l + 1) + 4 + max(0, l - 3)


def dp_flops_per_point(l: int) -> int:
    """Algorithmic FP64 flops per row per p(l)-CG iteration on the 7-point
    constant-coefficient stencil: the SpMV (5 neighbour adds, center*c +
    off*sum: 8 flops) plus the (6l + 10) flops of AXPYs and dot products
    that Table 1 of the paper counts."""
    return 8 + 6 * l + 10


# Flops per row and iteration that the FP64 p(1)-CG stencil sweep (scaled
# bases, two rows per thread) issues on the FP64 pipe: 8 FMAs -- K4's two
# recurrences, K6 and the two K5 dots; the six-neighbour sum runs on the
# integer units and the SpMV's multiplies are folded into the recurrences.
DP_PIPE_FLOPS_L1 = 16


def stencil_roofline(*, n, nx, l, prec, iters, seconds, hbm_peak, hbm_src, dp_peak_tf, dp_src, rec=None):
    """The roofline object of the 3D 7-point p(l)-CG solve (one launch of
    ``iters`` iterations and 2 FP64 residual sweeps in ``seconds``): the HBM
    fraction (algorithmic bytes over the measured copy bandwidth) and, for
    FP64 sweeps, the FP64 one (flops over the measured FMA rate); "bound"
    names the larger, the other sits beside it.  ``rec``: the committed ncu
    record of the same kernel (DRAM bytes per row per sweep), or None."""
    vb = 8 if prec == "fp64" else 4
    bytes_iter = passes_per_iter(l, "plcg") * vb * n
    bytes_launch = iters * bytes_iter + 3 * 8 * n * 2   # + 2 FP64 residual sweeps
    achieved_gbs = bytes_launch / seconds / 1e9
    achieved_dp_tf = iters * dp_flops_per_point(l) * n / seconds / 1e12
    # measured DRAM traffic per launch: bytes per row per sweep of an ncu
    # capture (smaller grid, same kernel) x rows x sweeps of this solve
    traffic = None if rec is None else round(rec["dram_bytes_per_point_iter"] * n * (iters + 2))
    hbm_frac = achieved_gbs / hbm_peak
    dp_frac = achieved_dp_tf / dp_peak_tf
    hbm_part = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(hbm_frac, 4), "peak_source": hbm_src,
                "bytes_per_iter": bytes_iter}
    alu_part = {"bound": "alu", "achieved": round(achieved_dp_tf, 4), "peak": dp_peak_tf,
                "unit": "TFLOP/s", "frac": round(dp_frac, 4), "peak_source": dp_src,
                "flops_per_row_iter": dp_flops_per_point(l),
                "ncu_fp64_pipe_pct": None if rec is None else rec.get("fp64_pipe_pct")}
    if (prec, l) == ("fp64", 1) and n >= (1 << 19) and nx % 2 == 0:
        # the kernel of this solve (scaled bases, two rows per thread) executes
        # 16 of the paper's 24 flops per row on the FP64 pipe (the neighbour
        # sum runs on the integer units): the FP64 roofline counts those, the
        # paper's count stays beside them
        pipe = DP_PIPE_FLOPS_L1 / dp_flops_per_point(1)
        dp_frac *= pipe
        alu_part.update({"achieved": round(achieved_dp_tf * pipe, 4), "frac": round(dp_frac, 4),
                         "flops_per_row_iter": DP_PIPE_FLOPS_L1,
                         "flops_counted": "FP64-pipe flops: 8 FMA per row (K4's two recurrences, K6, "
                                          "the two K5 dots); the six-neighbour sum runs on the integer units",
                         "paper_flops_per_row_iter": dp_flops_per_point(1),
                         "paper_flops_tflops": round(achieved_dp_tf, 4)})
    if prec != "fp64":   # FP32 sweeps: no FP64 roof (FP64 only in dots and scalars)
        return dict(hbm_part, traffic=traffic)
    if dp_frac >= hbm_frac:
        return dict(alu_part, traffic=traffic, hbm=hbm_part)
    return dict(hbm_part, traffic=traffic, alu=alu_part)


# ---------------------------------------------------------------- oracle errors
class OracleErrors:
    """FP64 oracle solves run on the host cores while the GPU legs run (a
    process pool created with the spawn method before the first GPU call);
    ``error(key, x)`` is ||x - x_oracle|| / ||x_oracle|| and the oracle's
    iteration count, once the job has finished."""

    def __init__(self, enabled: bool):
        self.pool = None
        self.futures = {}
        if enabled:
            from oracle import jobs
            self.pool = jobs.pool()
            self.run = jobs.run

    def submit(self, key, **job):
        if self.pool is not None and key not in self.futures:
            self.futures[key] = self.pool.submit(self.run, dict(job, key=key))

    def result(self, key):
        f = self.futures.get(key)
        if f is None:
            return None
        _, x, iters, restarts, secs = f.result()
        return x, iters, restarts, secs

    def annotate(self, entry: dict, key: str, x_gpu) -> dict:
        """Adds err_vs_oracle, the oracle's iterations and restarts to entry."""
        r = self.result(key)
        if r is None:
            entry["err_vs_oracle"] = None
            return entry
        x, iters, restarts, _ = r
        entry["err_vs_oracle"] = float(np.linalg.norm(x_gpu - x) / max(np.linalg.norm(x), 1e-300))
        entry["oracle_iters"] = iters
        entry["oracle_restarts"] = restarts
        return entry

    def close(self):
        if self.pool is not None:
            self.pool.shutdown(wait=False, cancel_futures=True)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1905_06850_gb300 import plcg
    from paper_1905_06850_gb300 import workloads as W

    rank, world, local = dist_env()
    # FP64 oracle solves for the error of every FP32 result: rank 0, started
    # before the first GPU call
    orc = OracleErrors(rank == 0 and not args.quick and not args.no_oracle_errors)
    for l in (1, 2):
        orc.submit(f"3d.l{l}", workload={"kind": "3d", "nx": args.nx}, method="plcg", l=l,
                   interval=(0.0, 12.0), rtol=RTOL)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    plcg.load()
    dev = torch.device("cuda", local)

    cfg = W.config_3d(nx=args.nx, seed=2)
    op, b_np = cfg["op"], cfg["b"]
    n = W.op_size(op)
    interval = cfg["interval"]
    b = torch.tensor(b_np, device=dev)
    A = plcg.Matrix(op)
    stream = torch.cuda.current_stream()

    def solve_once(x, **kw):
        if args.maxit:
            kw.setdefault("maxit", args.maxit)
        return A.solve(b, x, l=kw.pop("l", args.l), interval=interval, rtol=RTOL,
                       prec=kw.pop("prec", args.prec), check=not args.maxit, **kw)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also builds the workspace)
    xs = [torch.zeros(n, dtype=torch.float64, device=dev) for _ in range(args.warmup + args.steps)]
    for w in range(args.warmup):
        solve_once(xs[w])
    results = []
    barrier()
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for s in range(args.steps):
            results.append(solve_once(xs[args.warmup + s]))
        ev1.record(stream)
        barrier()
    iters = [r.iters for r in results]
    # max over ranks of the device time, iterations summed over ranks
    t_total, total_iters = aggregate_over_ranks(ev0.elapsed_time(ev1) * 1e-3, sum(iters), world, dev)
    if not args.maxit:
        assert all(r.ok for r in results), [r.status for r in results]
    value = total_iters / t_total
    ms_per_step = t_total / args.steps * 1e3
    kern_s = [r.seconds for r in results]
    # true residual of the last solve, checked on the host (independent stencil apply)
    x_last = xs[-1].cpu().numpy()
    host_relres = float(np.linalg.norm(b_np - W.rhs(op, x_last)) / np.linalg.norm(b_np))

    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    hbm_src = "measured" if peaks.get("hbm_gbs") else "fallback"
    # FP64 peak: measured on this GPU (independent FMA chains on every
    # resident thread, plcg_measure_fp64_fma_rate); nominal 1.25 if that fails
    try:
        dp_peak_tf, dp_src = round(plcg.measure_fp64_fma_rate() / 1e12, 4), "measured (plcg_measure_fp64_fma_rate)"
    except Exception as exc:   # noqa: BLE001
        dp_peak_tf, dp_src = 1.25, f"nominal (measurement failed: {exc})"
    rec = profiled_record("plcg_3d_fp64_l1.json") if (args.prec, args.l) == ("fp64", 1) else None
    roofline = stencil_roofline(n=n, nx=args.nx, l=args.l, prec=args.prec, iters=statistics.mean(iters),
                                seconds=statistics.mean(kern_s), hbm_peak=hbm_peak, hbm_src=hbm_src,
                                dp_peak_tf=dp_peak_tf, dp_src=dp_src, rec=rec)
    achieved_gbs = roofline["hbm"]["achieved"] if "hbm" in roofline else roofline["achieved"]

    extra = {}
    if rank == 0 and not args.quick:
        # classic CG on the same system and GPU
        xc = torch.zeros(n, dtype=torch.float64, device=dev)
        A.solve(b, xc, method="cg", rtol=RTOL)
        xc.zero_()
        rc = A.solve(b, xc, method="cg", rtol=RTOL)
        extra["classic_cg"] = {"iters": rc.iters, "time_to_rtol_s": round(rc.seconds, 5),
                               "iters_per_s": round(rc.iters / rc.seconds, 1),
                               "hbm_gbs": round(rc.iters * 10 * 8 * n / rc.seconds / 1e9, 1)}
        # l sweep (FP64)
        sweep = {}
        for l in (2, 3, 4, 5):
            xl = torch.zeros(n, dtype=torch.float64, device=dev)
            r = A.solve(b, xl, l=l, interval=interval, rtol=RTOL)
            sweep[f"l{l}"] = {"iters": r.iters, "time_to_rtol_s": round(r.seconds, 5),
                              "iters_per_s": round(r.iters / r.seconds, 1),
                              "hbm_gbs": round(r.iters * passes_per_iter(l, "plcg") * 8 * n
                                               / r.seconds / 1e9, 1)}
        extra["plcg_l_sweep_fp64"] = sweep
        # FP32 vectors with FP64 dots / scalars / refinement
        mp = {}
        for l in (1, 2):
            xf = torch.zeros(n, dtype=torch.float64, device=dev)
            A.solve(b, xf, l=l, interval=interval, rtol=RTOL, prec="fp32")
            xf.zero_()
            r = A.solve(b, xf, l=l, interval=interval, rtol=RTOL, prec="fp32")
            xf_np = xf.cpu().numpy()
            err = float(np.linalg.norm(b_np - W.rhs(op, xf_np)) / np.linalg.norm(b_np))
            byt = r.iters * passes_per_iter(l, "plcg") * 4 * n
            rec32 = profiled_record("plcg_3d_fp32_l1.json") if l == 1 else None
            mp[f"l{l}"] = {"iters": r.iters, "refinements": r.refinements,
                           "traffic": None if rec32 is None else
                           round(rec32["dram_bytes_per_point_iter"] * n * (r.iters + 2 * (r.refinements + 1))),
                           "time_to_rtol_s": round(r.seconds, 5),
                           "iters_per_s": round(r.iters / r.seconds, 1),
                           "hbm_gbs": round(byt / r.seconds / 1e9, 1),
                           "hbm_frac": round(byt / r.seconds / 1e9 / hbm_peak, 4),
                           "true_relres": err}
            mp[f"l{l}"]["_x"] = xf_np
        xf = torch.zeros(n, dtype=torch.float64, device=dev)
        r = A.solve(b, xf, method="cg", rtol=RTOL, prec="fp32")
        mp["classic_cg"] = {"iters": r.iters, "time_to_rtol_s": round(r.seconds, 5),
                            "iters_per_s": round(r.iters / r.seconds, 1)}
        extra["fp32_fp64corr"] = mp

    if rank == 0 and not args.quick and not args.no_configs:
        extra["other_configs"] = other_configs(plcg, W, dev, hbm_peak, orc)

    # end to end through the host-pointer entry point (pinned host buffers)
    e2e = None
    if not args.quick:
        bh = torch.tensor(b_np).pin_memory()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory()
        A.solve_host(bh.numpy(), xh.numpy(), l=L_HEAD, interval=interval, rtol=RTOL)
        barrier()
        t0 = time.perf_counter()
        k_e2e = 0
        for _ in range(max(1, args.steps // 2)):
            xh.zero_()
            r = A.solve_host(bh.numpy(), xh.numpy(), l=L_HEAD, interval=interval, rtol=RTOL)
            k_e2e += r.iters
        t_e2e, k_all = aggregate_over_ranks(time.perf_counter() - t0, k_e2e, world, dev)
        e2e = {"value": round(k_all / t_e2e, 1), "unit": UNIT,
               "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n,
               "steps": max(1, args.steps // 2)}

    if world > 1:
        dist.barrier()
    if rank != 0:
        return
    if "fp32_fp64corr" in extra:
        for l in (1, 2):
            ent = extra["fp32_fp64corr"][f"l{l}"]
            orc.annotate(ent, f"3d.l{l}", ent.pop("_x"))
    finish_oracle_errors(extra.get("other_configs"), orc)
    orc.close()
    cpu = cpu_baseline(op, b_np, interval) if not args.quick else None
    cpu_cfgs = cpu_baseline_configs() if not args.quick and not args.no_configs else None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded x* ~ N(0,1), b = A x*)",
        "config": {"workload": f"3D 7-point Laplacian {args.nx}^3 (n={n}), FP64, p(1)-CG, "
                               f"Chebyshev shifts on [0, 12], rtol {RTOL}, x0 = 0",
                   "l": L_HEAD, "n": n, "iters_per_solve": iters[0],
                   "time_to_rtol_s": round(statistics.median(kern_s), 5),
                   "l2": "inputs larger than L2 (each vector 134 MB > 126 MB L2); no flush",
                   "host_check_true_relres": host_relres},
        "hbm_gbs": round(achieved_gbs, 1),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_baseline_configs": cpu_cfgs,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        **extra,
    }
    print(json.dumps(line), flush=True)


def other_configs(plcg, W, dev, hbm_peak, orc):
    """Time-to-rtol on the other workloads: the 2D 100^2 Laplacian (FP64,
    latency-bound), the diagonal toy of Sec. 4 (100^2 and 2000^2), the 27-point heterogeneous CSR on 128^3 (FP32 with FP64
    correction; unpreconditioned and with Jacobi) and the batch of 4096 shifted 2D Poisson systems (FP32 with
    FP64 correction, one persistent launch), each against classic CG."""
    import torch
    out = {}
    # ---- 2D 5-point 100^2, FP64, rtol 1e-6 (the workload's) and 1e-8 (the
    # metric's); small systems run on one thread-block cluster where that is
    # faster ("cluster": its CTAs, 0 = the grid path)
    c = W.config_2d()
    A = plcg.Matrix(c["op"])
    b = torch.tensor(c["b"], device=dev)
    for rtol in (c["rtol"], 1e-8):
        d = {}
        for name, kw in (("plcg_l1", {"l": 1}), ("plcg_l2", {"l": 2}), ("plcg_l3", {"l": 3}),
                         ("classic_cg", {"method": "cg"})):
            ts = []
            for _ in range(5):
                x = torch.zeros_like(b)
                r = A.solve(b, x, interval=c["interval"], rtol=rtol, **kw)
                ts.append(r.seconds)
            d[name] = {"iters": r.iters, "time_to_rtol_us": round(min(ts) * 1e6, 1),
                       "us_per_iter": round(min(ts) / r.iters * 1e6, 2),
                       "cluster": plcg.last_launch()["cluster"]}
        out[f"2d_100_fp64_rtol{rtol:g}"] = d
    A.close()
    # ---- the paper's communication-bound toy: diagonal operator with the 2D
    # Laplacian's eigenvalues (Sec. 4), 100^2 (barrier-latency bound) and the
    # paper's 2000^2 = 4M unknowns, FP64, rtol 1e-6
    for N in (100, 2000):
        e = W.e3_diagonal(N)
        A = plcg.Matrix(e["op"])
        b = torch.tensor(e["b"], device=dev)
        d = {"n": N * N}
        for name, kw in (("plcg_l1", {"l": 1}), ("plcg_l2", {"l": 2}), ("plcg_l3", {"l": 3}),
                         ("classic_cg", {"method": "cg"})):
            ts = []
            for _ in range(3 if N == 100 else 2):
                x = torch.zeros_like(b)
                r = A.solve(b, x, interval=e["interval"], rtol=e["rtol"], **kw)
                ts.append(r.seconds)
            d[name] = {"iters": r.iters, "time_to_rtol_us": round(min(ts) * 1e6, 1),
                       "us_per_iter": round(min(ts) / r.iters * 1e6, 2),
                       "cluster": plcg.last_launch()["cluster"]}
        A.close()
        out[f"e3_diag_{N}_fp64_rtol1e-6"] = d
    # ---- 27-point heterogeneous CSR 128^3 (M = I as specified, and Jacobi):
    # FP32 values and vectors with FP64 dots/scalars/refinement ("fp32"), and
    # FP32 values under FP64 vectors ("fp32_matrix"); error of every result
    # against the FP64 oracle on the same FP32-rounded operator
    c = W.config_hetero27(nx=128)
    op = c["op"]
    n, nnz = op["n"], int(op["rowptr"][-1])
    A = plcg.Matrix(op, prec="fp32")
    b = torch.tensor(c["b"], device=dev)
    jac = {"precond": "jacobi"}
    # Chebyshev shift intervals [0, 1.02 lambda_max] from plcg_estimate_interval
    # (30 CG steps on the GPU, once per operator; Sec. 2.2), for A and for
    # diag(A)^{-1} A (Jacobi)
    est = {}
    for key, pk in (("none", None), ("jacobi", "jacobi")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lo, hi = A.estimate_interval(steps=30, prec="fp32", precond=pk)
        torch.cuda.synchronize()
        est[key] = {"interval": [0.0, round(1.02 * hi, 6)], "ritz": [lo, hi],
                    "seconds": round(time.perf_counter() - t0, 5)}
    cases = (("plcg_l1", {"l": 1}), ("plcg_l2", {"l": 2}), ("plcg_l3", {"l": 3}),
             ("classic_cg", {"method": "cg"}),
             ("jacobi_plcg_l1", {"l": 1, **jac}), ("jacobi_plcg_l2", {"l": 2, **jac}),
             ("jacobi_plcg_l3", {"l": 3, **jac}), ("jacobi_classic_cg", {"method": "cg", **jac}))
    # square-root breakdowns (Sec. 2.2) are frequent on this operator without a
    # preconditioner -- the FP64 oracle itself restarts 50-100 times at l = 2, 3 --
    # so every solve gets a restart budget that covers them
    restarts = 1000
    for name, kw in cases:
        iv = est["jacobi" if "precond" in kw else "none"]["interval"]
        orc.submit(f"h27.{name}", workload={"kind": "h27", "nx": 128}, method=kw.get("method", "plcg"),
                   l=kw.get("l", 1), interval=tuple(iv), rtol=1e-8, precond=kw.get("precond"),
                   max_restarts=restarts)
    for prec in ("fp32", "fp32_matrix"):
        d = {"n": n, "nnz": nnz, "prec": prec, "max_restarts": restarts}
        if prec == "fp32":
            d["interval_estimates"] = est
        vb = 4 if prec == "fp32" else 8   # vector element bytes
        for name, kw in cases:
            interval = est["jacobi" if "precond" in kw else "none"]["interval"]
            ts = []
            for _ in range(2):
                x = torch.zeros_like(b)
                r = A.solve(b, x, interval=interval, rtol=1e-8, prec=prec, max_restarts=restarts,
                            check=False, **kw)
                ts.append(r.seconds)
            ll = kw.get("l", 1)
            vec_passes = 10 if "method" in kw else 3 * (ll + 1) + 4
            jac_bytes = (vb + 4) if "precond" in kw else 0   # 1/a_gg (vector type) and a_gg (FP32)
            byt = r.iters * (vec_passes * vb * n + 8 * nnz + 8 * n + jac_bytes * n)
            d[name] = {"status": r.status, "iters": r.iters, "restarts": r.restarts,
                       "refinements": r.refinements, "time_to_rtol_s": round(min(ts), 5),
                       "hbm_gbs": round(byt / min(ts) / 1e9, 1),
                       "hbm_frac": round(byt / min(ts) / 1e9 / hbm_peak, 4),
                       "_x": x.cpu().numpy(), "_okey": f"h27.{name}"}
        out["h27_csr_128_fp32" if prec == "fp32" else "h27_csr_128_fp32_matrix"] = d
    A.close()
    # ---- the same operator in the structured 27-point layout (diagonal + 13
    # forward weights per cell, no column indices), FP32, Jacobi
    c27 = W.config_hetero27_var27(nx=128)
    A = plcg.Matrix(c27["op"], prec="fp32")
    interval = est["jacobi"]["interval"]   # the same matrix as the CSR form
    d = {"n": n, "bytes_per_row_operator": 14 * 4, "interval": interval}
    for name, kw in (("jacobi_plcg_l1", {"l": 1}), ("jacobi_plcg_l2", {"l": 2}),
                     ("jacobi_plcg_l3", {"l": 3}), ("jacobi_classic_cg", {"method": "cg"})):
        ts = []
        for _ in range(2):
            x = torch.zeros_like(b)
            r = A.solve(b, x, interval=interval, rtol=1e-8, prec="fp32", max_restarts=64,
                        precond="jacobi", check=False, **kw)
            ts.append(r.seconds)
        ll = kw.get("l", 1)
        vec_passes = (10 if "method" in kw else 3 * (ll + 1) + 4) + 1   # + 1/a_rr
        byt = r.iters * (vec_passes * 4 * n + 14 * 4 * n)
        d[name] = {"status": r.status, "iters": r.iters, "restarts": r.restarts,
                   "time_to_rtol_s": round(min(ts), 5), "hbm_gbs": round(byt / min(ts) / 1e9, 1),
                   "hbm_frac": round(byt / min(ts) / 1e9 / hbm_peak, 4),
                   "_x": x.cpu().numpy(), "_okey": f"h27.{name}"}   # the same matrix as the CSR form
    A.close()
    out["h27_var27_128_fp32"] = d
    # ---- batched: 4096 shifted 2D Poisson systems, FP32 with FP64 correction
    systems = W.batched_systems(4096)
    mats = [plcg.Matrix(s_["op"]) for s_ in systems]
    bs = [torch.tensor(s_["b"], device=dev) for s_ in systems]
    lo = [s_["interval"][0] for s_ in systems]
    hi = [s_["interval"][1] for s_ in systems]
    unknowns = sum(W.op_size(s_["op"]) for s_ in systems)
    d = {"systems": len(systems), "unknowns": unknowns}
    from paper_1905_06850_gb300 import autotune
    sample = list(range(0, len(systems), len(systems) // 16))[:16]   # systems checked against the oracle
    for name, kw in (("plcg_l1", {"l": 1}), ("plcg_l2", {"l": 2}), ("plcg_l3", {"l": 3}),
                     ("classic_cg", {"method": "cg"})):
        for i in sample:
            orc.submit(f"batched.{name}.{i}", workload={"kind": "batched", "count": len(systems), "index": i},
                       method=kw.get("method", "plcg"), l=kw.get("l", 1), interval=systems[i]["interval"],
                       rtol=1e-8)
        sched, shape, _ = autotune.tune_batched(mats, bs, lo, hi, prec="fp32", rtol=1e-8, **kw)
        best = None
        for _ in range(2):
            xs = [torch.zeros_like(b_) for b_ in bs]
            st, res = plcg.solve_batched(mats, bs, xs, lmins=lo, lmaxs=hi, prec="fp32", rtol=1e-8,
                                         check=False, **kw)
            t = res[0].seconds
            best = t if best is None else min(best, t)
        its = np.array([r.iters for r in res])
        lat = np.array([r.latency for r in res]) * 1e3   # launch start -> each system's result
        ok = sum(r.status == 0 for r in res)
        ll = kw.get("l", 1)
        vec_passes = 10 if "method" in kw else 3 * (ll + 1) + 4
        byt = sum(W.op_size(s_["op"]) * r.iters for s_, r in zip(systems, res)) * vec_passes * 4
        d[name] = {"status": st, "converged": ok, "batch_time_s": round(best, 5),
                   "schedule": {"gang_size": sched[0], "large_work_factor": sched[1],
                                "max_gang_fraction": sched[2]},
                   "launch_shape": {"ctas_per_sm": shape[0], "rows_per_thread": shape[1],
                                    "vector_width": shape[2]},
                   "system_completion_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                                            "p99": round(float(np.percentile(lat, 99)), 3),
                                            "max": round(float(lat.max()), 3)},
                   "solves_per_s": round(len(systems) / best, 1),
                   "iters_mean": round(float(its.mean()), 1), "iters_max": int(its.max()),
                   "hbm_gbs": round(byt / best / 1e9, 1),
                   "hbm_frac": round(byt / best / 1e9 / hbm_peak, 4),
                   "_xs": {i: xs[i].cpu().numpy() for i in sample}, "_okey": f"batched.{name}"}
    autotune.set_schedule(0)
    autotune.set_launch(0, 0)
    for m in mats:
        m.close()
    out["batched_4096_2d_fp32"] = d
    out["serving_mixed_fp32"] = serving(plcg, W, dev)
    return out


def serving(plcg, W, dev):
    """Open-loop serving run: Poisson arrivals (2000/s) over a 0.25 s window
    of requests with n log-uniform in [1e3, 4e6] and operator type uniform
    over {2D stencil, 3D stencil, random SPD CSR}; FP32 with FP64 correction,
    p(1)-CG, rtol 1e-8.  The offered load exceeds one GPU (the window then
    drains); a second run at 70% of the measured completion rate follows.
    CSR sizes are rounded to 12 log-spaced buckets whose matrices are built
    once (random CSR generation for every request would take minutes)."""
    import torch
    buckets = np.exp(np.linspace(np.log(1e3), np.log(4e6), 12))
    mats = {}

    def realise(req):
        n = req["n_target"]
        if req["type"] == "2d":
            s_ = max(4, int(round(n ** 0.5)))
            key = ("2d", s_)
            if key not in mats:
                mats[key] = plcg.Matrix(W.fp32_rounded(W.stencil2d(s_, s_)), prec="fp32")
            iv = (0.0, 8.0)
        elif req["type"] == "3d":
            s_ = max(4, int(round(n ** (1 / 3))))
            key = ("3d", s_)
            if key not in mats:
                mats[key] = plcg.Matrix(W.fp32_rounded(W.stencil3d(s_, s_, s_)), prec="fp32")
            iv = (0.0, 12.0)
        else:
            nb = int(round(buckets[int(np.argmin(np.abs(np.log(buckets) - np.log(n))))]))
            key = ("csr", nb)
            if key not in mats:
                op = W.random_spd_csr(nb, seed=1000 + nb)
                mats[key] = (plcg.Matrix(op, prec="fp32"), W.shift_interval(op))
            m, iv = mats[key]
            return m, iv
        return mats[key], iv

    def run(reqs):
        items = []
        for q in reqs:
            m, iv = realise(q)
            g = torch.Generator(device=dev)
            g.manual_seed(q["seed"])
            b = torch.randn(m.n, generator=g, device=dev, dtype=torch.float64)
            items.append((q["t"], m, iv, b, torch.zeros_like(b)))
        torch.cuda.synchronize()
        S = plcg.Server()
        t0 = time.perf_counter()
        pending, results, i = {}, [], 0
        t_last = t0
        while i < len(items) or pending:
            now = time.perf_counter() - t0
            while i < len(items) and items[i][0] <= now:
                _, m, iv, b, x = items[i]
                pending[S.submit(m, b, x, l=1, interval=iv, rtol=1e-8, prec="fp32",
                                 max_restarts=64)] = i
                i += 1
            for tk in list(pending):
                r = S.poll(tk)
                if r is not None:
                    results.append((pending[tk], r))
                    del pending[tk]
                    t_last = time.perf_counter()
            if i < len(items) and not pending:
                time.sleep(max(0.0, items[i][0] - (time.perf_counter() - t0)))
        S.close()
        span = t_last - t0
        lat = np.array([r.latency for _, r in results]) * 1e3
        ok = sum(r.status == 0 for _, r in results)
        # latency by size class (each request's grid is capped at half the
        # GPU's resident CTAs, so that a request's bits do not depend on the mix)
        classes = {}
        for lo_, hi_, name in ((0, 3e4, "n<3e4"), (3e4, 3e5, "3e4<=n<3e5"), (3e5, 1e12, "n>=3e5")):
            rs = [r for i_, r in results if lo_ <= items[i_][1].n < hi_]
            sel = np.array([r.latency for r in rs]) * 1e3
            if sel.size:
                # run: the request's own kernel time on the device; the rest of
                # its latency is the wait for admission
                run_ms = np.array([r.seconds for r in rs]) * 1e3
                classes[name] = {"requests": int(sel.size), "p50_ms": round(float(np.percentile(sel, 50)), 2),
                                 "p99_ms": round(float(np.percentile(sel, 99)), 2),
                                 "run_p50_ms": round(float(np.percentile(run_ms, 50)), 2),
                                 "wait_p50_ms": round(float(np.percentile(sel - run_ms, 50)), 2)}
        return {"requests": len(items), "converged": ok, "window_s": round(items[-1][0], 3),
                "makespan_s": round(span, 3), "solves_per_s": round(len(items) / span, 1),
                "p50_latency_ms": round(float(np.percentile(lat, 50)), 2),
                "p99_latency_ms": round(float(np.percentile(lat, 99)), 2),
                "latency_by_size": classes,
                "backlog_drain_s": round(span - items[-1][0], 3)}

    reqs = W.serving_stream(duration_s=0.25, rate=2000.0, seed=5)
    full = run(reqs)
    rate2 = 0.7 * full["solves_per_s"]
    reqs2 = W.serving_stream(duration_s=3.0, rate=rate2, seed=6, max_requests=400)
    light = run(reqs2)
    light["rate_per_s"] = round(rate2, 1)
    for m in mats.values():
        (m[0] if isinstance(m, tuple) else m).close()
    return {"offered_2000_per_s": full, "at_70pct_capacity": light,
            "note": "FP32 vectors with FP64 correction, p(1)-CG, rtol 1e-8; CSR sizes bucketed"}


def finish_oracle_errors(configs, orc):
    """Replaces the kept GPU solutions of the other workloads by their error
    against the FP64 oracle (err_vs_oracle, with the oracle's iterations and
    restarts; batched: the largest error over the sampled systems)."""
    if not configs:
        return
    for d in configs.values():
        if not isinstance(d, dict):
            continue
        for ent in d.values():
            if not isinstance(ent, dict):
                continue
            if "_x" in ent:
                orc.annotate(ent, ent.pop("_okey"), ent.pop("_x"))
                if ent.get("oracle_iters"):
                    ent["iters_vs_oracle"] = round(ent["iters"] / ent["oracle_iters"], 4)
            elif "_xs" in ent:
                key, errs = ent.pop("_okey"), []
                for i, x in ent.pop("_xs").items():
                    tmp = orc.annotate({}, f"{key}.{i}", x)
                    if tmp.get("err_vs_oracle") is not None:
                        errs.append(tmp["err_vs_oracle"])
                ent["err_vs_oracle"] = max(errs) if errs else None
                ent["err_vs_oracle_systems"] = len(errs)


# ---------------------------------------------------------------- CPU oracle
def cpu_baseline(op, b, interval, iters=12):
    """The FP64 oracle (serial C, as it stands) on a bounded sample of the same
    workload: `iters` iterations of p(1)-CG on the full 256^3 system."""
    from oracle import oracle as O
    sig = O.chebyshev_shifts(L_HEAD, *interval)
    t0 = time.perf_counter()
    r = O.plcg(op, b, l=L_HEAD, sigma=sig, rtol=RTOL, maxit=iters, dots_2l1=False)
    dt = time.perf_counter() - t0
    return {"value": round(r.iters / dt, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{r.iters} iterations of p(1)-CG on the full {op['nx']}^3 system "
                      f"(serial C oracle, plus its 2 residual evaluations), {dt:.1f} s"}


def cpu_baseline_configs():
    """The serial FP64 oracle (as it stands) on the other workloads, each on a
    bounded sample: the whole 2D 100^2 solve (p(1)-CG and CG, rtol 1e-6), 10
    iterations of p(2)-CG on the 27-point heterogeneous CSR 128^3, and 16
    systems of the 4096-system batch (p(1)-CG, rtol 1e-8) scaled to solves/s
    of the batch's size mix; then the same oracle on all host cores at once
    (cpu_all_cores)."""
    from oracle import oracle as O
    from paper_1905_06850_gb300 import workloads as W
    out = {"host_cores": os.cpu_count(), "cores_used": 1, "kind": "oracle"}
    try:
        with open("/proc/cpuinfo") as f:
            models = [ln.split(":", 1)[1].strip() for ln in f if ln.lower().startswith(("model name", "cpu part"))]
        out["cpu"] = models[0] if models else None
    except OSError:
        out["cpu"] = None
    c = W.config_2d()
    d = {}
    for name, kw in (("plcg_l1", {"l": 1, "sigma": O.chebyshev_shifts(1, *c["interval"])}), ("classic_cg", {})):
        t0 = time.perf_counter()
        r = O.plcg(c["op"], c["b"], rtol=c["rtol"], dots_2l1=False, **kw) if kw else O.cg(c["op"], c["b"], rtol=c["rtol"])
        dt = time.perf_counter() - t0
        d[name] = {"iters": r.iters, "time_to_rtol_s": round(dt, 5), "iters_per_s": round(r.iters / dt, 1)}
    out["2d_100_fp64_rtol1e-6"] = d
    c = W.config_hetero27(nx=128)
    sig = O.chebyshev_shifts(2, *c["interval"])
    t0 = time.perf_counter()
    r = O.plcg(c["op"], c["b"], l=2, sigma=sig, rtol=1e-8, maxit=10, dots_2l1=False)
    dt = time.perf_counter() - t0
    out["h27_csr_128"] = {"iters_per_s": round(r.iters / dt, 2), "sample": "10 iterations of p(2)-CG (FP64)",
                          "seconds": round(dt, 2)}
    systems = W.batched_systems(4096)
    pick = list(range(0, 4096, 256))
    t0 = time.perf_counter()
    unknowns = 0
    for i in pick:
        s_ = systems[i]
        O.plcg(s_["op"], s_["b"], l=1, sigma=O.chebyshev_shifts(1, *s_["interval"]), rtol=1e-8, dots_2l1=False)
        unknowns += W.op_size(s_["op"])
    dt = time.perf_counter() - t0
    total = sum(W.op_size(s_["op"]) for s_ in systems)
    out["batched_4096_2d"] = {"sample": f"{len(pick)} systems (every 256th), p(1)-CG, rtol 1e-8",
                              "seconds": round(dt, 2),
                              "solves_per_s_scaled": round(len(systems) / (dt * total / unknowns), 2)}
    out["all_cores"] = cpu_all_cores(systems)
    return out


def cpu_all_cores(systems):
    """The same serial oracle on every host core at once: one spawn worker
    process per core (started and loaded before the clock starts), each
    solving whole systems -- 256 systems of the batch (every 16th, p(1)-CG,
    rtol 1e-8, scaled to solves/s of the batch's size mix) and 2D 100^2
    p(1)-CG solves (rtol 1e-6, eight per core).  A throughput figure for
    independent solves, not a faster single solve."""
    from oracle import jobs
    from paper_1905_06850_gb300 import workloads as W
    cores = os.cpu_count() or 1
    out = {"cores": cores, "kind": "oracle, one process per core"}
    with jobs.pool(max_workers=cores) as ex:
        list(ex.map(jobs.warm, range(cores)))
        pick = list(range(0, len(systems), 16))
        t0 = time.perf_counter()
        futs = [ex.submit(jobs.run, {"key": i, "workload": {"kind": "batched", "index": i, "count": len(systems)},
                                     "method": "plcg", "l": 1, "interval": systems[i]["interval"], "rtol": 1e-8})
                for i in pick]
        for f in futs:
            f.result()
        dt = time.perf_counter() - t0
        unknowns = sum(W.op_size(systems[i]["op"]) for i in pick)
        total = sum(W.op_size(s_["op"]) for s_ in systems)
        out["batched_4096_2d"] = {"sample": f"{len(pick)} systems (every 16th), p(1)-CG, rtol 1e-8",
                                  "seconds": round(dt, 2),
                                  "solves_per_s_scaled": round(len(systems) / (dt * total / unknowns), 2)}
        c = W.config_2d()
        t0 = time.perf_counter()
        futs = [ex.submit(jobs.run, {"key": k, "workload": {"kind": "2d", "nx": 100}, "method": "plcg", "l": 1,
                                     "interval": c["interval"], "rtol": c["rtol"]}) for k in range(8 * cores)]
        for f in futs:
            f.result()
        dt = time.perf_counter() - t0
        out["2d_100_fp64_rtol1e-6"] = {"solves": 8 * cores, "seconds": round(dt, 3),
                                       "solves_per_s": round(8 * cores / dt, 1)}
    return out


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host's cores, same
    metric and workload, each step a bounded sample (a few iterations)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1905_06850_gb300 import workloads as W
    cfg = W.config_3d(nx=args.nx, seed=2)
    op, b = cfg["op"], cfg["b"]
    sig = O.chebyshev_shifts(L_HEAD, *cfg["interval"])
    per_step = 4
    for _ in range(args.warmup):
        O.plcg(op, b, l=L_HEAD, sigma=sig, rtol=RTOL, maxit=1, dots_2l1=False)
    t0 = time.perf_counter()
    k = 0
    for _ in range(args.steps):
        k += O.plcg(op, b, l=L_HEAD, sigma=sig, rtol=RTOL, maxit=per_step, dots_2l1=False).iters
    dt = time.perf_counter() - t0
    value = k / dt
    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded x* ~ N(0,1), b = A x*)", "impl": "reference",
            "config": {"workload": f"3D 7-point Laplacian {args.nx}^3, FP64, p(1)-CG, rtol {RTOL}",
                       "sample_per_step": f"{per_step} iterations (+2 residual evaluations)"},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} iterations per step of the full system"},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--quick", action="store_true", help="headline only (no sweeps, e2e, CPU)")
    ap.add_argument("--maxit", type=int, default=0, help="cap iterations (profiling runs)")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--l", type=int, default=L_HEAD)
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-oracle-errors", action="store_true",
                    help="skip the FP64 oracle solves that state each FP32 result's error")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
