"""Autotuner for batched solves: picks the gang schedule of plcg_solve_batched.

The batched launch solves large systems with gangs of thread blocks and the
rest with one block each (see ``plcg_set_batched_schedule`` in
include/plcg.h).  Which split is fastest depends on the batch's size/work
distribution, so ``tune_batched`` times a small set of candidate schedules on
the batch itself, installs the fastest, and returns all timings.  Argument
marshalling and timing only; the solves run in the library's kernels.
"""
from __future__ import annotations

from . import plcg

CANDIDATES = [(1, 1.0, 0.0), (4, 1.0, 0.5), (8, 1.0, 0.5), (16, 1.0, 0.5), (8, 0.5, 0.5),
              (8, 2.0, 0.5), (8, 0.25, 0.75), (16, 0.5, 0.75)]


def set_schedule(gang_size: int, large_work_factor: float = 1.0, max_gang_fraction: float = 0.5):
    plcg._check(plcg.load().plcg_set_batched_schedule(int(gang_size), float(large_work_factor),
                                                      float(max_gang_fraction)))


def tune_batched(mats, bs, lmins=None, lmaxs=None, candidates=CANDIDATES, repeats=1, **kw):
    """Time each candidate (gang_size, large_work_factor, max_gang_fraction) on
    this batch (x0 = 0 each time), install the fastest and return
    (best, {candidate: seconds})."""
    import torch
    times = {}
    for cand in candidates:
        set_schedule(*cand)
        best = None
        for _ in range(repeats):
            xs = [torch.zeros_like(b) for b in bs]
            st, res = plcg.solve_batched(mats, bs, xs, lmins=lmins, lmaxs=lmaxs, check=False, **kw)
            if st != plcg.PLCG_OK:
                best = float("inf")
                break
            t = res[0].seconds
            best = t if best is None else min(best, t)
        times[cand] = best
    choice = min(times, key=times.get)
    set_schedule(*choice)
    return choice, times
