"""Autotuner for batched solves: picks the launch shape and the gang schedule
of plcg_solve_batched.

The batched launch solves large systems with gangs of thread blocks and the
rest with one block each (``plcg_set_batched_schedule`` in include/plcg.h),
with a kernel variant whose registers are sized for a number of blocks per SM
and whose one-block path gives each thread a number of row groups, or pairs
of adjacent rows as 2-wide vectors (``plcg_set_batched_launch``; FP32
solves).  Which choice is fastest depends
on the batch's size/work distribution and the method, so ``tune_batched``
times candidates on the batch itself -- first the launch shapes under the
default schedule, then the schedules under the best shape -- installs the
fastest pair and returns every timing.  Argument marshalling and timing
only; the solves run in the library's kernels.
"""
from __future__ import annotations

from . import plcg

# (gang_size, large_work_factor, max_gang_fraction)
CANDIDATES = [(1, 1.0, 0.0), (4, 1.0, 0.5), (8, 1.0, 0.5), (16, 1.0, 0.5), (8, 0.5, 0.5),
              (8, 2.0, 0.5), (8, 0.25, 0.75), (16, 0.5, 0.75), (32, 1.0, 0.5)]
# (blocks per SM, row groups per thread, vector width); (0, 0, 0) = each
# method's default
SHAPES = [(0, 0, 0), (4, 1, 1), (4, 2, 1), (4, 4, 1), (3, 1, 1), (3, 2, 1), (3, 4, 1), (4, 1, 2)]


def set_schedule(gang_size: int, large_work_factor: float = 1.0, max_gang_fraction: float = 0.5):
    plcg._check(plcg.load().plcg_set_batched_schedule(int(gang_size), float(large_work_factor),
                                                      float(max_gang_fraction)))


def set_launch(ctas_per_sm: int = 0, rows_per_thread: int = 0, vector_width: int = 0):
    """(0, 0, 0): each method's default.  A non-default shape with
    vector_width 0 means one-wide rows."""
    if (ctas_per_sm or rows_per_thread) and not vector_width:
        vector_width = 1
    plcg._check(plcg.load().plcg_set_batched_launch(int(ctas_per_sm), int(rows_per_thread),
                                                    int(vector_width)))


def _time(mats, bs, lmins, lmaxs, repeats, kw):
    import torch
    best = None
    for _ in range(repeats):
        xs = [torch.zeros_like(b) for b in bs]
        st, res = plcg.solve_batched(mats, bs, xs, lmins=lmins, lmaxs=lmaxs, check=False, **kw)
        if st != plcg.PLCG_OK:
            return float("inf")
        t = res[0].seconds
        best = t if best is None else min(best, t)
    return best


def tune_batched(mats, bs, lmins=None, lmaxs=None, candidates=CANDIDATES, shapes=None, repeats=1, **kw):
    """Time the launch shapes (FP32 solves) and then the gang schedules on
    this batch (x0 = 0 each time), install the fastest and return
    (schedule, shape, {("shape", s) or ("schedule", c): seconds})."""
    if shapes is None:
        shapes = SHAPES if kw.get("prec") == "fp32" else [(0, 0, 0)]
    times = {}
    set_schedule(0)
    for shp in shapes:
        set_launch(*shp)
        times[("shape", shp)] = _time(mats, bs, lmins, lmaxs, repeats, kw)
    shape = min(shapes, key=lambda s_: times[("shape", s_)])
    set_launch(*shape)
    for cand in candidates:
        set_schedule(*cand)
        times[("schedule", cand)] = _time(mats, bs, lmins, lmaxs, repeats, kw)
    choice = min(candidates, key=lambda c_: times[("schedule", c_)])
    set_schedule(*choice)
    return choice, shape, times
