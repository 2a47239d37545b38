"""The batched autotuner's search (host logic, no GPU): FP32 solves time
every launch shape -- including the 2-wide vector rows -- under the default
schedule, then every gang schedule under the fastest shape, and install the
fastest pair last; FP64 solves time the default shape only; a candidate
whose solve fails times as infinity and is never chosen.  The library
calls are replaced by recorders; the solves' times are synthetic."""
import math

from paper_1905_06850_gb300 import autotune


class Recorder:
    def __init__(self, shape_times, sched_times):
        self.shape_times, self.sched_times = shape_times, sched_times
        self.launch, self.sched, self.calls = None, None, []

    def set_launch(self, *shp):
        self.launch = tuple(shp)
        self.calls.append(("launch", self.launch))

    def set_schedule(self, *c):
        self.sched = tuple(c)
        self.calls.append(("schedule", self.sched))

    def time(self, mats, bs, lmins, lmaxs, repeats, kw):
        if self.sched in self.sched_times:
            return self.sched_times[self.sched]
        return self.shape_times.get(self.launch, 1.0)


def run(monkeypatch, shape_times, sched_times, **kw):
    r = Recorder(shape_times, sched_times)
    monkeypatch.setattr(autotune, "set_launch", r.set_launch)
    monkeypatch.setattr(autotune, "set_schedule", r.set_schedule)
    monkeypatch.setattr(autotune, "_time", r.time)
    return r, autotune.tune_batched([], [], **kw)


def test_shapes_include_the_vector_rows_and_the_default():
    assert (0, 0, 0) in autotune.SHAPES and (4, 1, 2) in autotune.SHAPES
    assert len(set(autotune.SHAPES)) == len(autotune.SHAPES)


def test_fp32_picks_the_fastest_shape_then_schedule(monkeypatch):
    shape_times = {s: 1.0 + 0.01 * i for i, s in enumerate(autotune.SHAPES)}
    shape_times[(4, 1, 2)] = 0.5
    sched_times = {c: 2.0 for c in autotune.CANDIDATES}
    sched_times[autotune.CANDIDATES[3]] = 0.4
    r, (sched, shape, times) = run(monkeypatch, shape_times, sched_times, prec="fp32", l=1)
    assert shape == (4, 1, 2) and sched == autotune.CANDIDATES[3]
    assert {k[1] for k in times if k[0] == "shape"} == set(autotune.SHAPES)
    assert {k[1] for k in times if k[0] == "schedule"} == set(autotune.CANDIDATES)
    # the chosen pair is what stays installed
    assert r.launch == (4, 1, 2) and r.sched == autotune.CANDIDATES[3]
    # shapes are timed under the default schedule
    first_launch = next(i for i, c in enumerate(r.calls) if c[0] == "launch")
    assert ("schedule", (0,)) in r.calls[:first_launch]


def test_fp64_times_the_default_shape_only(monkeypatch):
    r, (sched, shape, times) = run(monkeypatch, {}, {c: 1.0 for c in autotune.CANDIDATES}, prec="fp64", l=2)
    assert shape == (0, 0, 0)
    assert [k for k in times if k[0] == "shape"] == [("shape", (0, 0, 0))]


def test_a_failing_candidate_is_never_chosen(monkeypatch):
    shape_times = {s: math.inf for s in autotune.SHAPES}
    shape_times[(3, 2, 1)] = 0.9
    r, (sched, shape, times) = run(monkeypatch, shape_times, {c: 1.0 for c in autotune.CANDIDATES},
                                   prec="fp32", method="cg")
    assert shape == (3, 2, 1)
