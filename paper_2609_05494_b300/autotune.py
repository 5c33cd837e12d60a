"""Autotuner for single cases and batched sweeps.

Four choices are tuned by timing them on the device, not by a model:

* the cell grid of each case: the cell side as a multiple of the support
  2h (``cell_factor``).  Larger cells mean more candidates per particle in
  the interaction pass but fewer cells to scan in the sort; a factor of 0.5
  gives cells of side h and the 5 x 5 stencil (25 h^2 of candidates against
  at least 36 h^2);
* the block schedule of a batch: the order in which the blocks of each
  batched launch visit the cases (case after case, round robin, largest
  case first);
* the lanes per particle of a single case's interaction pass (1, 2 or 4);
* the block counts of a persistent batch: how many of the resident blocks
  each case gets.  Candidates share the capacity in proportion to
  particles^a x (estimated steps)^b; the estimated steps of a case are its
  stop time over its fixed-speed time step C h / (c0 + v0).  The split by
  particles x steps stays unless another is clearly faster.
Results do not depend on any of these choices: only time does.

Tuning runs work on throw-away copies of the cases, so the cases handed back
start from the same state as untuned ones.
"""
from __future__ import annotations

import numpy as np

from .api import Batch, Case

CELL_FACTORS = (0.5, 1.001, 1.1, 1.25)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_case(params: dict, xy, steps: int = 20, warmup: int = 3, stream=None) -> float:
    """Mean ms per step of one case over ``steps`` graph replays."""
    import torch
    with Case(params, xy, stream=stream) as c:
        c.run(warmup)
        a, b = _events()
        s = torch.cuda.current_stream() if stream is None else stream
        a.record(s)
        c.run(steps)
        b.record(s)
        b.synchronize()
        return a.elapsed_time(b) / steps


def tune_cell_factor(params: dict, xy, candidates=CELL_FACTORS, steps: int = 20,
                     stream=None) -> tuple[float, dict]:
    """Fastest cell_factor for this case and the timings of every candidate."""
    timings = {}
    for f in candidates:
        p = dict(params)
        p["cell_factor"] = float(f)
        timings[float(f)] = time_case(p, xy, steps=steps, stream=stream)
    best = min(timings, key=timings.get)
    return best, timings


def tune_pass_lanes(params: dict, xy, candidates=(1, 2, 4), steps: int = 20,
                    stream=None) -> tuple[int, dict]:
    """Lanes per particle of the interaction pass for a single case: the
    fastest of ``candidates`` and every candidate's ms per step.  More lanes
    shorten the pass's critical path in small, latency-bound cases and cost
    instructions in large ones."""
    import torch
    timings = {}
    for lanes in candidates:
        with Case(params, xy, stream=stream, lanes=lanes) as c:
            c.run(3)
            a, b = _events()
            s = torch.cuda.current_stream() if stream is None else stream
            a.record(s)
            c.run(steps)
            b.record(s)
            b.synchronize()
            timings[int(lanes)] = a.elapsed_time(b) / steps
    return min(timings, key=timings.get), timings


def tune_sweep(specs, classes: int = 3, stream=None):
    """Tunes a list of (params, xy) cases for a batched run.

    The cell grid is tuned once per size class (cases sorted by particle
    count and split into ``classes`` groups; the median case of each group
    is timed) and applied to every case of the class.  The block schedule is
    then tuned on a batch of all cases over 10 batched steps.
    Returns (tuned specs, schedule, report)."""
    import torch
    n = np.array([xy.shape[0] for _, xy in specs])
    order = np.argsort(n)
    groups = [g for g in np.array_split(order, max(1, min(classes, len(specs)))) if len(g)]
    chosen = {}
    report = {"classes": []}
    for g in groups:
        rep = int(g[len(g) // 2])
        best, timings = tune_cell_factor(specs[rep][0], specs[rep][1], stream=stream)
        for k in g:
            chosen[int(k)] = best
        report["classes"].append({"cases": len(g), "particles": int(n[rep]),
                                  "cell_factor": best, "ms_per_step": timings})
    tuned = []
    for k, (p, xy) in enumerate(specs):
        q = dict(p)
        q["cell_factor"] = chosen[k]
        tuned.append((q, xy))
    sched_ms = {}
    for sched in range(len(Batch.SCHEDULES)):
        cases = [Case(p, xy, stream=stream) for p, xy in tuned]
        with Batch(cases, 1.0, stream=stream, schedule=sched) as b:   # no case ends here
            b.run(max_steps=3)
            a, e = _events()
            s = torch.cuda.current_stream() if stream is None else stream
            a.record(s)
            for _ in range(10):
                b.step()
            e.record(s)
            e.synchronize()
            sched_ms[Batch.SCHEDULES[sched]] = a.elapsed_time(e) / 10
        for c in cases:
            c.close()
    schedule = min(range(len(Batch.SCHEDULES)), key=lambda k: sched_ms[Batch.SCHEDULES[k]])
    report["schedule_ms_per_step"] = sched_ms
    report["schedule"] = Batch.SCHEDULES[schedule]
    return tuned, schedule, report


BLOCK_WEIGHTS = ((1.0, 0.0), (1.0, 1.0), (1.0, 0.5), (0.5, 1.0))
# the split by particles x steps, the work each case has left: kept unless
# another split is faster over the horizon by more than this fraction (the
# horizon sees the cases' imbalance only in part, and near-ties go either way)
DEFAULT_WEIGHT = (1.0, 1.0)
PERSIST_MARGIN = 0.03


def block_counts(specs, capacity: int, a: float, b: float, t_end: float) -> np.ndarray:
    """Resident blocks per case: the capacity shared in proportion to
    particles^a x (t_end / dt_estimate)^b, at least one each."""
    w = []
    for p, xy in specs:
        h = p["h_over_dx"] * p["dx"]
        dt = p["cfl"] * h / (p["c0"] + p["v0"])
        w.append(float(xy.shape[0]) ** a * (t_end / dt) ** b)
    w = np.array(w)
    n = np.maximum(1, np.floor(capacity * w / w.sum())).astype(np.int64)
    while n.sum() > capacity:
        n[np.argmax(n)] -= 1
    return n.astype(np.int32)


def tune_persistent(specs, t_end: float, horizon: float = 250e-6, stream=None, weights=BLOCK_WEIGHTS,
                    margin: float = PERSIST_MARGIN):
    """Block counts of a persistent batch: each candidate split of the resident
    blocks (weights (a, b) of block_counts) runs the sweep's first ``horizon``
    seconds of simulated time on throw-away copies.  The split by particles x
    steps (DEFAULT_WEIGHT) is kept unless another is faster by more than
    ``margin`` (a fraction).  Cases tuned to the 5 x 5 stencil run on cells of
    side 2h here.  Returns (case_blocks, report)."""
    import torch
    closure = int(specs[0][0].get("closure", 0))
    cap = Batch.capacity(closure)
    # the persistent kernel takes the 3 x 3 stencil only
    specs = [(dict(p, cell_factor=max(float(p.get("cell_factor", 1.001)), 1.001)), xy)
             for p, xy in specs]
    report = {"capacity": cap, "candidates": []}
    for a, b in weights:
        nb = block_counts(specs, cap, a, b, t_end)
        cases = [Case(p, xy, stream=stream) for p, xy in specs]
        s = torch.cuda.current_stream() if stream is None else stream
        with Batch(cases, min(horizon, t_end), stream=stream, persistent=True,
                   case_blocks=nb) as bt:
            e0, e1 = _events()
            e0.record(s)
            bt.run()
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
        for c in cases:
            c.close()
        report["candidates"].append({"a": a, "b": b, "ms": ms,
                                     "blocks_min": int(nb.min()), "blocks_max": int(nb.max())})
    a, b, best_ms = choose_weight(report["candidates"], margin)
    best = block_counts(specs, cap, a, b, t_end)
    report["chosen"] = {"a": a, "b": b, "blocks": best.tolist(), "ms": best_ms}
    return best, report


def choose_weight(candidates, margin: float = PERSIST_MARGIN):
    """(a, b, ms) of the split to use among timed candidates (dicts with a, b,
    ms): DEFAULT_WEIGHT unless another is faster by more than ``margin``."""
    fast = min(candidates, key=lambda c: c["ms"])
    for c in candidates:
        if (c["a"], c["b"]) == DEFAULT_WEIGHT and c["ms"] <= fast["ms"] * (1.0 + margin):
            return c["a"], c["b"], c["ms"]
    return fast["a"], fast["b"], fast["ms"]
