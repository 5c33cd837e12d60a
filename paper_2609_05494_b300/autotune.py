"""Autotuner for single cases and batched sweeps.

Two choices are tuned by timing them on the device, not by a model:

* the cell grid of each case: the cell side as a multiple of the support
  2h (``cell_factor``).  Larger cells mean more candidates per particle in
  the interaction pass but fewer cells to scan in the sort;
* the block schedule of a batch: the order in which the blocks of each
  batched launch visit the cases (case after case, round robin, largest
  case first).  Results do not depend on either choice: only time does.

Tuning runs work on throw-away copies of the cases, so the cases handed back
start from the same state as untuned ones.
"""
from __future__ import annotations

import numpy as np

from .api import Batch, Case

CELL_FACTORS = (1.001, 1.1, 1.25)


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
