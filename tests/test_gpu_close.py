"""The deferred step close against the close inside each step's own graph.

By default a step graph leaves the step's close (the block-partial sums, the
probes, the FP64 accumulators, the CFL gate of eq. cfl) to the next step's
graph, where it runs beside that step's drift, and the drift takes its dt from
the last pass's maximum |v|.  The library runs a pending close before any call
that reads, saves, replaces or batches the case.  Whatever the sequence of
calls, every array, probe record and scalar must equal the inline close's bit
for bit.
"""
import os
import tempfile

import numpy as np
import pytest

from helpers import impact_case, perturbed

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_05494_b300 import Batch, Case  # noqa: E402


def _same(a, b):
    sa, sb = a.get_state(), b.get_state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(a.probe_pressure(), b.probe_pressure())
    assert np.array_equal(a.probe_times(), b.probe_times())
    assert a.scalars() == b.scalars()


def _calls(c):
    # single steps, runs through the four-step graph, reads in between
    for _ in range(3):
        c.step()
    c.scalars()
    c.run(9)
    c.probe_pressure()
    c.step()
    c.step()
    c.diagnostics()
    c.run(8)


def _case(kind):
    kw = {}
    if kind == "impact":
        p, xy = impact_case()
        vel = None
    elif kind == "split":
        p, xy = impact_case()
        vel = None
        kw = dict(split=True)
    elif kind == "paper":
        p, xy = impact_case(closure=1)
        vel = None
    elif kind == "fixed_dt":
        p, xy = impact_case(dt_mode=1)
        vel = None
    elif kind == "closed_box":
        p, xy = impact_case(end_walls=1)
        vel, _ = perturbed(p, xy, seed=9, v_amp=5.0, rho_rel=0.0)
    elif kind == "lanes4":
        p, xy = impact_case()
        vel = None
        kw = dict(lanes=4)
    else:   # cells of side h, the 5 x 5 stencil
        p, xy = impact_case(cell_factor=0.5)
        vel = None
    return p, xy, vel, kw


@pytest.mark.parametrize("kind", ["impact", "split", "paper", "fixed_dt", "closed_box",
                                  "lanes4", "cells_h"])
def test_deferred_close_bitwise(kind):
    p, xy, vel, kw = _case(kind)
    a = Case(p, xy, vel, close_inline=True, **kw)
    b = Case(p, xy, vel, **kw)
    assert a.info()["close_deferred"] == 0 and b.info()["close_deferred"] == 1
    _calls(a)
    _calls(b)
    _same(a, b)


def test_deferred_close_periodic_diagnostics_and_t_end():
    # the periodic diagnostics read the state between steps; hr_run with an
    # end time polls t and dt between its graph launches
    p, xy = impact_case()
    with Case(p, xy, close_inline=True, diag_every=3) as a, Case(p, xy, diag_every=3) as b:
        for c in (a, b):
            c.run(10)
            c.run(0, t_end=c.scalars()["t"] + 2e-6)
        assert np.array_equal(a.diag_history(), b.diag_history())
        _same(a, b)


def test_deferred_close_save_load_and_set_state():
    p, xy = impact_case()
    vel, rho = perturbed(p, xy, seed=3)
    a = Case(p, xy, close_inline=True)
    b = Case(p, xy)
    with tempfile.TemporaryDirectory() as d:
        for c, name in ((a, "a.bin"), (b, "b.bin")):
            c.run(7)
            c.save(os.path.join(d, name))
            c.run(5)          # left pending, then replaced by the load
            c.load(os.path.join(d, name))
            c.run(6)
            c.step()
            c.set_state(xy, vel, rho)   # a pending close is dropped with the state
            c.run(5)
    _same(a, b)


@pytest.mark.parametrize("persistent", [False, True])
def test_deferred_close_then_batch_and_back(persistent):
    # a case with a pending close taken into a batch (a graph of batched
    # launches, or one persistent launch) continues as the inline-closed
    # case does, and steps alone again after
    p, xy = impact_case()
    a = Case(p, xy, close_inline=True)
    b = Case(p, xy)
    for c in (a, b):
        c.run(6)
        c.step()
    t_end = a.scalars()["t"] + 2e-6
    for c in (a, b):
        with Batch([c], t_end, persistent=persistent) as bt:
            bt.run()
        c.run(5)
    _same(a, b)
