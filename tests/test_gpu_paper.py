"""CUDA path, the paper's closure (closure 1: cubic B-spline, summation
density, Mie-Grueneisen EOS, internal-energy equation) against the FP64
oracle on identical seeded inputs, with the gates of the closure-0 parity
tests: density 1e-5 relative, pressure 1e-5 of max(max |p|, rho0 c0^2),
positions 1e-6 m, probe histories 1e-3 relative L2 (plus, for weak probes,
the 1e-5 rho0 c0^2 pressure floor that float32 positions put on a summed
density)."""
import numpy as np
import pytest

import casegen
import oracle
from helpers import as64, assert_p_close, impact_case, perturbed, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_05494_b300 import Batch, Case, HramError, _lib  # noqa: E402


def paper_case(**kw):
    q = dict(closure=1, c0=1448.0, alpha=0.03, cfl=0.25, motion=1)
    q.update(kw)
    return impact_case(**q)


def both(p, xy32, vel=None, rho=None, **kw):
    return Case(p, xy32, vel, rho, **kw), oracle.OracleCase(p, as64(xy32), as64(vel), as64(rho))


def compare_state(p, g, o, dt, name, dens_rel=1e-5, e_rel=1e-4):
    sg, fo = g.get_state(), o.fluid()
    assert np.abs(sg["rho"] / fo["rho"] - 1.0).max() <= dens_rel
    assert_p_close(name, p, sg["p"], o, dt)
    assert np.abs(sg["xy"] - fo["xy"]).max() <= 1e-6
    vscale = max(np.abs(fo["vel"]).max(), 1.0)
    assert np.abs(sg["vel"] - fo["vel"]).max() <= 1e-4 * vscale
    eg, eo = g.energy(), o.energy()
    escale = max(np.abs(eo["e"]).max(), 1e-3)
    assert np.abs(eg["e"] - eo["e"]).max() <= e_rel * escale
    dscale = max(np.abs(eo["de"]).max(), 1e-3)
    assert np.abs(eg["de"] - eo["de"]).max() <= e_rel * dscale


def test_prime_summation_density_and_pressure():
    p, xy = paper_case()
    g, o = both(p, xy)
    sg, fo = g.get_state(), o.fluid()
    # the summed density replaces the given one, on both sides
    assert np.abs(sg["rho"] / fo["rho"] - 1.0).max() <= 1e-6
    assert_p_close("paper_prime", p, sg["p"], o, o.scalars()["dt"])
    assert np.all(g.energy()["e"] == 0.0)


@pytest.mark.parametrize("state", ["rest_impact", "perturbed"])
def test_one_step(state):
    p, xy = paper_case()
    vel = None
    if state == "perturbed":
        vel, _ = perturbed(p, xy)
    g, o = both(p, xy, vel)
    dt = o.scalars()["dt"]
    g.step()
    o.step()
    compare_state(p, g, o, dt, "paper_one_step " + state)
    assert abs(g.scalars()["dt"] / o.scalars()["dt"] - 1.0) <= 1e-6


def test_ghosts_after_steps():
    p, xy = paper_case()
    g, o = both(p, xy)
    g.run(5)
    o.run(5)
    gg, go = g.ghosts(), o.ghosts()
    pmax = max(np.abs(go["p"]).max(), 1.0)
    assert np.abs(gg["p"] - go["p"]).max() <= 1e-5 * max(pmax, p["rho0"] * p["c0"] ** 2)
    vmax = max(np.abs(go["vel"]).max(), 1.0)
    assert np.abs(gg["vel"] - go["vel"]).max() <= 1e-4 * vmax


def test_probe_history_and_diagnostics_window():
    p, xy = paper_case()
    p["probes"] = list(p["probes"]) + [(0.030, 0.0), (0.020, 0.030), (0.060, 0.0)]
    g, o = both(p, xy)
    n = p["n_steps"]
    g.run(n)
    o.run(n)
    pg, po = g.probe_pressure(), o.probes()[0]
    assert pg.shape == po.shape == (n, len(p["probes"]))
    # Summed density makes the pressure a direct function of the float32
    # positions: the GPU state carries a pressure floor of about 1e-5 rho0 c0^2
    # (the one-step gate's pressure scale).  Probes that see the entry shock
    # (peak > 10 MPa) meet 1e-3 relative L2 outright; every probe meets
    # 1e-3 relative L2 plus that floor.
    floor = 1e-5 * p["rho0"] * p["c0"] ** 2
    strong = 0
    for k in range(po.shape[1]):
        err = np.sqrt(np.mean((pg[:, k] - po[:, k]) ** 2))
        rms = np.sqrt(np.mean(po[:, k] ** 2))
        assert err <= 1e-3 * rms + floor, k
        if np.abs(po[:, k]).max() > 1e7:
            assert rel_l2(pg[:, k], po[:, k]) <= 1e-3, k
            strong += 1
    assert strong >= 2
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("KE", "E_el", "W_boundary", "dissipation", "wall_impulse"):
        assert dg[k] == pytest.approx(do[k], rel=1e-3), k
    assert dg["n_in"] == do["n_in"]


def test_state_moves_with_summation_not_input_density():
    # closure 1 ignores the density handed in: two uploads that differ only
    # in rho give bit-identical states
    p, xy = paper_case(Lx=0.04, W=0.04, x_c0=0.01, v0=100.0)
    _, rho = perturbed(p, xy)
    with Case(p, xy) as a, Case(p, xy, rho=rho) as b:
        a.run(10)
        b.run(10)
        sa, sb = a.get_state(), b.get_state()
        for key in sa:
            assert np.array_equal(sa[key], sb[key]), key


def test_closure_restrictions():
    p, xy = paper_case(Lx=0.04, W=0.04)
    with Case(p, xy) as c, Case(dict(p, closure=0), xy) as c0:
        # one closure per batch
        with pytest.raises(HramError) as e:
            Batch([c, c0], 1e-5)
        assert e.value.code == _lib.HR_EINVAL
    q = dict(p)
    q["dt_mode"] = 1
    q["motion"] = 0
    with pytest.raises(HramError):
        Case(q, xy, tangent=True)
    r = dict(p)
    r["mg_mu_max"] = 1.5      # 1 - (S1 - 1) mu would cross zero below the cap
    with pytest.raises(HramError):
        Case(r, xy)
    with Case(dict(p, closure=0), xy) as c0:
        with pytest.raises(HramError):
            c0.energy()


def test_paper_setup_runs_and_peaks_in_the_papers_range():
    # the paper's own geometry and closure (750 x 150 mm, dx = 1.5 mm, drag
    # law, centreline probes PTn / PTf), 40 us of the entry phase.  Magnitude
    # sanity only: the paper's table gives PTn peaks of 850-894 MPa at
    # 900 m/s; a planar 2-D run at this resolution is not a parity target.
    p = casegen.config_paper(900.0)
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                               disk=(p["x_c0"], p["y_c0"], p["R_disk"])).astype(np.float32)
    with Case(p, xy) as c:
        st = c.run(0, 40e-6)
        assert st >= 0
        pr = c.probe_pressure()
        d = c.diagnostics()
    assert np.all(np.isfinite(pr))
    ptn = pr[:, 0].max()
    assert 1e8 < ptn < 3e9
    assert d["n_in"] == xy.shape[0]


def test_hard_reflection_wall_matches_oracle():
    # the paper's baseline wall: no ghost layers, reflection at |y| = W/2
    p, xy = paper_case(wall_layers=0, wall_reflect=1)
    g, o = both(p, xy)
    dt = o.scalars()["dt"]
    g.run(3)
    o.run(3)
    sg, fo = g.get_state(), o.fluid()
    assert np.abs(sg["xy"] - fo["xy"]).max() <= 1e-6
    # a summed density turns float32 position rounding into pressure: the
    # floor of three steps
    assert_p_close("paper_hard_wall 3 steps", p, sg["p"], o, dt, steps=3)
    g.run(40)
    assert np.all(np.abs(g.get_state()["xy"][:, 1]) <= 0.5 * p["W"])
    assert g.scalars()["wall_impulse"] == 0.0


def test_checkpoint_resume_bitwise_paper_closure():
    # closure 1 carries the internal energy and its rate in the checkpoint
    import os
    import tempfile
    p, xy = paper_case()
    a = Case(p, xy)
    a.run(20)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        a.save(path)
        a.run(15)
        b = Case(p, xy)
        b.load(path)
        b.run(15)
    sa, sb = a.get_state(), b.get_state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    ea, eb = a.energy(), b.energy()
    assert np.array_equal(ea["e"], eb["e"]) and np.array_equal(ea["de"], eb["de"])
    assert np.array_equal(a.probe_pressure(), b.probe_pressure())


def test_batch_of_paper_cases_equals_cases_run_alone():
    # the paper's coefficient sweep in closure 1 (artificial viscosity and
    # impact speed varied per case, different channel widths so the cell
    # grids differ): batched cases end bit-for-bit where they end alone,
    # energies included, under every block schedule
    t_end = 8e-6
    specs = [paper_case(alpha=a, v0=v, W=w, probes=[(0.030, 0.5 * w), (0.060, -0.5 * w)])
             for a, v, w in ((0.01, 900.0, 0.15), (0.03, 600.0, 0.12), (0.1, 750.0, 0.10))]
    alone = []
    for p, xy in specs:
        a = Case(p, xy)
        a.run(0, t_end)
        alone.append(a)
    for schedule in (0, 1, 2):
        batched = [Case(p, xy) for p, xy in specs]
        with Batch(batched, t_end, schedule=schedule) as b:
            b.run()
            assert b.n_done() == len(batched)
        for a, g in zip(alone, batched):
            sa, sg = a.get_state(), g.get_state()
            for k in sa:
                assert np.array_equal(sa[k], sg[k]), (schedule, k)
            ea, eg = a.energy(), g.energy()
            assert np.array_equal(ea["e"], eg["e"]) and np.array_equal(ea["de"], eg["de"])
            assert np.array_equal(a.probe_pressure(), g.probe_pressure())
            assert a.scalars()["step"] == g.scalars()["step"]
