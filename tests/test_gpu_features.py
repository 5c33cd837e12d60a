"""CUDA path: diagnostics, boundary variants, edge cases, checkpoint/resume,
status codes and the full-size workload, each against the FP64 oracle or an
exact property."""
import math
import os
import tempfile

import numpy as np
import pytest

import casegen
import oracle
from helpers import as64, assert_p_close, csr_equal, impact_case, perturbed, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_05494_b300 import Case, HramError, _lib  # noqa: E402


def both(p, xy32, vel=None, rho=None, **kw):
    return Case(p, xy32, vel, rho, **kw), oracle.OracleCase(p, as64(xy32), as64(vel), as64(rho))


def test_diagnostics_match_oracle():
    p, xy = impact_case()
    g, o = both(p, xy)
    g.run(60)
    o.run(60)
    dg, do = g.diagnostics(), o.diagnostics()
    assert dg["mass"] == pytest.approx(do["mass"], rel=1e-6)
    assert dg["n_in"] == do["n_in"] and dg["step"] == do["step"] == 60
    assert dg["t"] == pytest.approx(do["t"], rel=1e-6)
    for k in ("KE", "E_el", "W_boundary", "dissipation"):
        assert dg[k] == pytest.approx(do[k], rel=1e-3), k
    scale = math.hypot(do["px"], do["py"])
    assert abs(dg["px"] - do["px"]) <= 1e-3 * scale and abs(dg["py"] - do["py"]) <= 1e-3 * scale
    assert dg["wall_impulse"] == pytest.approx(do["wall_impulse"], rel=1e-3, abs=1e-9)
    assert dg["p_max"] == pytest.approx(do["p_max"], rel=1e-4)
    assert dg["rho_max"] == pytest.approx(do["rho_max"], rel=1e-5)
    sg, so = g.scalars(), o.scalars()
    # t is a sum of CFL steps whose v_max agrees to ~1e-7, so the kinematics
    # (exact functions of t) agree to that level here
    for k in ("xc", "vproj", "aproj"):
        assert sg[k] == pytest.approx(so[k], rel=1e-6), k
    assert sg["Fdisk_x"] == pytest.approx(so["Fdisk_x"], rel=1e-3)


def test_periodic_diagnostics_recorded():
    p, xy = impact_case()
    with Case(p, xy, diag_every=5) as g:
        g.run(20)
        h = g.diag_history()
        assert h.shape[0] == 4
        assert np.allclose(h[:, -1], [5, 10, 15, 20])
        assert np.all(np.diff(h[:, 13]) > 0)


@pytest.mark.parametrize("motion", [0, 1, 2])
def test_motion_laws_match_oracle(motion):
    # fixed dt: both sides accumulate the same t, so the FP64 closed forms agree
    p, xy = impact_case(motion=motion, a_const=2.0e7, dt_mode=1)
    g, o = both(p, xy)
    g.run(40)
    o.run(40)
    sg, so = g.scalars(), o.scalars()
    assert sg["t"] == so["t"]
    for k in ("xc", "vproj", "aproj"):
        assert sg[k] == pytest.approx(so[k], rel=1e-13), k
    pg, po = g.get_state()["p"], o.fluid()["p"]
    assert np.abs(pg - po).max() <= 1e-3 * np.abs(po).max()


def test_closed_box_rest_state_exact():
    p, xy = impact_case(Lx=0.03, W=0.02, dx=1e-3, end_walls=1, gx=0.0, gy=0.0, v0=0.0,
                        x_c0=0.012, R_disk=3e-3, Ng=40)
    with Case(p, xy) as g:
        s0 = g.get_state()
        g.run(30)
        s1 = g.get_state()
        assert np.array_equal(s0["xy"], s1["xy"])
        assert np.all(s1["vel"] == 0.0) and np.all(s1["rho"] == p["rho0"])


def test_hydrostatic_column_gpu_vs_oracle():
    L = 0.03
    p, xy = impact_case(Lx=L, W=L, dx=1e-3, end_walls=1, Ng=0, c0=10 * math.sqrt(9.81 * L))
    B = p["rho0"] * p["c0"] ** 2 / p["gamma"]
    pr = p["rho0"] * 9.81 * (0.5 * L - xy[:, 1].astype(np.float64))
    rho = (p["rho0"] * (1 + pr / B) ** (1 / p["gamma"])).astype(np.float32)
    p["probes"] = [(0.5 * L, 0.0), (0.5 * L, -0.25 * L)]
    g, o = both(p, xy, None, rho)
    g.run(1500)
    o.run(1500)
    pg, po = g.probe_pressure(), o.probes()[0]
    expect = np.array([p["rho0"] * 9.81 * 0.5 * L, p["rho0"] * 9.81 * 0.75 * L])
    # the GPU column is in hydrostatic balance too (mean over the run's last 2/3)
    assert np.abs(pg[500:].mean(0) / expect - 1).max() < 0.05
    assert rel_l2(pg[:, 0], po[:, 0]) < 2e-2


@pytest.mark.parametrize("n", [1, 2, 37, 129])
def test_ragged_and_tiny_cases(n):
    p = casegen.base_params()
    p.update(Lx=0.02, W=0.02, dx=1e-3, Ng=0, wall_layers=0, gx=0.0, gy=0.0)
    rng = np.random.default_rng(n)
    xy = np.stack([rng.random(n) * 0.006 + 0.007, rng.random(n) * 0.006 - 0.003], 1).astype(np.float32)
    vel, rho = perturbed(p, xy, seed=n, v_amp=5.0)
    g, o = both(p, xy, vel, rho)
    off_g, ids_g = g.neighbours()
    off_o, ids_o = o.neighbours()
    assert csr_equal(off_g, ids_g, off_o, ids_o)
    g.run(3)
    o.run(3)
    sg, fo = g.get_state(), o.fluid()
    assert np.abs(sg["rho"] / fo["rho"] - 1).max() <= 1e-5
    assert np.abs(sg["xy"] - fo["xy"]).max() <= 1e-6


def test_frozen_particles_outside_box():
    p, xy = impact_case(Lx=0.03, W=0.03, dx=1e-3, Ng=0)
    xy = xy.copy()
    xy[:5, 0] = 1.0            # far outside the box: frozen from the start
    g, o = both(p, xy)
    g.run(10)
    o.run(10)
    sg, fo = g.get_state(), o.fluid()
    assert np.array_equal(sg["xy"][:5], xy[:5])
    assert np.all(fo["out"][:5] == 1)
    assert np.abs(sg["rho"] / fo["rho"] - 1).max() <= 1e-5
    assert g.diagnostics()["n_in"] == fo["out"].size - 5


def test_checkpoint_resume_bitwise():
    p, xy = impact_case()
    a = Case(p, xy)
    a.run(30)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        a.save(path)
        a.run(25)
        b = Case(p, xy)
        b.load(path)
        b.run(25)
    sa, sb = a.get_state(), b.get_state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(a.probe_pressure(), b.probe_pressure())
    assert a.scalars() == b.scalars()


@pytest.mark.parametrize("variant", [dict(stage=1), dict(newton3=True), dict(lanes=4),
                                     dict(cell_factor=0.5)])
def test_pass_variants_with_frozen_particles(variant):
    # particles outside the box keep their state in every pass variant
    kw = dict(variant)
    cf = kw.pop("cell_factor", None)
    p, xy = impact_case(Lx=0.03, W=0.03, dx=1e-3, Ng=0, **({"cell_factor": cf} if cf else {}))
    xy = xy.copy()
    xy[:5, 0] = 1.0
    g = Case(p, xy, **kw)
    o = oracle.OracleCase(p, as64(xy))
    g.run(10)
    o.run(10)
    sg, fo = g.get_state(), o.fluid()
    assert np.array_equal(sg["xy"][:5], xy[:5])
    assert np.abs(sg["rho"] / fo["rho"] - 1).max() <= 1e-5
    assert np.abs(sg["xy"] - fo["xy"]).max() <= 1e-6
    assert g.diagnostics()["n_in"] == fo["out"].size - 5


def test_caller_owned_output_buffers():
    # pinned (page-locked) caller buffers receive exactly what the library's
    # own arrays receive; wrong shapes or dtypes are refused before any copy
    p, xy = impact_case()
    with Case(p, xy) as c:
        c.run(12)
        ref_state, ref_probe = c.get_state(), c.probe_pressure()
        n = xy.shape[0]

        def pinned(shape):
            return torch.empty(shape, dtype=torch.float32).pin_memory().numpy()
        out = dict(xy=pinned((n, 2)), vel=pinned((n, 2)), rho=pinned((n,)), p=pinned((n,)))
        got = c.get_state(out=out)
        for k in ref_state:
            assert np.array_equal(got[k], ref_state[k]), k
            assert got[k] is out[k]
        buf = pinned((40, len(p["probes"])))
        pr = c.probe_pressure(out=buf)
        assert pr.shape == ref_probe.shape and np.array_equal(pr, ref_probe)
        with pytest.raises(ValueError):
            c.probe_pressure(out=np.zeros((5, len(p["probes"])), np.float32))
        with pytest.raises(ValueError):
            c.get_state(out=dict(out, rho=np.zeros(n, np.float64)))


def test_invalid_parameters_rejected():
    p, xy = impact_case()
    for bad in (dict(dx=0.0), dict(Ng=5000), dict(cfl=-1.0), dict(rho_hi=0.2),
                dict(cell_factor=0.4)):
        q = dict(p)
        q.update(bad)
        with pytest.raises(HramError) as e:
            Case(q, xy)
        assert e.value.code == _lib.HR_EINVAL
    # the staged pass variants take the 3 x 3 stencil, one variant at a time
    for kw, stage in ((dict(cell_factor=0.5), 1), (dict(cell_factor=0.5), 2)):
        with pytest.raises(HramError) as e:
            Case(dict(p, **kw), xy, stage=stage)
        assert e.value.code == _lib.HR_EINVAL
    # two pass variants at once; lanes or Newton-3 on cells of side h
    for kw in (dict(stage=1, newton3=True), dict(lanes=2, newton3=True), dict(stage=2, lanes=4)):
        with pytest.raises(HramError) as e:
            Case(p, xy, **kw)
        assert e.value.code == _lib.HR_EINVAL
    for kw in (dict(lanes=2), dict(newton3=True)):
        with pytest.raises(HramError) as e:
            Case(dict(p, cell_factor=0.5), xy, **kw)
        assert e.value.code == _lib.HR_EINVAL


def test_nan_state_reported():
    p, xy = impact_case()
    vel = np.zeros_like(xy)
    vel[7, 0] = np.nan                     # a NaN planted in the host-side state
    with pytest.raises(HramError) as e:
        Case(p, xy, vel)
    assert e.value.code == _lib.HR_ENAN


def test_probe_capacity_warning():
    p, xy = impact_case()
    with Case(p, xy, probe_capacity=4) as g:
        st = g.run(6)
        assert st & _lib.HR_WPROBEFULL
        assert g.probe_pressure().shape[0] == 4


def test_full_size_one_step_against_oracle():
    """The bench workload (1.125M particles) in the bench's launch
    configuration: one step from a perturbed state, every particle."""
    p = casegen.config_scaling(2e-4)
    p, xy = impact_case(p)
    vel, rho = perturbed(p, xy, seed=3, v_amp=10.0, rho_rel=0.005)
    g, o = both(p, xy, vel, rho)
    assert g.info()["split"] == 1   # the size takes the split pass by default
    dt = o.scalars()["dt"]
    g.step()
    o.step()
    sg, fo = g.get_state(), o.fluid()
    assert np.abs(sg["rho"] / fo["rho"] - 1).max() <= 1e-5
    # float32 positions at |x| ~ 0.3 m carry 3e-8 m rounding (6e-5 of 2h): the
    # per-particle rounding floor of the gate grows with |x| / h
    assert_p_close("full_size_1.125M", p, sg["p"], o, dt)
    assert np.abs(sg["xy"] - fo["xy"]).max() <= 1e-6
    assert g.scalars()["dt"] == pytest.approx(o.scalars()["dt"], rel=1e-6)


def test_full_size_split_pass_bitwise():
    # the bench workload's split pass against the one-kernel pass over a few
    # impact steps: every array, probe and scalar equal
    p = casegen.config_scaling(2e-4)
    p, xy = impact_case(p)
    a = Case(p, xy, split=False, probe_capacity=64)
    b = Case(p, xy, probe_capacity=64)
    assert a.info()["split"] == 0 and b.info()["split"] == 1
    a.run(6)
    b.run(6)
    sa, sb = a.get_state(), b.get_state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(a.probe_pressure(), b.probe_pressure())
    assert a.scalars() == b.scalars()


def test_two_way_coupling_matches_oracle():
    p, xy = impact_case(motion=3, t_ramp=2e-6, v0=300.0)
    g, o = both(p, xy)
    g.run(80)
    o.run(80)
    sg, so = g.scalars(), o.scalars()
    assert sg["vproj"] < 300.0
    for k in ("xc", "vproj"):
        assert sg[k] == pytest.approx(so[k], rel=1e-5), k
    assert sg["aproj"] == pytest.approx(so["aproj"], rel=1e-3)
    assert np.abs(g.get_state()["rho"] / o.fluid()["rho"] - 1).max() <= 1e-4


def test_fp32_rate_measurement():
    # the measured FMA rate is positive and within the unit-count bound
    # (SMs x 128 lanes x 2 x the maximum clock, with a margin for the
    # packed form, whose rate the measurement settles)
    from paper_2609_05494_b300 import fp32_rate
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * 2.2e9 / 1e12
    for packed in (False, True):
        r = fp32_rate(packed)
        assert 0.05 * bound < r < 2.2 * bound, (packed, r, bound)


def test_caller_workspace_must_be_aligned():
    # a caller-owned workspace 16 bytes off a 256-byte boundary is refused
    # before any device work; the aligned one is taken
    import ctypes as C
    from paper_2609_05494_b300 import make_params
    p, xy = impact_case()
    L = _lib.lib()
    par = make_params(p, 0, 64, 0)
    n = xy.shape[0]
    nbytes = C.c_size_t(0)
    assert L.hr_workspace_bytes(C.byref(par), n, C.byref(nbytes)) == 0
    ws = torch.empty(nbytes.value + 512, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    xyc = np.ascontiguousarray(xy, dtype=np.float32)
    h = C.c_void_p()
    rc = L.hr_init_case(C.byref(par), xyc.ctypes.data, n, None, None, C.c_void_p(base + 16),
                        nbytes.value, None, C.byref(h))
    assert rc == _lib.HR_EINVAL and not h.value
    rc = L.hr_init_case(C.byref(par), xyc.ctypes.data, n, None, None, C.c_void_p(base),
                        nbytes.value, None, C.byref(h))
    assert rc >= 0 and h.value
    L.hr_destroy(h)
    torch.cuda.synchronize()
