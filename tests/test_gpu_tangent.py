"""CUDA path, tangent-linear mode: derivatives of the peak probe-0 pressure
and the wall impulse along ln alpha, ln c0, ln tau against central finite
differences of the FP64 oracle on the same seeded inputs, plus the mode's
exact properties (the forward state is untouched, parameters that cannot
act give exactly zero, unsupported set-ups are refused)."""
import os
import tempfile

import numpy as np
import pytest

import casegen
import oracle
from helpers import as64, impact_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_05494_b300 import (Batch, Case, HramError, TANGENT_PARAMS, _lib,  # noqa: E402
                                   jacobian, peak_and_impulse)

N_STEPS = 250
FD_EPS = 1e-5      # relative central-difference step of the oracle
# FP32 tangents against FP64 differences: 2e-3 of the derivative, with a floor
# of 1e-5 of the output per unit ln(theta) for derivatives that are nearly
# zero.  Measured on B300: 3e-7 .. 6e-4 (the worst is d peak / d ln c0 under
# the drag law, where the peak's step sits on a steep front).
REL_TOL = 2e-3
FLOOR = 1e-5


def tangent_case(**kw):
    p, xy = impact_case(casegen.config_parity(), dt_mode=1, **kw)
    return p, xy


def oracle_outputs(p, xy, n_steps):
    o = oracle.OracleCase(p, as64(xy))
    o.run(n_steps)
    pr, _ = o.probes()
    return pr[:, 0], o.scalars()["wall_impulse"]


def oracle_fd(p, xy, n_steps, name):
    hi, lo = dict(p), dict(p)
    hi[name] = p[name] * (1.0 + FD_EPS)
    lo[name] = p[name] * (1.0 - FD_EPS)
    ph, jh = oracle_outputs(hi, xy, n_steps)
    pl, jl = oracle_outputs(lo, xy, n_steps)
    return (ph.max() - pl.max()) / (2 * FD_EPS), (jh - jl) / (2 * FD_EPS)


def gpu_tangent(p, xy, n_steps):
    with Case(p, xy, tangent=True) as c:
        c.run(n_steps)
        c.sync()
        return c.tangent_outputs(), c.probe_pressure()


def close(tan, fd, scale):
    return abs(tan - fd) <= REL_TOL * abs(fd) + FLOOR * abs(scale)


def test_tangents_match_oracle_central_differences():
    p, xy = tangent_case()
    out, hist = gpu_tangent(p, xy, N_STEPS)
    pr, J = oracle_outputs(p, xy, N_STEPS)
    # the outputs themselves and the peak's step
    assert out["peak_row"] == int(np.argmax(pr)) == int(np.argmax(hist[:, 0]))
    assert out["peak"] == pytest.approx(pr.max(), rel=1e-3)
    assert out["peak"] == float(hist[:, 0].max())
    assert out["impulse"] == pytest.approx(J, rel=1e-3)
    for k, name in enumerate(TANGENT_PARAMS):
        dP, dJ = oracle_fd(p, xy, N_STEPS, name)
        assert close(out["dpeak"][k], dP, out["peak"]), (name, out["dpeak"][k], dP)
        assert close(out["dimpulse"][k], dJ, out["impulse"]), (name, out["dimpulse"][k], dJ)


def test_tangent_mode_leaves_forward_state_bitwise():
    p, xy = tangent_case()
    with Case(p, xy) as a, Case(p, xy, tangent=True) as b:
        a.run(80)
        b.run(80)
        sa, sb = a.get_state(), b.get_state()
        for key in sa:
            assert np.array_equal(sa[key], sb[key]), key
        assert np.array_equal(a.probe_pressure(), b.probe_pressure())
        assert a.scalars() == b.scalars()


@pytest.mark.parametrize("motion", [1, 2])
def test_tau_derivative_exactly_zero_without_decay(motion):
    # motions 1 (drag) and 2 (constant acceleration) do not contain tau
    p, xy = tangent_case(motion=motion, a_const=2e6)
    out, _ = gpu_tangent(p, xy, 120)
    assert out["dpeak"][2] == 0.0 and out["dimpulse"][2] == 0.0
    assert np.all(np.isfinite(out["dpeak"])) and np.all(np.isfinite(out["dimpulse"]))


def test_motion_law_derivative_matches_oracle_drag():
    p, xy = tangent_case(motion=1)
    out, _ = gpu_tangent(p, xy, N_STEPS)
    for k, name in enumerate(("alpha", "c0")):
        dP, dJ = oracle_fd(p, xy, N_STEPS, name)
        assert close(out["dpeak"][k], dP, out["peak"]), (name, out["dpeak"][k], dP)
        assert close(out["dimpulse"][k], dJ, out["impulse"]), (name, out["dimpulse"][k], dJ)


def test_autograd_bridge_returns_library_jacobian():
    p, xy = tangent_case()
    theta = torch.tensor([p[k] for k in TANGENT_PARAMS], dtype=torch.float64,
                         requires_grad=True)
    y = peak_and_impulse(theta, p, xy, 60)
    y0, J = jacobian(theta.detach().numpy(), p, xy, 60)
    assert np.array_equal(y.detach().numpy(), y0)
    (y[0] + 2.0 * y[1]).backward()
    assert np.allclose(theta.grad.numpy(), J[0] + 2.0 * J[1], rtol=1e-12, atol=0.0)


def test_unsupported_set_ups_are_refused():
    p, xy = tangent_case()
    for kw in (dict(dt_mode=0), dict(motion=3), dict(cell_factor=0.5)):
        q = dict(p)
        q.update(kw)
        with pytest.raises(HramError) as e:
            Case(q, xy, tangent=True)
        assert e.value.code == _lib.HR_EINVAL
    with Case(p, xy) as plain:
        with pytest.raises(HramError):
            plain.tangent_outputs()
    with Case(p, xy, tangent=True) as t:
        with pytest.raises(HramError):
            Batch([t], 1e-5)
        t.run(5)
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "ck.bin")
            t.save(path)
            with pytest.raises(HramError):
                t.load(path)


def test_adjoint_workload_gradients_within_two_percent():
    # the 22,500-particle fixed-dt workload (150 x 150 mm, dx = 1 mm, 400
    # steps): every derivative against central differences of the FP64
    # oracle with relative step 1e-4, within 2 % (the workload's own bar)
    p = casegen.config_adjoint()
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                               disk=(p["x_c0"], p["y_c0"], p["R_disk"])).astype(np.float32)
    n = int(p["n_steps"])
    out, _ = gpu_tangent(p, xy, n)
    pr, J = oracle_outputs(p, xy, n)
    assert out["peak"] == pytest.approx(pr.max(), rel=1e-3)
    assert out["impulse"] == pytest.approx(J, rel=1e-3)
    for k, name in enumerate(TANGENT_PARAMS):
        hi, lo = dict(p), dict(p)
        hi[name] = p[name] * (1.0 + 1e-4)
        lo[name] = p[name] * (1.0 - 1e-4)
        ph, jh = oracle_outputs(hi, xy, n)
        pl, jl = oracle_outputs(lo, xy, n)
        dP, dJ = (ph.max() - pl.max()) / 2e-4, (jh - jl) / 2e-4
        assert abs(out["dpeak"][k] - dP) <= 0.02 * abs(dP) + 1e-6 * out["peak"], (name, out["dpeak"][k], dP)
        assert abs(out["dimpulse"][k] - dJ) <= 0.02 * abs(dJ) + 1e-6 * out["impulse"], (name, out["dimpulse"][k], dJ)


def test_tangents_on_rows_over_32_candidates():
    # the tangent pass's path for stencil rows longer than one mask: a patch
    # at half the spacing the smoothing length is set for, thrown at the
    # upper wall, against central differences of the oracle
    p = casegen.base_params()
    p.update(dx=1e-3, Lx=0.02, W=0.02, Ng=0, wall_layers=3, gy=0.0, dt_mode=1, v0=0.0)
    p["probes"] = [(0.010, 0.010)]
    xy = casegen.fluid_lattice(0.012, 0.012, 0.5e-3, 0.01, 21, disk=None)
    xy[:, 0] += 0.004
    xy[:, 1] += 0.003
    xy = xy.astype(np.float32)
    vel = np.zeros_like(xy)
    vel[:, 1] = 20.0
    n = 30

    def orc(q):
        o = oracle.OracleCase(q, as64(xy), as64(vel))
        o.run(n)
        pr, _ = o.probes()
        return pr[:, 0].max(), o.scalars()["wall_impulse"]

    with Case(p, xy, vel, tangent=True) as c:
        c.run(n)
        c.sync()
        out = c.tangent_outputs()
    P0, J0 = orc(p)
    assert out["peak"] == pytest.approx(P0, rel=1e-3) and out["impulse"] == pytest.approx(J0, rel=1e-3)
    for k, name in enumerate(("alpha", "c0")):
        hi, lo = dict(p), dict(p)
        hi[name] = p[name] * (1.0 + FD_EPS)
        lo[name] = p[name] * (1.0 - FD_EPS)
        (ph, jh), (pl, jl) = orc(hi), orc(lo)
        dP, dJ = (ph - pl) / (2 * FD_EPS), (jh - jl) / (2 * FD_EPS)
        assert close(out["dpeak"][k], dP, out["peak"]), (name, out["dpeak"][k], dP)
        assert close(out["dimpulse"][k], dJ, out["impulse"]), (name, out["dimpulse"][k], dJ)
