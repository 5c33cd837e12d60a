"""CUDA path, reverse mode: the adjoint sweep with checkpoints and
recomputation gives the derivatives of the peak probe-0 pressure and the wall
impulse along ln alpha, ln c0, ln tau.  It is checked against the tangent
(forward) mode, which computes the same discrete derivative in another
order, against central finite differences of the FP64 oracle on the
22,500-particle workload, and for its exact properties: the result does not
depend on the checkpoint interval, the forward state is left as a plain run
leaves it, and unsupported set-ups are refused."""
import numpy as np
import pytest

import casegen
import oracle
from helpers import as64, impact_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_05494_b300 import (Case, HramError, TANGENT_PARAMS, _lib,  # noqa: E402
                                   jacobian, peak_and_impulse)


def case0(**kw):
    return impact_case(casegen.config_parity(), dt_mode=1, **kw)


def adjoint(p, xy, n, every=20, vel=None):
    with Case(p, xy, vel) as c:
        y = c.adjoint_forward(n, every)
        d = c.adjoint_backward()
        return y, d


def tangent(p, xy, n, vel=None):
    with Case(p, xy, vel, tangent=True) as c:
        c.run(n)
        c.sync()
        return c.tangent_outputs()


def agree(a, t, scale, rel=1e-4, floor=1e-4):
    # 1e-4 of the derivative, or of the output itself per unit ln(theta) where
    # the derivative nearly cancels (the float32 sums behind both modes carry
    # terms of the output's size)
    return abs(a - t) <= rel * abs(t) + floor * abs(scale)


@pytest.mark.parametrize("n", [1, 60, 250])
def test_adjoint_equals_tangent(n):
    p, xy = case0()
    y, d = adjoint(p, xy, n)
    t = tangent(p, xy, n)
    assert y["peak"] == t["peak"] and y["peak_row"] == t["peak_row"]
    assert y["impulse"] == t["impulse"]
    for k, name in enumerate(TANGENT_PARAMS):
        print("ADJ n=%d %s dP adj %.9g tan %.9g | dJ adj %.9g tan %.9g"
              % (n, name, d["dpeak"][k], t["dpeak"][k], d["dimpulse"][k], t["dimpulse"][k]))
    for k, name in enumerate(TANGENT_PARAMS):
        assert agree(d["dpeak"][k], t["dpeak"][k], t["peak"]), (name, d["dpeak"][k], t["dpeak"][k])
        assert agree(d["dimpulse"][k], t["dimpulse"][k], t["impulse"]), \
            (name, d["dimpulse"][k], t["dimpulse"][k])


def test_adjoint_with_velocity_field_equals_tangent():
    # a moving, compressed start state: every term of the pass (AV switch,
    # laminar, XSPH, predictor) carries derivative from the first step
    p, xy = case0()
    rng = np.random.default_rng(4)
    vel = (20.0 * rng.standard_normal(xy.shape)).astype(np.float32)
    y, d = adjoint(p, xy, 40, vel=vel)
    t = tangent(p, xy, 40, vel=vel)
    for k, name in enumerate(TANGENT_PARAMS):
        print("ADJV %s dP adj %.9g tan %.9g | dJ adj %.9g tan %.9g"
              % (name, d["dpeak"][k], t["dpeak"][k], d["dimpulse"][k], t["dimpulse"][k]))
        assert agree(d["dpeak"][k], t["dpeak"][k], t["peak"]), name
        assert agree(d["dimpulse"][k], t["dimpulse"][k], t["impulse"]), name


def test_checkpoint_interval_does_not_change_the_result():
    # recomputation from checkpoints reproduces the forward records bit for
    # bit, so the Jacobian is the same for every interval
    p, xy = case0()
    ref = adjoint(p, xy, 90, every=20)[1]
    for every in (1, 7, 90, 200):
        d = adjoint(p, xy, 90, every=every)[1]
        assert np.array_equal(d["dpeak"], ref["dpeak"]), every
        assert np.array_equal(d["dimpulse"], ref["dimpulse"]), every


def test_forward_state_is_a_plain_run_and_backward_repeats():
    p, xy = case0()
    with Case(p, xy) as a, Case(p, xy) as b:
        a.run(70)
        b.adjoint_forward(70, 20)
        d1 = b.adjoint_backward()
        sa, sb = a.get_state(), b.get_state()
        for key in sa:
            assert np.array_equal(sa[key], sb[key]), key
        assert np.array_equal(a.probe_pressure(), b.probe_pressure())
        assert a.scalars() == b.scalars()
        d2 = b.adjoint_backward()
        assert np.array_equal(d1["dpeak"], d2["dpeak"])
        assert np.array_equal(d1["dimpulse"], d2["dimpulse"])
        # the case goes on as the plain one does
        a.run(5)
        b.run(5)
        assert np.array_equal(a.get_state()["xy"], b.get_state()["xy"])


@pytest.mark.parametrize("n,every,diag", [(15, 20, 0), (40, 20, 0), (40, 20, 5)])
def test_taped_last_segment(n, every, diag):
    # the forward run records its last segment as it goes (not with periodic
    # diagnostics): the state it leaves, and the derivatives of one or more
    # backward sweeps, equal those of a plain run and of the recomputing path
    p, xy = case0()
    with Case(p, xy) as a, Case(p, xy, diag_every=diag) as b:
        a.run(n)
        b.adjoint_forward(n, every)
        sa, sb = a.get_state(), b.get_state()
        for key in sa:
            assert np.array_equal(sa[key], sb[key]), key
        assert a.scalars() == b.scalars()
        d1 = b.adjoint_backward()
        d2 = b.adjoint_backward()
        assert np.array_equal(d1["dpeak"], d2["dpeak"])
        assert np.array_equal(d1["dimpulse"], d2["dimpulse"])
    ref = adjoint(p, xy, n, every=1)[1]      # every segment recomputed (one step each)
    assert np.array_equal(d1["dpeak"], ref["dpeak"])
    assert np.array_equal(d1["dimpulse"], ref["dimpulse"])


@pytest.mark.parametrize("motion", [1, 2])
def test_tau_derivative_exactly_zero_without_decay(motion):
    p, xy = case0(motion=motion, a_const=2e6)
    _, d = adjoint(p, xy, 80)
    assert d["dpeak"][2] == 0.0 and d["dimpulse"][2] == 0.0
    assert np.all(np.isfinite(d["dpeak"])) and np.all(np.isfinite(d["dimpulse"]))


def test_adjoint_workload_gradients_within_two_percent():
    # the 22,500-particle workload (150 x 150 mm, dx = 1 mm, 400 steps, fixed
    # dt, a checkpoint every 20 steps) against central differences of the FP64
    # oracle with relative step 1e-4: every derivative within 2 %
    p = casegen.config_adjoint()
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                               disk=(p["x_c0"], p["y_c0"], p["R_disk"])).astype(np.float32)
    n = int(p["n_steps"])
    y, d = adjoint(p, xy, n, every=20)

    def orc(q):
        o = oracle.OracleCase(q, as64(xy))
        o.run(n)
        pr, _ = o.probes()
        return pr[:, 0].max(), o.scalars()["wall_impulse"]

    P0, J0 = orc(p)
    assert y["peak"] == pytest.approx(P0, rel=1e-3)
    assert y["impulse"] == pytest.approx(J0, rel=1e-3)
    for k, name in enumerate(TANGENT_PARAMS):
        hi, lo = dict(p), dict(p)
        hi[name] = p[name] * (1.0 + 1e-4)
        lo[name] = p[name] * (1.0 - 1e-4)
        (ph, jh), (pl, jl) = orc(hi), orc(lo)
        dP, dJ = (ph - pl) / 2e-4, (jh - jl) / 2e-4
        print("ADJFD %s dP adj %.6g fd %.6g | dJ adj %.6g fd %.6g"
              % (name, d["dpeak"][k], dP, d["dimpulse"][k], dJ))
        assert abs(d["dpeak"][k] - dP) <= 0.02 * abs(dP) + 1e-6 * y["peak"], name
        assert abs(d["dimpulse"][k] - dJ) <= 0.02 * abs(dJ) + 1e-6 * y["impulse"], name


def test_autograd_reverse_mode():
    p, xy = case0()
    theta = torch.tensor([p[k] for k in TANGENT_PARAMS], dtype=torch.float64,
                         requires_grad=True)
    y = peak_and_impulse(theta, p, xy, 60)
    y0, J = jacobian(theta.detach().numpy(), p, xy, 60)
    yt, Jt = jacobian(theta.detach().numpy(), p, xy, 60, mode="tangent")
    assert np.array_equal(y.detach().numpy(), y0) and np.array_equal(y0, yt)
    (y[0] + 2.0 * y[1]).backward()
    assert np.allclose(theta.grad.numpy(), J[0] + 2.0 * J[1], rtol=1e-12, atol=0.0)
    assert np.allclose(J, Jt, rtol=1e-4, atol=1e-7 * np.abs(y0)[:, None])


def test_reverse_mode_refusals():
    p, xy = case0()
    for kw in (dict(dt_mode=0), dict(motion=3), dict(closure=1, c0=1448.0),
               dict(cell_factor=0.5)):
        with Case(dict(p, **kw), xy) as c:
            with pytest.raises(HramError) as e:
                c.adjoint_forward(10)
            assert e.value.code == _lib.HR_EINVAL
    with Case(p, xy, tangent=True) as c:
        with pytest.raises(HramError):
            c.adjoint_forward(10)
    with Case(p, xy) as c:
        with pytest.raises(HramError):
            c.adjoint_backward()          # no forward run yet
        c.run(3)
        with pytest.raises(HramError):
            c.adjoint_forward(10)         # not at the uploaded state
    with Case(p, xy, probe_capacity=8) as c:
        with pytest.raises(HramError):
            c.adjoint_forward(10)         # history shorter than the run
