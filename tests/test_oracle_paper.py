"""Pins of the oracle's paper closure (closure 1): the cubic B-spline kernel,
the summation density, the Mie-Grueneisen equation of state and the
internal-energy equation, each against what the paper and the mathematics
fix -- quadrature, the Rankine-Hugoniot jump conditions, brute-force sums and
exact conservation -- with planted mistakes showing that the pins bite."""
import math

import numpy as np
import pytest
from scipy import integrate

import casegen
import oracle

H = 1.3e-3


def paper_params(**kw):
    p = casegen.base_params()
    p.update(closure=1, c0=1448.0, alpha=0.03, cfl=0.25)
    p.update(kw)
    return p


# ------------------------------------------------------------------ kernel

def test_cubic_kernel_normalised_in_two_dimensions():
    # eq. cubic-kernel: integral of W over the plane is 1 (sigma = 10/(7 pi h^2))
    f = lambda r: oracle.cubic_W(r, H) * 2.0 * math.pi * r
    a, _ = integrate.quad(f, 0.0, H, epsabs=1e-14)
    b, _ = integrate.quad(f, H, 2.0 * H, epsabs=1e-14)
    assert a + b == pytest.approx(1.0, abs=1e-10)


def test_cubic_kernel_support_and_smoothness():
    assert oracle.cubic_W(2.0 * H, H) == 0.0
    assert oracle.cubic_W(2.0 * H * 1.0001, H) == 0.0
    # W and dW/dr continuous at q = 1 (the spline's knot)
    e = 1e-9 * H
    assert oracle.cubic_W(H - e, H) == pytest.approx(oracle.cubic_W(H + e, H), rel=1e-7)
    assert (oracle.cubic_F(H - e, H) * (H - e) ==
            pytest.approx(oracle.cubic_F(H + e, H) * (H + e), rel=1e-6))
    # F r = dW/dr by central differences across both pieces
    for q in (0.1, 0.5, 0.9, 1.2, 1.7, 1.95):
        r, d = q * H, 1e-7 * H
        dW = (oracle.cubic_W(r + d, H) - oracle.cubic_W(r - d, H)) / (2 * d)
        assert oracle.cubic_F(r, H) * r == pytest.approx(dW, rel=1e-6)


# ------------------------------------------------------- summation density

def lattice_case(**kw):
    p = paper_params(Ng=0, wall_layers=0, Lx=0.04, W=0.04, dx=1e-3, gy=0.0)
    p.update(kw)
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], 0.0, 1, disk=None)
    return p, xy


def test_summation_density_equals_brute_force_lattice_sum():
    # eq. density-sum on an unperturbed lattice: an interior particle's
    # density is the brute-force sum of m W over every particle (itself
    # included)
    p, xy = lattice_case(mutation=0)
    o = oracle.OracleCase(p, xy)
    rho = o.fluid()["rho"]
    i = int(np.argmin(np.hypot(xy[:, 0] - 0.02, xy[:, 1])))
    h = p["h_over_dx"] * p["dx"]
    m = p["rho0"] * p["dx"] ** 2
    r = np.hypot(xy[:, 0] - xy[i, 0], xy[:, 1] - xy[i, 1])
    brute = m * sum(oracle.cubic_W(float(x), h) for x in r)
    assert rho[i] == pytest.approx(brute, rel=1e-12)
    # the lattice sum is within 1e-4 of rho0 at h = 1.3 dx
    assert abs(rho[i] / p["rho0"] - 1.0) < 1e-4


def test_summation_density_planted_mistake_drops_self():
    p, xy = lattice_case()
    good = oracle.OracleCase(p, xy).fluid()["rho"]
    bad = oracle.OracleCase(p, xy, mutation=oracle.MUT["sum_no_self"]).fluid()["rho"]
    i = int(np.argmin(np.hypot(xy[:, 0] - 0.02, xy[:, 1])))
    assert abs(bad[i] / good[i] - 1.0) > 0.2


def test_wall_ghosts_complete_the_summed_density():
    # ghost layers continue the lattice across the wall: rows next to the
    # wall get the interior density; without them the first row sags
    p, xy = lattice_case(wall_layers=3)
    rho = oracle.OracleCase(p, xy).fluid()["rho"]
    x, y = xy[:, 0], xy[:, 1]
    mid = np.abs(x - 0.02) < 0.004
    interior = rho[mid & (np.abs(y) < 0.005)]
    near_wall = rho[mid & (np.abs(y) > 0.017)]
    assert np.allclose(near_wall, interior.mean(), rtol=1e-12)
    q, _ = lattice_case(wall_layers=0)
    free = oracle.OracleCase(q, xy).fluid()["rho"]
    first_row = free[mid & (y > 0.019)]
    assert np.all(first_row < 0.8 * p["rho0"])


# ------------------------------------------------------ Mie-Grueneisen EOS

def hugoniot(p, up):
    """Linear Us-Up Hugoniot of water from the jump conditions, shock into
    water at rest: Us = C + S1 up, p = rho0 Us up, rho0 Us = rho (Us - up),
    e = up^2 / 2."""
    C, S1, rho0 = p["c0"], p["mg_S1"], p["rho0"]
    us = C + S1 * up
    rho = rho0 * us / (us - up)
    return rho, rho0 * us * up, 0.5 * up * up


def test_mg_reproduces_the_shock_hugoniot_to_second_order():
    # eq. eos has the linear Us-Up Hugoniot as its reference: on the
    # Hugoniot states (rho_H, e_H) it returns p_H up to O(mu^3)
    p = paper_params(p_cav=-1e12)
    rel = []
    for up in (2.0, 5.0, 10.0, 20.0, 40.0):
        rho, pH, eH = hugoniot(p, up)
        mu = rho / p["rho0"] - 1.0
        err = (oracle.mg_p(p, rho, eH) - pH) / pH
        rel.append((mu, err))
        assert abs(err) < 2.0 * mu * mu
    # and the error does scale as mu^2 (not as mu): a wrong first-order
    # coefficient would break this
    (m1, e1), (m2, e2) = rel[1], rel[-1]
    assert abs(e2 / e1) == pytest.approx((m2 / m1) ** 2, rel=0.25)


def test_mg_branches_bulk_modulus_cap_and_cutoff():
    p = paper_params(p_cav=-1e12)
    rho0, C = p["rho0"], p["c0"]
    # the two branches meet at mu = 0 (a jump there would show up as a gap
    # far above the 2e-12 rho0 C^2 that the density step itself makes)
    for e in (0.0, 500.0):
        gap = oracle.mg_p(p, rho0 * (1 + 1e-12), e) - oracle.mg_p(p, rho0 * (1 - 1e-12), e)
        assert abs(gap) <= 1e-11 * rho0 * C * C
    # dp/drho = C^2 at rho0 from both sides (C is the bulk sound speed)
    d = 1e-7 * rho0
    up = (oracle.mg_p(p, rho0 + d, 0.0) - oracle.mg_p(p, rho0, 0.0)) / d
    dn = (oracle.mg_p(p, rho0, 0.0) - oracle.mg_p(p, rho0 - d, 0.0)) / d
    assert up == pytest.approx(C * C, rel=1e-5) and dn == pytest.approx(C * C, rel=1e-5)
    # compression cap mu <= 0.25
    assert oracle.mg_p(p, 1.40 * rho0, 300.0) == oracle.mg_p(p, 1.25 * rho0, 300.0)
    # cavitation cutoff
    q = paper_params()
    assert oracle.mg_p(q, 0.9 * rho0, 0.0) == q["p_cav"]
    # monotone in density below the cap
    rs = np.linspace(0.99, 1.25, 200) * rho0
    ps = [oracle.mg_p(p, r, 100.0) for r in rs]
    assert np.all(np.diff(ps) > 0)


# ----------------------------------------------- internal-energy equation

def energy_patch(mutation=0, cfl=0.2, steps=120):
    """A free patch (no walls, disk or gravity), random velocities, artificial
    viscosity on, no XSPH or laminar term, no cutoff, soft water (C = 30 m/s)."""
    p = paper_params(Ng=0, wall_layers=0, Lx=0.03, W=0.03, dx=1e-3, gx=0.0, gy=0.0,
                     c0=30.0, v0=0.0, p_cav=-1e12, alpha=0.1, eps_xsph=0.0, mu_lam=0.0,
                     dt_mode=1, cfl=cfl, box_pad=1.0)
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], 0.01, 3, disk=None)
    vel, _ = casegen.perturbed_state(xy.shape[0], 5, 3.0, p["rho0"], 0.0)
    o = oracle.OracleCase(p, xy, vel=vel, mutation=mutation)

    def total():
        d = o.diagnostics()
        return d["KE"] + d["E_el"], d["KE"]

    E0, KE0 = total()
    o.run(int(steps))
    E1, KE1 = total()
    return E0, E1, KE0, KE1, o


def test_energy_equation_conserves_total_energy():
    # KE + sum m e is conserved by the pair terms for any equation of state;
    # what is left is the time-stepping error of the step.  The patch's free
    # surfaces collapse violently (summation density sags there), so the
    # check is a bound at two step sizes rather than a convergence rate.
    for cfl, steps in ((0.1, 240), (0.05, 480)):
        E0, E1, KE0, KE1, o = energy_patch(cfl=cfl, steps=steps)
        assert o.diagnostics()["dissipation"] > 0.5 * KE0   # AV did work
        assert abs(KE1 - KE0) > 0.3 * KE0                   # energy changed form
        assert abs(E1 - E0) / KE0 < 2e-3, cfl


def test_energy_equation_planted_mistake():
    E0, E1, KE0, _, _ = energy_patch(mutation=oracle.MUT["energy_half"], cfl=0.1, steps=240)
    assert abs(E1 - E0) / KE0 > 0.05


def test_paper_closure_momentum_and_galilean_invariance():
    p, xy = lattice_case(Lx=0.02, W=0.02)
    vel, _ = casegen.perturbed_state(xy.shape[0], 7, 10.0, p["rho0"], 0.0)
    o = oracle.OracleCase(p, xy, vel=vel)
    f = o.fluid()
    m = p["rho0"] * p["dx"] ** 2
    # sum m a = 0 for a free patch (no gravity, no ghosts)
    assert np.abs((m * f["acc"]).sum(axis=0)).max() <= 1e-10 * np.abs(m * f["acc"]).sum()
    shift = np.array([37.0, -12.0])
    o2 = oracle.OracleCase(p, xy, vel=vel + shift)
    f2 = o2.fluid()
    assert np.allclose(f2["acc"], f["acc"], rtol=1e-9, atol=1e-9 * np.abs(f["acc"]).max())
    e1, e2 = o.energy(), o2.energy()
    assert np.allclose(e2["de"], e1["de"], rtol=1e-9, atol=1e-9 * np.abs(e1["de"]).max())


def test_hard_reflection_wall_keeps_particles_in_the_channel():
    # the paper's baseline wall (Section "The Channel Walls"): no ghosts, a
    # particle crossing |y| = W/2 is put back inside and its normal velocity
    # reversed; it carries no pressure, so no wall impulse is recorded
    p = paper_params(wall_layers=0, wall_reflect=1, Lx=0.04, W=0.02, dx=1e-3, Ng=0,
                     gy=0.0, box_pad=0.05)
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], 0.01, 9, disk=None)
    vel = np.zeros_like(xy)
    vel[:, 1] = np.where(xy[:, 1] > 0, 40.0, -40.0)     # everything pushed at the walls
    o = oracle.OracleCase(p, xy, vel=vel)
    o.run(60)
    f = o.fluid()
    assert np.all(np.abs(f["xy"][:, 1]) <= 0.5 * p["W"])
    assert o.scalars()["wall_impulse"] == 0.0 and o.ngh == 0
    q = dict(p, wall_reflect=0)
    o2 = oracle.OracleCase(q, xy, vel=vel)
    o2.run(60)
    assert np.any(np.abs(o2.fluid()["xy"][:, 1]) > 0.5 * p["W"])
