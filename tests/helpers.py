"""Shared set-up of the GPU parity tests: the same seeded inputs for the CUDA
path and the oracle (positions rounded once to float32 and given to both)."""
import numpy as np

import casegen


def impact_case(p=None, **kw):
    p = dict(p or casegen.config_parity())
    p.update(kw)
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                               disk=(p["x_c0"], p["y_c0"], p["R_disk"]) if p["Ng"] > 0 else None)
    return p, xy.astype(np.float32)


def perturbed(p, xy32, seed=11, v_amp=20.0, rho_rel=0.01):
    vel, rho = casegen.perturbed_state(xy32.shape[0], seed, v_amp, p["rho0"], rho_rel)
    return vel.astype(np.float32), rho.astype(np.float32)


def as64(a):
    return None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) /
                 max(np.linalg.norm(np.asarray(b, float)), 1e-300))


def csr_equal(off1, ids1, off2, ids2):
    return np.array_equal(off1, off2) and np.array_equal(ids1, ids2)


FP32_EPS = 2.0 ** -24

# Multiple of the rounding floor that the one-step pressure gate allows: the
# floor is the pressure that one float32 rounding of one position is worth
# (below), and a particle's density sums about 20 neighbours' terms.
K_P = 8.0


def local_speed(o, fo):
    """V_i: the largest speed over particle i and its neighbours (fluid and
    ghosts) in the FP64 reference case o, whose fluid arrays are fo."""
    off, ids = o.neighbours()
    nf = fo["vel"].shape[0]
    speed = np.concatenate([np.hypot(fo["vel"][:, 0], fo["vel"][:, 1]),
                            np.hypot(*o.ghosts()["vel"].T)])
    V = speed[:nf].copy()
    rows = np.diff(off[:nf + 1])
    nz = rows > 0
    if ids.size:
        m = np.maximum.reduceat(speed[ids], off[:nf][nz])
        V[nz] = np.maximum(V[nz], m)
    return V


def p_floor(p, fo, dt, steps=1, V=None):
    """Per-particle pressure resolution of a float32 state after `steps`
    steps, against an FP64 reference state fo (oracle fluid arrays).

    A position r carries a rounding of 2^-24 |r| (|r| up to the particle's
    own coordinate plus the support 2h), which moves kernel values and
    gradients by 2^-24 |r| / h relative.  With the continuity equation
    (closure 0) each term m_j v_ij . grad W_ij of the density rate moves by
    that relative amount; the terms add up to at most (7/3) (2 V_i) / h in
    units of the density deviation per second (sum_j (m_j / rho0) |grad W_ij|
    is the kernel's integral of |dW/dr|, 7 / (3 h) for Wendland C2, and
    |v_ij| <= 2 V_i with V_i the largest speed in the support), so the
    density deviation moves by dt times that in a step.  With the summed
    density (closure 1) the density moves by the relative amount itself.
    The pressure moves by dp/drho = c^2 times the density: c0^2 (rho /
    rho0)^(gamma - 1) for Tait, C^2 for Mie-Grueneisen near rho0."""
    h = p["h_over_dx"] * p["dx"]
    reach = (np.abs(fo["xy"]).max(axis=1) + 2.0 * h) / h
    dens = np.maximum(fo["rho"] / p["rho0"], 1.0)
    if p.get("closure", 0) == 1:
        stiff = p["rho0"] * p["c0"] ** 2 * dens ** 2
        moved = 1.0
    else:
        stiff = p["rho0"] * p["c0"] ** 2 * dens ** (p["gamma"] - 1.0)
        moved = dt * (7.0 / 3.0) * 2.0 * V / h
    return steps * stiff * FP32_EPS * reach * moved


def assert_p_close(name, p, p_gpu, o, dt, steps=1, rel=1e-5):
    """The one-step pressure gate against the FP64 reference case o:
    |p_gpu - p_ref| <= rel max|p_ref| plus K_P times the per-particle
    rounding floor of p_floor (reading R26)."""
    fo = o.fluid()
    err = np.abs(np.asarray(p_gpu, float) - fo["p"])
    base = rel * np.abs(fo["p"]).max()
    V = None if p.get("closure", 0) == 1 else local_speed(o, fo)
    floor = p_floor(p, fo, dt, steps, V)
    ratio = float((err / (base + floor)).max())
    print("GATE %s: max|dp| %.3g Pa, rel part %.3g Pa, max floor %.3g Pa, err/(rel+floor) %.3g"
          % (name, err.max(), base, floor.max(), ratio))
    assert np.all(err <= base + K_P * floor), (name, ratio)
