"""Seeded synthetic inputs for the planar WCSPH hydrodynamic-ram pass.

This module is the one place that both the FP64 oracle (``oracle/``) and the
CUDA path (``paper_2609_05494_b300``) take their inputs from.  It holds none of
the method's arithmetic: no kernel, no equation of state, no ghost operator,
no integrator.  It only

* lays out the initial fluid lattice of the channel (Section "Validation
  Problem Setup": particles seeded on a Cartesian lattice at spacing dx, the
  ones inside the projectile disk removed),
* draws the +-jitter of that lattice from SplitMix64 (Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014),
* names the parameter sets of the workloads (values only), and
* makes seeded perturbed states used as parity inputs.

Conventions shared by every caller (SI units):
  fluid x in [0, Lx], y in [-W/2, W/2]; lattice point (i, j) sits at
  ((i + 1/2) dx, -W/2 + (j + 1/2) dx); fluid IDs run row-major, j (y) outer,
  i (x) inner, over the points that survive the disk removal.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "GOLDEN_GAMMA",
    "splitmix64",
    "uniform53",
    "fluid_lattice",
    "perturbed_state",
    "base_params",
    "config_parity",
    "config_production",
    "config_scaling",
    "config_adjoint",
    "sweep_draws",
    "DEFAULT_SEED",
]

DEFAULT_SEED = 20260905
GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray | int) -> np.ndarray:
    """Output number ``index`` (0-based) of the SplitMix64 stream seeded by ``seed``.

    SplitMix64 is counter based: state_k = seed + (k + 1) * GOLDEN_GAMMA (mod
    2^64), then the published 64-bit finaliser (xor-shift 30, multiply, xor-shift
    27, multiply, xor-shift 31).
    """
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform53(seed: int, index: np.ndarray | int) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits of SplitMix64 output ``index``."""
    z = splitmix64(seed, index)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def fluid_lattice(Lx: float, W: float, dx: float, jitter: float = 0.01,
                  seed: int = DEFAULT_SEED, disk: tuple[float, float, float] | None = None
                  ) -> np.ndarray:
    """Initial fluid positions, float64 array of shape (N, 2), in fluid-ID order.

    Lattice point L = j * nx + i draws jitter from SplitMix64 outputs 2L (x) and
    2L + 1 (y): delta = (2u - 1) * jitter * dx.  ``disk`` = (xc, yc, R) removes
    the points strictly inside that circle (after jitter).  IDs are assigned to
    the survivors in lattice order.
    """
    nx = int(round(Lx / dx))
    ny = int(round(W / dx))
    if nx <= 0 or ny <= 0:
        raise ValueError("empty lattice")
    j, i = np.meshgrid(np.arange(ny, dtype=np.int64), np.arange(nx, dtype=np.int64), indexing="ij")
    lat = (j * nx + i).reshape(-1)
    x = (i.reshape(-1) + 0.5) * dx
    y = -0.5 * W + (j.reshape(-1) + 0.5) * dx
    if jitter != 0.0:
        ux = uniform53(seed, 2 * lat)
        uy = uniform53(seed, 2 * lat + 1)
        x = x + (2.0 * ux - 1.0) * jitter * dx
        y = y + (2.0 * uy - 1.0) * jitter * dx
    xy = np.stack([x, y], axis=1)
    if disk is not None:
        xc, yc, R = disk
        keep = (x - xc) ** 2 + (y - yc) ** 2 >= R * R
        xy = xy[keep]
    return np.ascontiguousarray(xy)


def perturbed_state(n: int, seed: int, v_amp: float, rho0: float, rho_rel: float
                    ) -> tuple[np.ndarray, np.ndarray]:
    """Seeded velocities (N, 2) uniform in [-v_amp, v_amp] and densities uniform
    in rho0 * [1 - rho_rel, 1 + rho_rel].  Uses SplitMix64 outputs from a stream
    offset by 2^40 so it never overlaps the lattice jitter draws."""
    base = np.uint64(1) << np.uint64(40)
    k = np.arange(3 * n, dtype=np.uint64) + base
    u = uniform53(seed, k).reshape(n, 3)
    vel = (2.0 * u[:, :2] - 1.0) * v_amp
    rho = rho0 * (1.0 + (2.0 * u[:, 2] - 1.0) * rho_rel)
    return np.ascontiguousarray(vel), np.ascontiguousarray(rho)


def base_params() -> dict:
    """Physical and numerical constants common to the workloads.

    Tait water (gamma 7, rho0 1000 kg/m^3, c0 1480 m/s), cavitation cutoff
    -0.1 MPa, Monaghan artificial viscosity alpha 0.02 with eta^2 0.01 (the
    paper's alpha is 0.03; the workloads use 0.02), XSPH epsilon 0.02, water
    dynamic viscosity 8.9e-4 Pa s, gravity (0, -9.81) m/s^2, CFL 0.2, h = 1.3 dx,
    3 ghost layers per side wall, a 5 mm disk entering at the mid-height of the
    x = 0 face with a 5 us ramp and exponential deceleration tau = 200 us;
    disk density 7850 kg/m^3 (steel) for the two-way coupled motion.
    closure 0 selects the workloads' closure (Wendland, continuity, Tait);
    closure 1 the paper's (cubic B-spline, summation density, Mie-Grueneisen
    water with S1 1.979, gamma0 0.11, a 3.0, compression cap mu <= 0.25).
    """
    return dict(
        dx=2e-3, h_over_dx=1.3, Lx=0.150, W=0.150,
        wall_layers=3, end_walls=0,
        R_disk=5e-3, v0=900.0, tau=200e-6, t_ramp=5e-6, x_c0=-5e-3, y_c0=0.0,
        Ng=100, motion=0, a_const=0.0, drag_M=8.01e-3, drag_Cd=0.05, drag_R=6.25e-3,
        rho0=1000.0, c0=1480.0, gamma=7.0, p_cav=-1e5, alpha=0.02, eta2=0.01,
        eps_xsph=0.02, mu_lam=8.9e-4, gx=0.0, gy=-9.81, cfl=0.2, dt_mode=0,
        rho_lo=0.5, rho_hi=1.5, box_pad=-1.0, cell_factor=1.001,
        seed=DEFAULT_SEED, jitter=0.01, disk_density=7850.0,
        closure=0, mg_S1=1.979, mg_gamma0=0.11, mg_a=3.0, mg_mu_max=0.25, wall_reflect=0,
        probes=[],
    )


def _wall_probes(W: float, xs) -> list:
    return [(float(x), 0.5 * W) for x in xs]


def config_parity() -> dict:
    """150 x 150 mm channel, dx = 2 mm (5,625 fluid particles), 250 steps."""
    p = base_params()
    p.update(dx=2e-3, Lx=0.150, W=0.150)
    p["probes"] = _wall_probes(p["W"], (0.030, 0.060, 0.090, 0.120))
    p["n_steps"] = 250
    return p


def config_production(v0: float = 900.0) -> dict:
    """300 x 150 mm channel, dx = 0.5 mm (180,000 fluid particles), 1 ms."""
    p = base_params()
    p.update(dx=5e-4, Lx=0.300, W=0.150, v0=float(v0))
    p["probes"] = _wall_probes(p["W"], (0.030, 0.105, 0.180, 0.255))
    p["t_end"] = 1e-3
    return p


def config_scaling(dx: float) -> dict:
    """300 x 150 mm channel at spacing dx (dx = 0.2 mm gives 1,125,000 particles)."""
    p = config_production(900.0)
    p.update(dx=float(dx))
    p.pop("t_end")
    return p


def config_paper(v0: float = 900.0) -> dict:
    """The paper's own set-up (closure 1): a 750 x 150 mm channel at dx = 1.5 mm
    (500 x 100 lattice points before the disk interior is removed), a
    12.5 mm disk entering on the centreline at v0 with the 5 us ramp and then
    the quadratic drag law (M = 8.01 g, Cd = 0.05, R = 6.25 mm), water with
    C = c0 = 1448 m/s, alpha 0.03, CFL 0.25, and the probes PTn and PTf on the
    centreline at x = 30 and 105 mm; the 150 us event of the paper's timing."""
    p = base_params()
    p.update(dx=1.5e-3, Lx=0.750, W=0.150, R_disk=6.25e-3, x_c0=-6.25e-3, v0=float(v0),
             motion=1, c0=1448.0, alpha=0.03, cfl=0.25, closure=1)
    p["probes"] = [(0.030, 0.0), (0.105, 0.0)]
    p["t_end"] = 150e-6
    return p


def config_adjoint() -> dict:
    """150 x 150 mm channel at dx = 1 mm (22,500 particles), 400 steps, fixed dt."""
    p = config_parity()
    p.update(dx=1e-3, dt_mode=1)
    p["n_steps"] = 400
    return p


def sweep_draws(seed: int, n_cases: int) -> list[dict]:
    """Per-case coefficient draws of the batched sweep: alpha ~ U[0.01, 0.1],
    c0 ~ {1480, 740, 370}, p_cav ~ U[-1e6, 0], v0 ~ U[600, 900], W ~ U[100, 200] mm,
    Lx = 1.5 W, dx = 1 mm.  Case k uses the SplitMix64 stream seeded with
    seed XOR k, outputs 0..4 in that order."""
    out = []
    for k in range(n_cases):
        s = (seed ^ k) & 0xFFFFFFFFFFFFFFFF
        u = uniform53(s, np.arange(5, dtype=np.uint64))
        p = config_parity()
        W = 0.100 + 0.100 * float(u[4])
        W = round(W / 1e-3) * 1e-3
        p.update(
            dx=1e-3,
            alpha=0.01 + 0.09 * float(u[0]),
            c0=(1480.0, 740.0, 370.0)[min(int(u[1] * 3.0), 2)],
            p_cav=-1e6 * float(u[2]),
            v0=600.0 + 300.0 * float(u[3]),
            W=W, Lx=round(1.5 * W / 1e-3) * 1e-3,
        )
        p["probes"] = _wall_probes(W, (0.030, 0.060))
        p["t_end"] = 0.5e-3
        out.append(p)
    return out


def n_lattice(Lx: float, W: float, dx: float) -> int:
    return int(round(Lx / dx)) * int(round(W / dx))


def describe(p: dict) -> str:
    return "Lx=%g mm W=%g mm dx=%g mm N~%d" % (p["Lx"] * 1e3, p["W"] * 1e3, p["dx"] * 1e3,
                                                n_lattice(p["Lx"], p["W"], p["dx"]))

