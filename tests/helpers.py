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


def p_scale(p, p_ref):
    """Pressure scale of the one-step gate "pressure within 1e-5 relative":
    the larger of max |p_ref| and the EOS stiffness rho0 c0^2.  p = B((rho /
    rho0)^gamma - 1) maps the density gate (1e-5 relative) onto 1e-5 rho0 c0^2;
    near rest max |p| is far below that and p is a cancellation."""
    return max(float(np.abs(p_ref).max()), p["rho0"] * p["c0"] ** 2)
