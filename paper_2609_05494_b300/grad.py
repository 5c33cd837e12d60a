"""PyTorch autograd bridge of the library's derivatives.

``peak_and_impulse(theta, params, xy, n_steps)`` runs one case on the GPU and
returns the peak probe-0 pressure and the wall impulse as a tensor of two
values whose gradient with respect to theta = (alpha, c0, tau) is the
library's exact derivative of the discrete run: the artificial-viscosity
coefficient of eq. artificial-viscosity, the reference sound speed of the
Tait equation of state (which also sets the fixed step dt = C h / (c0 + v0))
and the decay time of the prescribed disk motion.

mode="adjoint" (the default) is reverse mode: forward() runs the case with a
checkpoint every ``checkpoint_every`` steps (hr_adjoint_forward), backward()
sweeps the run backwards, recomputing each segment from its checkpoint
(hr_adjoint_backward), and contracts the incoming gradient with the 2 x 3
Jacobian it returns.  mode="tangent" is forward mode: one run carrying the
three directional derivatives (flag HR_FLAG_TANGENT); backward() only
contracts the stored Jacobian.  The two give the same Jacobian (the same
discrete derivative, evaluated in a different order).
"""
from __future__ import annotations

import numpy as np

from .api import TANGENT_PARAMS, Case


def _run(theta: np.ndarray, params: dict, xy, n_steps: int, vel=None, rho=None, stream=None):
    q = dict(params)
    for name, v in zip(TANGENT_PARAMS, theta):
        q[name] = float(v)
    with Case(q, xy, vel, rho, stream=stream, tangent=True) as c:
        c.run(int(n_steps))
        c.sync()
        return c.tangent_outputs()


def _params_at(theta: np.ndarray, params: dict) -> dict:
    q = dict(params)
    for name, v in zip(TANGENT_PARAMS, theta):
        q[name] = float(v)
    return q


def _check_theta(theta) -> np.ndarray:
    th = np.asarray(theta, dtype=np.float64)
    if np.any(th == 0.0):
        # the library differentiates along theta_k d/dtheta_k; at theta_k = 0
        # that direction is zero and the absolute derivative is not recoverable
        raise ValueError("jacobian: every parameter (alpha, c0, tau) must be nonzero, got %s"
                         % (th.tolist(),))
    return th


def jacobian(theta, params: dict, xy, n_steps: int, vel=None, rho=None, stream=None,
             mode: str = "adjoint", checkpoint_every: int = 20):
    """(outputs [peak, impulse], J) with J[i, k] = d output_i / d theta_k,
    by reverse mode (mode="adjoint") or forward mode (mode="tangent")."""
    th = _check_theta(theta)
    if mode == "tangent":
        o = _run(th, params, xy, n_steps, vel, rho, stream)
        rel = np.stack([o["dpeak"], o["dimpulse"]])
        # relative derivatives theta_k d/dtheta_k -> absolute
        return np.array([o["peak"], o["impulse"]]), rel / th
    if mode != "adjoint":
        raise ValueError("mode must be 'adjoint' or 'tangent'")
    with Case(_params_at(th, params), xy, vel, rho, stream=stream) as c:
        y = c.adjoint_forward(int(n_steps), checkpoint_every)
        g = c.adjoint_backward()
    rel = np.stack([g["dpeak"], g["dimpulse"]])
    return np.array([y["peak"], y["impulse"]]), rel / th


def _functions():
    import torch

    class PeakImpulseTangent(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, params, xy, n_steps, vel, rho, every):
            y, J = jacobian(theta.detach().cpu().numpy(), params, xy, n_steps, vel, rho,
                            mode="tangent")
            ctx.save_for_backward(torch.as_tensor(J, dtype=theta.dtype, device=theta.device))
            return torch.as_tensor(y, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, g):
            (J,) = ctx.saved_tensors
            return g @ J, None, None, None, None, None, None

    class PeakImpulseAdjoint(torch.autograd.Function):
        # forward: the run with its checkpoints; backward: the reverse sweep
        @staticmethod
        def forward(ctx, theta, params, xy, n_steps, vel, rho, every):
            th = _check_theta(theta.detach().cpu().numpy())
            case = Case(_params_at(th, params), xy, vel, rho)
            y = case.adjoint_forward(int(n_steps), int(every))
            ctx.case, ctx.theta = case, th
            return torch.tensor([y["peak"], y["impulse"]], dtype=theta.dtype,
                                device=theta.device)

        @staticmethod
        def backward(ctx, g):
            case = ctx.case
            try:
                d = case.adjoint_backward()
            finally:
                case.close()
                ctx.case = None
            J = np.stack([d["dpeak"], d["dimpulse"]]) / ctx.theta
            Jt = torch.as_tensor(J, dtype=g.dtype, device=g.device)
            return g @ Jt, None, None, None, None, None, None

    return {"tangent": PeakImpulseTangent, "adjoint": PeakImpulseAdjoint}


_FUNCS = None


def peak_and_impulse(theta, params: dict, xy, n_steps: int, vel=None, rho=None,
                     mode: str = "adjoint", checkpoint_every: int = 20):
    """Differentiable [peak probe-0 pressure, wall impulse] of a run of
    n_steps steps; theta is a tensor (alpha, c0, tau)."""
    global _FUNCS
    if _FUNCS is None:
        _FUNCS = _functions()
    if mode not in _FUNCS:
        raise ValueError("mode must be 'adjoint' or 'tangent'")
    return _FUNCS[mode].apply(theta, params, xy, n_steps, vel, rho, checkpoint_every)
