"""PyTorch autograd bridge of the tangent-linear mode.

``peak_and_impulse(theta, params, xy, n_steps)`` runs one case on the GPU with
the library's tangent kernels (flag HR_FLAG_TANGENT) and returns the peak
probe-0 pressure and the wall impulse as a tensor of two values whose
gradient with respect to theta = (alpha, c0, tau) is the library's exact
derivative of the discrete run: the artificial-viscosity coefficient of eq.
artificial-viscosity, the reference sound speed of the Tait equation of state
(which also sets the fixed step dt = C h / (c0 + v0)) and the decay time of
the prescribed disk motion.  With three parameters and two outputs the
forward (tangent) mode costs one run whatever the number of outputs asked
for; backward() only contracts the stored 2 x 3 Jacobian.
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


def jacobian(theta, params: dict, xy, n_steps: int, vel=None, rho=None, stream=None):
    """(outputs [peak, impulse], J) with J[i, k] = d output_i / d theta_k."""
    th = np.asarray(theta, dtype=np.float64)
    if np.any(th == 0.0):
        # the library differentiates along theta_k d/dtheta_k; at theta_k = 0
        # that direction is zero and the absolute derivative is not recoverable
        raise ValueError("jacobian: every parameter (alpha, c0, tau) must be nonzero, got %s"
                         % (th.tolist(),))
    o = _run(th, params, xy, n_steps, vel, rho, stream)
    rel = np.stack([o["dpeak"], o["dimpulse"]])
    # relative derivatives theta_k d/dtheta_k -> absolute
    return np.array([o["peak"], o["impulse"]]), rel / th


def _function():
    import torch

    class PeakImpulse(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, params, xy, n_steps, vel, rho):
            y, J = jacobian(theta.detach().cpu().numpy(), params, xy, n_steps, vel, rho)
            ctx.save_for_backward(torch.as_tensor(J, dtype=theta.dtype, device=theta.device))
            return torch.as_tensor(y, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, g):
            (J,) = ctx.saved_tensors
            return g @ J, None, None, None, None, None

    return PeakImpulse


_PeakImpulse = None


def peak_and_impulse(theta, params: dict, xy, n_steps: int, vel=None, rho=None):
    """Differentiable [peak probe-0 pressure, wall impulse] of a run of
    n_steps steps; theta is a tensor (alpha, c0, tau)."""
    global _PeakImpulse
    if _PeakImpulse is None:
        _PeakImpulse = _function()
    return _PeakImpulse.apply(theta, params, xy, n_steps, vel, rho)
