"""Differentiable sphere-averaged scalar signal (torch.autograd.Function over grf_tlm_rk4).

theta = (lambda, g2, A): the Gauss-Bonnet coupling, the X^2 coupling and the amplitude of the
initial scalar profile. The caller supplies the initial state at the current A together with
its derivative with respect to A (for phi = A f(x) that is the state with phi = f and every
other field zero). The forward pass runs the tangent-linear evolution (value and the three
derivatives together, in one pass over the steps) and keeps dL/dtheta for backward.
"""
from __future__ import annotations

import torch

from . import (alloc_state, alloc_workspace, grf_params, grf_sphere, grf_tlm_rk4, grf_tlm_workspace_bytes)


def _with_couplings(params: grf_params, lam, g2) -> grf_params:
    p = grf_params()
    C_fields = [f[0] for f in grf_params._fields_]
    for name in C_fields:
        setattr(p, name, getattr(params, name))
    p.lambda_ = float(lam)
    p.g2 = float(g2)
    return p


def sphere_signal_and_grad(box, params, theta, state0, dstate0_dA, dt, nsteps, sphere, stream=None):
    """Returns (L, dL/dtheta) as Python floats / a 3-element tensor (float64, CPU). theta holds
    (lambda, g2, A); pass it in float64 (a float32 theta would round the couplings)."""
    if hasattr(theta, "dtype") and str(theta.dtype) not in ("torch.float64",):
        raise TypeError("theta must be float64")
    lam, g2, _ = (float(x) for x in theta)
    p = _with_couplings(params, lam, g2)
    state = state0.clone()
    tang = alloc_state(box, 27 * 3)
    # direction 2: d/dA (the state's derivative); directions 0, 1: d/d lambda, d/d g2 (zero state tangent)
    tang.view(3, -1)[2].copy_(dstate0_dA.reshape(-1))
    loss = torch.zeros(4, dtype=torch.float64, device=state0.device)
    ws = alloc_workspace(grf_tlm_workspace_bytes(box))
    grf_tlm_rk4(box, p, [1.0, 0.0, 0.0, 1.0, 0.0, 0.0], state, tang, dt, nsteps, sphere, loss, ws=ws, stream=stream)
    out = loss.cpu()
    return float(out[0]), out[1:4].clone()


class SphereSignal(torch.autograd.Function):
    """L(theta) with theta = (lambda, g2, A); backward returns grad_out * dL/dtheta."""

    @staticmethod
    def forward(ctx, theta, box, params, state0, dstate0_dA, dt, nsteps, sphere):
        L, grad = sphere_signal_and_grad(box, params, theta.detach().cpu(), state0, dstate0_dA, dt, nsteps, sphere)
        ctx.save_for_backward(grad.to(theta.dtype))
        return torch.tensor(L, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None, None, None, None, None, None, None


def sphere(radius=6.0, centre=(0.0, 0.0, 0.0)) -> grf_sphere:
    return grf_sphere(float(radius), float(centre[0]), float(centre[1]), float(centre[2]))
