"""Differentiable sphere-averaged scalar signal, as torch.autograd.Functions.

theta = (lambda, g2, A): the Gauss-Bonnet coupling, the X^2 coupling and the amplitude of the
initial scalar profile. The caller supplies the initial state at the current A together with
its derivative with respect to A (for phi = A f(x) that is the state with phi = f and every
other field zero).

SignalAdjoint (reverse mode): forward evolves the state with grf_signal_forward, storing a
checkpoint every `checkpoint_every` RK4 steps; backward runs the reverse sweep grf_adjoint_rk4
from those checkpoints (recomputing each segment and each step's stages) and returns
grad_out * dL/dtheta, the A component as <d L/d state_0, d state_0/dA> (grf_state_dot).

SphereSignal (forward mode): the tangent-linear evolution grf_tlm_rk4 gives L and the three
derivatives in one pass; backward returns the stored gradient. It is the cross-check of the
reverse sweep.
"""
from __future__ import annotations

import torch

from . import (alloc_state, alloc_workspace, checkpoint_count, grf_adjoint_rk4, grf_adjoint_workspace_bytes,
               grf_params, grf_signal_forward, grf_sphere, grf_state_dot, grf_tlm_rk4, grf_tlm_workspace_bytes)


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
        ctx.save_for_backward(grad.to(device=theta.device, dtype=theta.dtype))
        return torch.tensor(L, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None, None, None, None, None, None, None


class SignalAdjoint(torch.autograd.Function):
    """L(theta) with theta = (lambda, g2, A); backward runs the reverse sweep over the forward
    pass's checkpoints."""

    @staticmethod
    def forward(ctx, theta, box, params, state0, dstate0_dA, dt, nsteps, sphere, checkpoint_every=20):
        if str(theta.dtype) != "torch.float64":
            raise TypeError("theta must be float64")
        lam, g2, _ = (float(x) for x in theta.detach().cpu())
        p = _with_couplings(params, lam, g2)
        state = state0.clone()
        ck = torch.empty((max(checkpoint_count(nsteps, checkpoint_every), 1),) + tuple(state.shape),
                         dtype=torch.float64, device=state.device)
        loss = torch.zeros(1, dtype=torch.float64, device=state.device)
        ws = alloc_workspace(grf_adjoint_workspace_bytes(box, checkpoint_every), state.device)
        grf_signal_forward(box, p, state, dt, nsteps, sphere, checkpoint_every, ck, loss, ws=ws)
        ctx.saved = (box, p, ck, dstate0_dA, float(dt), int(nsteps), sphere, int(checkpoint_every), ws)
        return loss[0].to(device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        box, p, ck, dstate0_dA, dt, nsteps, sphere, ce, ws = ctx.saved
        sbar = torch.zeros_like(dstate0_dA)
        pbar = torch.zeros(2, dtype=torch.float64, device=sbar.device)
        grf_adjoint_rk4(box, p, ck, dt, nsteps, sphere, ce, float(grad_out), sbar, pbar, ws=ws)
        dA = torch.zeros(1, dtype=torch.float64, device=sbar.device)
        grf_state_dot(box, sbar, dstate0_dA, -1, dA)
        grad = torch.cat([pbar, dA]).to(device=grad_out.device)
        ctx.saved = None
        return grad, None, None, None, None, None, None, None, None


def sphere(radius=6.0, centre=(0.0, 0.0, 0.0)) -> grf_sphere:
    return grf_sphere(float(radius), float(centre[0]), float(centre[1]), float(centre[2]))
