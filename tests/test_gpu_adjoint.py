"""The reverse sweep (grf_signal_forward + grf_adjoint_rk4) of the RK4 evolution and of the
sphere-averaged scalar signal:
  * dot-product tests against the oracle's tangent-linear model: for random directions
    (delta state_0, delta lambda, delta g2) and random cotangents (state_bar_N, L_bar),
        L_bar dL + <state_bar_N, delta state_N>   (oracle TLM, forward)
      = <state_bar_0, delta state_0> + lambda_bar delta lambda + g2_bar delta g2   (GPU, reverse)
    to 1e-10, on periodic and frozen boxes, every coupling kind, with and without
    backreaction, with the cubic Horndeski term, with checkpoint segments shorter and longer
    than the run;
  * the gradient in (lambda, g2, A) against the GPU tangent-linear evolution (grf_tlm_rk4);
  * the 96^3 differentiation workload (dx = 0.2, periodic, R = 6) for 40 steps with a checkpoint
    every 20, and for its stated 400 steps through the torch.autograd.Function: against central
    finite differences (h = 1e-6) to 1e-5 and against the tangents;
  * determinism, and the torch.autograd.Function whose backward runs the sweep.
"""
import numpy as np
import pytest

import grf_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    import paper_2309_06225_gb300 as grf
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return grf


def forward_and_adjoint(g, box, params, s0, dt, n, sphere, ce, loss_bar, ubar_n, ws=None):
    import torch
    b, p = g.box_like(box), g.params_like(params)
    st = g.to_device(s0, b)
    ck = torch.empty((max(g.checkpoint_count(n, ce), 1),) + tuple(st.shape), dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    if ws is None:
        ws = g.alloc_workspace(g.grf_adjoint_workspace_bytes(b, ce))
    sph = g.grf_sphere(*[float(x) for x in sphere])
    g.grf_signal_forward(b, p, st, dt, n, sph, ce, ck, loss, ws=ws)
    sbar = g.to_device(ubar_n, b)
    pbar = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.grf_adjoint_rk4(b, p, ck, dt, n, sph, ce, loss_bar, sbar, pbar, ws=ws)
    return float(loss.cpu()[0]), g.to_host(st, b), g.to_host(sbar, b), pbar.cpu().numpy()


def interior_random(box, rng, scale):
    a = np.zeros(box.shape)
    box.interior(a)[...] = rng.normal(size=box.interior(a).shape) * scale
    return a


DOT_CASES = {
    "periodic_quadratic": lambda: (gi.cube_box(12, -3.0, 3.0), gi.Params(lam=0.05, g2=0.02, beta_kind=gi.BETA_QUADRATIC),
                                   (1.7, 0.1, -0.05, 0.07), 3, 2),
    "frozen_linear_ragged": lambda: (gi.Box(13, 11, 12, 0.45, -2.6, -2.3, -2.4, bc=gi.BC_FROZEN),
                                     gi.Params(lam=0.3, g2=0.2, beta_kind=gi.BETA_LINEAR), (1.4, 0.2, 0.0, 0.1), 2, 1),
    "frozen_linear_cubic": lambda: (gi.Box(12, 11, 10, 0.45, -2.5, -2.3, -2.1, bc=gi.BC_FROZEN),
                                    gi.Params(lam=0.3, g2=0.2, beta_kind=gi.BETA_LINEAR, g3=0.4), (1.4, 0.2, 0.0, 0.1),
                                    2, 1),
    "periodic_exponential_decoupled": lambda: (gi.cube_box(10, -2.5, 2.5),
                                               gi.Params(lam=0.2, g2=0.1, beta_kind=gi.BETA_EXPONENTIAL,
                                                         beta_kappa=0.8, decoupled=1), (1.3, 0.0, 0.1, -0.1), 2, 5),
}


@pytest.mark.parametrize("case", list(DOT_CASES))
def test_dot_product_against_the_oracle_tangent_linear_model(g, orc, case):
    box, params, sphere, n, ce = DOT_CASES[case]()
    dt = 0.25 * box.dx
    rng = np.random.default_rng(11)
    s0 = gi.random_perturbed_state(box, 5, base=gi.single_puncture(box, amp=0.05), eps=1e-2)
    orc.fill_ghosts(box, s0)
    du0 = interior_random(box, rng, 1e-2)   # frozen ghosts are constants: no perturbation there
    dp = np.array([0.3, -0.2])
    ubar_n = interior_random(box, rng, 1.0)
    loss_bar = 0.7
    # oracle: tangent-linear model forward
    s, ds = s0.copy(), du0.copy()
    if box.bc == gi.BC_PERIODIC:
        orc.fill_ghosts(box, ds)
    st, L_cpu, dL = orc.tlm_rk4(box, params, s, ds, dp, dt, n, sphere, mode="dual")
    assert st == 0
    lhs = loss_bar * dL + np.sum(box.interior(ubar_n) * box.interior(ds))
    # GPU: reverse sweep
    L_gpu, _, sbar0, pbar = forward_and_adjoint(g, box, params, s0, dt, n, sphere, ce, loss_bar, ubar_n)
    rhs = np.sum(box.interior(sbar0) * box.interior(du0)) + pbar @ dp
    assert abs(L_gpu - L_cpu) <= 1e-11 * abs(L_cpu)
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs)), (lhs, rhs)


TLM_BOX = gi.Box(16, 16, 16, 0.75, -5.625, -5.625, -5.625, bc=gi.BC_FROZEN)


def test_gradient_equals_the_gpu_tangent_linear_evolution(g):
    """dL/d(lambda, g2, A) from the reverse sweep equals grf_tlm_rk4's forward-mode derivatives."""
    import torch
    box, params, A = TLM_BOX, gi.Params(lam=0.4, g2=0.2, beta_kind=gi.BETA_LINEAR), 0.05
    dt, n, R = 0.25 * box.dx, 6, 3.0
    s0 = gi.single_puncture(box, amp=A, r0=2.0)
    dphi = np.zeros(box.shape)
    dphi[25] = gi.single_puncture(box, amp=1.0)[25]
    b, p = g.box_like(box), g.params_like(params)
    state = g.to_device(s0, b)
    tang = g.alloc_state(b, 81)
    tang.view(3, -1)[2].copy_(g.to_device(dphi, b).reshape(-1))
    loss = torch.zeros(4, dtype=torch.float64, device="cuda")
    g.grf_tlm_rk4(b, p, [1.0, 0.0, 0.0, 1.0, 0.0, 0.0], state, tang, dt, n, g.grf_sphere(R, 0.0, 0.0, 0.0), loss)
    tlm = loss.cpu().numpy()
    L, _, sbar0, pbar = forward_and_adjoint(g, box, params, s0, dt, n, (R, 0.0, 0.0, 0.0), 4, 1.0, np.zeros(box.shape))
    dA = np.sum(box.interior(sbar0) * box.interior(dphi))
    grad = np.array([pbar[0], pbar[1], dA])
    assert L == tlm[0]  # same stage kernels, same bits
    np.testing.assert_allclose(grad, tlm[1:], rtol=1e-10)


@pytest.fixture(scope="module")
def workload96(g):
    box = gi.cube_box(96, -9.6, 9.6)
    params = gi.Params(lam=0.01, g2=0.01)
    amp = 1e-3
    dphi = np.zeros(box.shape)
    dphi[25] = gi.single_puncture(box, amp=1.0)[25]
    return box, params, amp, dphi, 0.25 * box.dx


def test_full_size_96_gradient_against_finite_differences_and_tangents(g, workload96):
    """The 96^3 differentiation workload, 40 RK4 steps with a checkpoint every 20: the reverse
    sweep's dL/d(lambda, g2, A) against central differences of the GPU evolution (h = 1e-6,
    relative 1e-5) and against the forward-mode tangents (1e-9)."""
    import torch
    box, params, amp, dphi, dt = workload96
    n, ce, R = 40, 20, 6.0
    b = g.box_like(box)
    ws = g.alloc_workspace(g.grf_adjoint_workspace_bytes(b, ce))
    s0 = gi.single_puncture(box, amp=amp)
    L, _, sbar0, pbar = forward_and_adjoint(g, box, params, s0, dt, n, (R, 0.0, 0.0, 0.0), ce, 1.0,
                                            np.zeros(box.shape), ws=ws)
    grad = np.array([pbar[0], pbar[1], np.sum(box.interior(sbar0) * box.interior(dphi))])
    sph = g.grf_sphere(R, 0.0, 0.0, 0.0)

    def signal(lam, g2, A):
        p = g.params_like(gi.Params(lam=lam, g2=g2))
        st = g.to_device(gi.single_puncture(box, amp=A), b)
        ck = torch.empty((g.checkpoint_count(n, ce),) + tuple(st.shape), dtype=torch.float64, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        g.grf_signal_forward(b, p, st, dt, n, sph, ce, ck, loss, ws=ws)
        return float(loss.cpu()[0])

    h = 1e-6
    fd = np.array([(signal(params.lam + h, params.g2, amp) - signal(params.lam - h, params.g2, amp)) / (2 * h),
                   (signal(params.lam, params.g2 + h, amp) - signal(params.lam, params.g2 - h, amp)) / (2 * h),
                   (signal(params.lam, params.g2, amp + h) - signal(params.lam, params.g2, amp - h)) / (2 * h)])
    # each quotient's rounding floor: 20 eps |L| / h
    floor = 20 * np.finfo(float).eps * abs(L) / h
    for k in range(3):
        assert abs(fd[k] - grad[k]) <= max(1e-5 * abs(grad[k]), floor), (k, fd, grad, floor)
    # forward-mode tangents of the same evolution
    p = g.params_like(params)
    state = g.to_device(s0, b)
    tang = g.alloc_state(b, 81)
    tang.view(3, -1)[2].copy_(g.to_device(dphi, b).reshape(-1))
    loss = torch.zeros(4, dtype=torch.float64, device="cuda")
    g.grf_tlm_rk4(b, p, [1.0, 0.0, 0.0, 1.0, 0.0, 0.0], state, tang, dt, n, sph, loss)
    tlm = loss.cpu().numpy()
    assert L == tlm[0]
    np.testing.assert_allclose(grad, tlm[1:], rtol=1e-9)


def test_config_96_400_steps_through_the_autograd_function(g, workload96):
    """The differentiation workload as stated: 96^3 (dx = 0.2, periodic), 400 RK4 steps, a
    checkpoint every 20 with recomputation, the sphere signal at r = 6. The gradient in
    (lambda, g2, A) from SignalAdjoint's backward (the reverse sweep, 20 segments) against central
    differences of the GPU evolution (h = 1e-6, relative 1e-5) and against the forward-mode
    tangents of the same evolution (1e-9). About six minutes on a GB300."""
    import torch
    from paper_2309_06225_gb300 import diff
    box, params, amp, dphi, dt = workload96
    n, ce, R = 400, 20, 6.0
    b, p = g.box_like(box), g.params_like(params)
    s0 = g.to_device(gi.single_puncture(box, amp=amp), b)
    dA = g.to_device(dphi, b)
    sph = diff.sphere(R)
    theta = torch.tensor([params.lam, params.g2, amp], dtype=torch.float64, requires_grad=True)
    L = diff.SignalAdjoint.apply(theta, b, p, s0, dA, dt, n, sph, ce)
    L.backward()
    grad = theta.grad.numpy().copy()
    L = float(L.detach())
    ws = g.alloc_workspace(g.grf_adjoint_workspace_bytes(b, ce))
    ck = torch.empty((g.checkpoint_count(n, ce),) + tuple(s0.shape), dtype=torch.float64, device="cuda")

    def signal(lam, g2, A):
        st = g.to_device(gi.single_puncture(box, amp=A), b)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        g.grf_signal_forward(b, g.params_like(gi.Params(lam=lam, g2=g2)), st, dt, n, sph, ce, ck, loss, ws=ws)
        return float(loss.cpu()[0])

    h = 1e-6
    fd = np.array([(signal(params.lam + h, params.g2, amp) - signal(params.lam - h, params.g2, amp)) / (2 * h),
                   (signal(params.lam, params.g2 + h, amp) - signal(params.lam, params.g2 - h, amp)) / (2 * h),
                   (signal(params.lam, params.g2, amp + h) - signal(params.lam, params.g2, amp - h)) / (2 * h)])
    floor = 20 * np.finfo(float).eps * abs(L) / h
    for k in range(3):
        assert abs(fd[k] - grad[k]) <= max(1e-5 * abs(grad[k]), floor), (k, fd, grad, floor)
    del ws, ck
    state = g.to_device(gi.single_puncture(box, amp=amp), b)
    tang = g.alloc_state(b, 81)
    tang.view(3, -1)[2].copy_(dA.reshape(-1))
    loss = torch.zeros(4, dtype=torch.float64, device="cuda")
    g.grf_tlm_rk4(b, p, [1.0, 0.0, 0.0, 1.0, 0.0, 0.0], state, tang, dt, n, sph, loss)
    tlm = loss.cpu().numpy()
    assert L == tlm[0]
    np.testing.assert_allclose(grad, tlm[1:], rtol=1e-9)


def test_reverse_sweep_is_deterministic(g):
    box, params, sphere, n, ce = DOT_CASES["periodic_quadratic"]()
    dt = 0.25 * box.dx
    s0 = gi.random_perturbed_state(box, 5, base=gi.single_puncture(box, amp=0.05), eps=1e-2)
    ubar = interior_random(box, np.random.default_rng(3), 1.0)
    r1 = forward_and_adjoint(g, box, params, s0, dt, n, sphere, ce, 0.5, ubar)
    r2 = forward_and_adjoint(g, box, params, s0, dt, n, sphere, ce, 0.5, ubar)
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[3], r2[3])


def test_reverse_sweep_is_deterministic_across_waves(g, workload96):
    """At 96^3 a reversed stage runs in six waves of tape columns, each taped then swept, the
    columns' parameter sums accumulating across the waves. Two runs give the same bits."""
    box, params, amp, dphi, dt = workload96
    s0 = gi.single_puncture(box, amp=amp)
    ubar = interior_random(box, np.random.default_rng(9), 1.0)
    r1 = forward_and_adjoint(g, box, params, s0, dt, 2, (6.0, 0.0, 0.0, 0.0), 20, 0.5, ubar)
    r2 = forward_and_adjoint(g, box, params, s0, dt, 2, (6.0, 0.0, 0.0, 0.0), 20, 0.5, ubar)
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[3], r2[3])
    assert np.any(r1[2] != 0.0)


def test_autograd_backward_runs_the_reverse_sweep(g):
    """SignalAdjoint.backward returns grad_out * dL/dtheta from the sweep; the forward-mode
    SphereSignal agrees and keeps theta's device."""
    import torch
    from paper_2309_06225_gb300 import diff
    box, A = TLM_BOX, 0.05
    params = gi.Params(lam=0.4, g2=0.2, beta_kind=gi.BETA_LINEAR)
    dt, n = 0.25 * box.dx, 4
    b = g.box_like(box)
    s0 = g.to_device(gi.single_puncture(box, amp=A), b)
    dphi = np.zeros(box.shape)
    dphi[25] = gi.single_puncture(box, amp=1.0)[25]
    dA = g.to_device(dphi, b)
    sph = diff.sphere(3.0)
    theta = torch.tensor([params.lam, params.g2, A], dtype=torch.float64, device="cuda", requires_grad=True)
    L = diff.SignalAdjoint.apply(theta, b, g.params_like(params), s0, dA, dt, n, sph, 2)
    (2.0 * L).backward()
    grad_rev = theta.grad.detach().clone()
    assert grad_rev.device.type == "cuda"
    theta2 = theta.detach().clone().requires_grad_(True)
    L2 = diff.SphereSignal.apply(theta2, b, g.params_like(params), s0, dA, dt, n, sph)
    assert L2.device.type == "cuda"
    (2.0 * L2).backward()
    assert float(L.detach()) == float(L2.detach())
    np.testing.assert_allclose(grad_rev.cpu().numpy(), theta2.grad.cpu().numpy(), rtol=1e-10)
