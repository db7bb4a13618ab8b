"""Gradients of the sphere-averaged scalar signal with respect to (lambda, g2, A) from the
tangent-linear evolution (grf_tlm_rk4), checked against central finite differences of the
GPU evolution and of the CPU oracle, and through the torch.autograd.Function."""
import math

import numpy as np
import pytest

import grf_inputs as gi

pytestmark = pytest.mark.gpu

S2, S3 = 1.0 / math.sqrt(2.0), 1.0 / math.sqrt(3.0)


def lebedev26():
    """26-point degree-7 rule on the unit sphere (axis, edge-midpoint and corner directions)."""
    pts, w = [], []
    for a in range(3):
        for s in (1.0, -1.0):
            p = [0.0, 0.0, 0.0]
            p[a] = s
            pts.append(p)
            w.append(1.0 / 21.0)
    for (a, b) in ((0, 1), (0, 2), (1, 2)):
        for sa in (1.0, -1.0):
            for sb in (1.0, -1.0):
                p = [0.0, 0.0, 0.0]
                p[a], p[b] = sa * S2, sb * S2
                pts.append(p)
                w.append(4.0 / 105.0)
    for sx in (1.0, -1.0):
        for sy in (1.0, -1.0):
            for sz in (1.0, -1.0):
                pts.append([sx * S3, sy * S3, sz * S3])
                w.append(9.0 / 280.0)
    return np.array(pts), np.array(w)


def host_signal(box, state, R):
    """sum_q w_q phi(R x_q) by trilinear interpolation on the interior points."""
    pts, w = lebedev26()
    phi = box.interior(state)[25]
    tot = 0.0
    for p, wq in zip(pts, w):
        f = [(R * p[0] - box.x0) / box.dx, (R * p[1] - box.y0) / box.dx, (R * p[2] - box.z0) / box.dx]
        i0 = [int(math.floor(x)) for x in f]
        t = [x - i for x, i in zip(f, i0)]
        val = 0.0
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    wt = (t[0] if dx else 1 - t[0]) * (t[1] if dy else 1 - t[1]) * (t[2] if dz else 1 - t[2])
                    val += wt * phi[i0[2] + dz, i0[1] + dy, i0[0] + dx]
        tot += wq * val
    return tot


BOX = gi.Box(16, 16, 16, 0.75, -5.625, -5.625, -5.625, bc=gi.BC_FROZEN)
R = 3.0
NSTEPS = 6
THETA = (0.4, 0.2, 0.05)  # lambda, g2, A


def initial(A):
    return gi.single_puncture(BOX, amp=A, r0=2.0)


def dstate_dA():
    s = np.zeros(BOX.shape)
    s[25] = gi.single_puncture(BOX, amp=1.0)[25]
    return s


def params_of(theta):
    return gi.Params(lam=theta[0], g2=theta[1], beta_kind=gi.BETA_LINEAR)


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_06225_gb300 import build
    build.build()
    import paper_2309_06225_gb300 as grf
    grf.lib()
    return grf


def gpu_signal(g, theta):
    b = g.box_like(BOX)
    t = g.to_device(initial(theta[2]), b)
    dt = 0.25 * BOX.dx
    ws = g.alloc_workspace(g.grf_workspace_bytes(b, g.GRF_OP_RK4))
    L = 0.0
    for _ in range(NSTEPS):
        g.grf_rk4_step(b, g.params_like(params_of(theta)), t, dt, 1, ws=ws)
        L += dt * host_signal(BOX, g.to_host(t, b), R)
    return L


def oracle_signal(orc, theta):
    s = initial(theta[2])
    dt = 0.25 * BOX.dx
    L = 0.0
    for _ in range(NSTEPS):
        orc.rk4(BOX, params_of(theta), s, dt, 1)
        L += dt * host_signal(BOX, s, R)
    return L


@pytest.fixture(scope="module")
def tlm(g):
    import torch
    from paper_2309_06225_gb300 import diff
    b = g.box_like(BOX)
    s0 = g.to_device(initial(THETA[2]), b)
    ds = g.to_device(dstate_dA(), b)
    L, grad = diff.sphere_signal_and_grad(b, g.params_like(params_of(THETA)), torch.tensor(THETA, dtype=torch.float64), s0, ds,
                                          0.25 * BOX.dx, NSTEPS, diff.sphere(R))
    return L, grad.numpy()


def test_tlm_value_matches_primal_signal(g, tlm):
    L, _ = tlm
    ref = gpu_signal(g, THETA)
    assert abs(L - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tlm_gradient_matches_gpu_finite_differences(g, tlm, k):
    _, grad = tlm
    h = 1e-4 * max(abs(THETA[k]), 1e-2)
    tp = list(THETA); tm = list(THETA)
    tp[k] += h
    tm[k] -= h
    fd = (gpu_signal(g, tp) - gpu_signal(g, tm)) / (2 * h)
    assert abs(grad[k] - fd) <= 1e-5 * abs(fd), (k, grad[k], fd)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tlm_gradient_matches_oracle_finite_differences(orc, tlm, k):
    _, grad = tlm
    h = 1e-4 * max(abs(THETA[k]), 1e-2)
    tp = list(THETA); tm = list(THETA)
    tp[k] += h
    tm[k] -= h
    fd = (oracle_signal(orc, tp) - oracle_signal(orc, tm)) / (2 * h)
    assert abs(grad[k] - fd) <= 1e-5 * abs(fd), (k, grad[k], fd)


def test_autograd_function(g, tlm):
    import torch
    from paper_2309_06225_gb300 import diff
    b = g.box_like(BOX)
    s0 = g.to_device(initial(THETA[2]), b)
    ds = g.to_device(dstate_dA(), b)
    theta = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
    L = diff.SphereSignal.apply(theta, b, g.params_like(params_of(THETA)), s0, ds, 0.25 * BOX.dx, NSTEPS, diff.sphere(R))
    (gr,) = torch.autograd.grad(3.0 * L, theta)
    np.testing.assert_allclose(gr.numpy(), 3.0 * tlm[1], rtol=1e-12)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tlm_gradient_matches_richardson_differences(g, tlm, k):
    """Forward mode differentiates the discrete evolution exactly, so the gradient must agree with
    Richardson-extrapolated central differences of the GPU evolution, (4 D(h/2) - D(h)) / 3 with
    truncation error O(h^4), down to the rounding floor of the difference quotient:
    ~eps |L| / (h |dL/dtheta|), or 1e-10 relative where that is smaller (lambda and A reach
    1e-12; dL/dg2 is small, so its quotient carries ~1e-7 of rounding)."""
    L, grad = tlm
    h = 1e-3 * max(abs(THETA[k]), 1e-2)

    def central(hh):
        tp = list(THETA); tm = list(THETA)
        tp[k] += hh
        tm[k] -= hh
        return (gpu_signal(g, tp) - gpu_signal(g, tm)) / (2 * hh)

    rich = (4.0 * central(h / 2) - central(h)) / 3.0
    floor = 20 * np.finfo(float).eps * abs(L) / (h * abs(grad[k]))
    assert abs(rich / grad[k] - 1.0) <= max(1e-10, floor), (k, grad[k], rich, floor)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tlm_gradient_matches_oracle_richardson_differences(orc, tlm, k):
    """The oracle's own derivative of the same discrete evolution, taken by Richardson-extrapolated
    central differences (truncation O(h^4)), against the GPU's forward-mode derivative: they agree
    to the rounding floor of the oracle's difference quotient, or 1e-10 relative where that is
    smaller. The two codes share no arithmetic, so this pins the tangent to the oracle well
    below the 1e-5 of plain differences."""
    L, grad = tlm
    h = 1e-3 * max(abs(THETA[k]), 1e-2)

    def central(hh):
        tp = list(THETA); tm = list(THETA)
        tp[k] += hh
        tm[k] -= hh
        return (oracle_signal(orc, tp) - oracle_signal(orc, tm)) / (2 * hh)

    rich = (4.0 * central(h / 2) - central(h)) / 3.0
    floor = 20 * np.finfo(float).eps * abs(L) / (h * abs(grad[k]))
    assert abs(rich / grad[k] - 1.0) <= max(1e-10, floor), (k, grad[k], rich, floor)


def test_tlm_exponential_coupling_gradients(g, orc):
    """The tangent evolution with the exponential coupling (exp of the dual numbers): the
    gradients in (lambda, g2, A) agree with central differences of the oracle's evolution."""
    import torch
    from paper_2309_06225_gb300 import diff
    theta = (0.4, 0.2, 0.3)  # an amplitude large enough for e^{-kappa phi^2} to matter

    def params(t):
        return gi.Params(lam=t[0], g2=t[1], beta_kind=gi.BETA_EXPONENTIAL, beta_kappa=3.0)

    b = g.box_like(BOX)
    s0 = g.to_device(initial(theta[2]), b)
    ds = g.to_device(dstate_dA(), b)
    _, grad = diff.sphere_signal_and_grad(b, g.params_like(params(theta)), torch.tensor(theta, dtype=torch.float64),
                                          s0, ds, 0.25 * BOX.dx, NSTEPS, diff.sphere(R))
    grad = grad.numpy()

    def signal(t):
        s = initial(t[2])
        dt = 0.25 * BOX.dx
        L = 0.0
        for _ in range(NSTEPS):
            orc.rk4(BOX, params(t), s, dt, 1)
            L += dt * host_signal(BOX, s, R)
        return L

    for k in range(3):
        h = 1e-4 * max(abs(theta[k]), 1e-2)
        tp = list(theta); tm = list(theta)
        tp[k] += h
        tm[k] -= h
        fd = (signal(tp) - signal(tm)) / (2 * h)
        assert abs(grad[k] - fd) <= 1e-5 * abs(fd), (k, grad[k], fd)
