"""The cubic Horndeski term (1/16 pi) g3 X box(phi) on the GPU against the oracle:
  * RHS and 3 RK4 steps on every boundary type, with and without backreaction, the 4th- and
    6th-order schemes and lopsided advection (the general stage instantiation, chosen whenever
    g3 != 0);
  * the term changes the right-hand sides (the switch takes effect), and g3 = 0 through the
    general instantiation gives the default instantiation's bits;
  * the hyperbolicity diagnostics (the cubic effective metric needs d_t Pi, so it is evaluated at
    the solution of the coupled system);
  * the batched launch with a cubic instance in the batch, bit for bit against the single-box path;
  * the tangent-linear evolution's gradients in (lambda, g2, A) against central differences of
    the oracle's evolution.
"""
import numpy as np
import pytest

import grf_inputs as gi
from parity import describe, field_errors

pytestmark = pytest.mark.gpu

G3 = 0.4


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


def P(**kw):
    p = gi.Params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def state_for(box, seed):
    """The puncture plus seeded sinusoids in every field, and a scalar bump whose second
    derivatives make the cubic terms of order one percent of the others."""
    if box.bc == gi.BC_REFLECT_LOW:
        s = gi.random_perturbed_state(box, seed, base=gi.mirror_symmetric_state(box), eps=2e-2)
    else:
        s = gi.random_perturbed_state(box, seed, base=gi.single_puncture(box, amp=0.05), eps=3e-2)
    X, Y, Z = box.coords()
    s[25] += 0.2 * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 2.0)
    return s


def gpu_rhs(g, box, params, s):
    b = g.box_like(box)
    t = g.to_device(s, b)
    r = g.alloc_state(b)
    g.grf_rhs(b, g.params_like(params), t, r)
    assert g.grf_check_status() == 0
    return g.to_host(r, b)


def gpu_rk4(g, box, params, s, dt, n):
    b = g.box_like(box)
    t = g.to_device(s, b)
    g.grf_rk4_step(b, g.params_like(params), t, dt, n)
    assert g.grf_check_status() == 0
    return g.to_host(t, b)


def check_rhs_and_rk4(g, orc, box, params, seed, nsteps=3):
    s0 = state_for(box, seed)
    filled = s0.copy()
    orc.fill_ghosts(box, filled)
    ref = orc.rhs(box, params, filled)
    out = gpu_rhs(g, box, params, s0)
    errs = field_errors(out, ref, box, state=filled, sigma=params.sigma_ko)
    assert np.max(errs) < 1e-11, describe(errs)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, nsteps)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, nsteps)
    errs = field_errors(gpu, cpu, box)
    assert np.max(errs) < 1e-10, describe(errs)
    return s0, out


BOXES = {
    gi.BC_PERIODIC: gi.Box(14, 11, 9, 0.3, -2.0, -1.6, -1.3, bc=gi.BC_PERIODIC),
    gi.BC_FROZEN: gi.Box(14, 11, 9, 0.3, -2.0, -1.6, -1.3, bc=gi.BC_FROZEN),
    gi.BC_REFLECT_LOW: gi.Box(14, 11, 9, 0.3, 0.15, 0.15, 0.15, bc=gi.BC_REFLECT_LOW),
}


@pytest.mark.parametrize("decoupled", [0, 1])
@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN, gi.BC_REFLECT_LOW])
def test_cubic_rhs_and_rk4_parity(g, orc, bc, decoupled):
    box = BOXES[bc]
    params = P(lam=0.3, g2=0.2, beta_kind=1, g3=G3, decoupled=decoupled)
    s0, out = check_rhs_and_rk4(g, orc, box, params, 61 + bc)
    # the cubic term takes effect: d_t Pi (and with backreaction d_t K) move by far more than
    # the parity tolerance
    base = gpu_rhs(g, box, P(lam=0.3, g2=0.2, beta_kind=1, decoupled=decoupled), s0)
    for f in ([26] if decoupled else [26, 7]):
        d = np.max(np.abs(box.interior(out)[f] - box.interior(base)[f]))
        assert d > 1e-4 * np.max(np.abs(box.interior(base)[f])), f


@pytest.mark.parametrize("ng,advection", [(3, 1), (4, 0), (4, 1)])
def test_cubic_schemes_parity(g, orc, ng, advection):
    """Lopsided advection and the 6th-order scheme with the cubic term."""
    box = gi.Box(13, 11, 10, 0.3, -1.9, -1.6, -1.5, bc=gi.BC_FROZEN, ng=ng)
    check_rhs_and_rk4(g, orc, box, P(lam=0.3, g2=0.2, beta_kind=1, g3=-G3, advection=advection), 67)


def test_zero_g3_general_instantiation_matches_default(g):
    """g3 = 0 leaves the general instantiation's arithmetic as it was without the cubic term: the
    batched launch (which always runs the general instantiation, cubic branch included) gives the
    bits of the default single-box instantiation (which has no cubic code)."""
    import torch
    box = gi.Box(14, 11, 9, 0.3, -2.0, -1.6, -1.3)
    params = P(lam=0.3, g2=0.2, beta_kind=1)
    s0 = state_for(box, 71)
    ref = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 2)
    b = g.box_like(box)
    gp = g.params_array([g.params_like(params)])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dev = [g.to_device(s0, b)]
        items = g.batch_items([b], dev, [0], [0.25 * box.dx])
        cfg = g.batch_config(g.GRF_BATCH_GRAPH, (32, 4, 1))
        ws = g.alloc_workspace(g.grf_batched_workspace_bytes(items, cfg))
        g.grf_batched_rk4(items, gp, 2, cfg, ws=ws, stream=stream)
    stream.synchronize()
    assert np.array_equal(g.to_host(dev[0], b), ref)


@pytest.mark.parametrize("decoupled", [0, 1])
def test_cubic_hyperbolicity_parity(g, orc, decoupled):
    """grf_hyperbolicity with the cubic term: det M of the coupled system, det(g_eff)/det(g) by the
    Schur complement at the solved d_t Pi, and -g_eff^nn = 1 + 2 g2 X + 2 g2 Pi^2 + 2 g3 tr H, against
    the oracle (full-pivot determinants of its Jacobian and of the 4x4 g_eff) to 1e-11."""
    box = gi.Box(13, 17, 11, 0.3, -1.9, -2.3, -1.6)
    params = P(lam=0.3, g2=0.2, beta_kind=1, g3=G3, decoupled=decoupled)
    s = state_for(box, 73)
    filled = s.copy()
    orc.fill_ghosts(box, filled)
    ref = orc.hyperbolicity(box, params, filled)
    b = g.box_like(box)
    t = g.to_device(s, b)
    out = g.alloc_state(b, 4)
    g.grf_hyperbolicity(b, g.params_like(params), t, out)
    got = box.interior(g.to_host(out, b)[:4])
    for m in range(4):
        den = max(np.max(np.abs(ref[m])), 1e-300)
        assert np.max(np.abs(got[m] - ref[m])) <= 1e-11 * den, (m, np.max(np.abs(got[m] - ref[m])) / den)
    no_cubic = orc.hyperbolicity(box, P(lam=0.3, g2=0.2, beta_kind=1, decoupled=decoupled), filled)
    assert np.max(np.abs(ref[2] - no_cubic[2])) > 1e-4  # the cubic term moves -g_eff^nn


@pytest.mark.parametrize("variant", [1, 2])
def test_cubic_batched_equals_single_box_path(g, variant):
    """A batch whose instances mix the cubic term in and out: every box equals, bit for bit, the
    single-box path (which runs the general instantiation for the cubic instances)."""
    import torch
    boxes = [gi.Box(13, 9, 7, 0.25, -1.6, -1.1, -0.9, bc=gi.BC_FROZEN),
             gi.Box(8, 8, 8, 0.3, -1.05, -1.05, -1.05, bc=gi.BC_PERIODIC),
             gi.Box(16, 16, 8, 0.5, -3.75, -3.75, -1.75, bc=gi.BC_PERIODIC)]
    params = [P(lam=0.05, g2=0.02, g3=G3), P(lam=0.3, g2=0.1, beta_kind=1), P(lam=0.2, g2=0.1, g3=-G3, decoupled=1)]
    pidx = [0, 1, 2]
    states = [state_for(b, 80 + i) for i, b in enumerate(boxes)]
    dts = [0.25 * b.dx for b in boxes]
    gb = [g.box_like(b) for b in boxes]
    gp = g.params_array([g.params_like(p) for p in params])
    ref = []
    for b, s, pi, dt in zip(gb, states, pidx, dts):
        t = g.to_device(s, b)
        g.grf_rk4_step(b, gp[pi], t, dt, 2)
        ref.append(g.to_host(t, b))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dev = [g.to_device(s, b) for s, b in zip(states, gb)]
        items = g.batch_items(gb, dev, pidx, dts)
        cfg = g.batch_config(variant, (32, 4, 1))
        ws = g.alloc_workspace(g.grf_batched_workspace_bytes(items, cfg))
        g.grf_batched_rk4(items, gp, 2, cfg, ws=ws, stream=stream)
    stream.synchronize()
    for q, b in enumerate(gb):
        assert np.array_equal(g.to_host(dev[q], b), ref[q]), q


def test_cubic_tangent_linear_gradients(g, orc):
    """The tangent evolution (dual numbers in lambda, g2 and the scalar's amplitude A) with the
    cubic term: its gradients of the sphere-averaged signal agree with central differences of
    the oracle's evolution to 1e-5."""
    import torch
    from paper_2309_06225_gb300 import diff
    from test_gpu_tlm import BOX, NSTEPS, R, dstate_dA, host_signal, initial
    theta = (0.4, 0.2, 0.1)

    def params(t):
        return gi.Params(lam=t[0], g2=t[1], beta_kind=gi.BETA_LINEAR, g3=0.5)

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
        tp = list(theta)
        tm = list(theta)
        tp[k] += h
        tm[k] -= h
        fd = (signal(tp) - signal(tm)) / (2 * h)
        assert abs(grad[k] - fd) <= 1e-5 * abs(fd), (k, grad[k], fd)
