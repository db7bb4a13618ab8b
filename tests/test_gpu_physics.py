"""The GPU evolution against exact linear solutions on flat space (the GPU counterparts of the
oracle's wave pins): a weak gravitational plane wave and the longitudinal gauge modes of the
modified puncture gauge, evolved by grf_rk4_step, converge at 4th order to the closed forms."""
import math

import numpy as np
import pytest

import grf_inputs as gi
import waves

pytestmark = pytest.mark.gpu


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


def evolve(g, b, params, s, dt, nsteps):
    gb = g.box_like(b)
    t = g.to_device(s, gb)
    g.grf_rk4_step(gb, g.params_like(params), t, dt, nsteps)
    assert g.grf_check_status() == 0
    return g.to_host(t, gb)


def convergence(g, make, params, fields, scales, L=2.0, T=0.6):
    errs = []
    for n in (16, 32):
        b = gi.Box(n, 4, 4, L / n, 0.5 * L / n, 0.0, 0.0)
        dt = 0.25 * b.dx
        nsteps = int(round(T / dt))
        got = evolve(g, b, params, make(b, 0.0), dt, nsteps)
        ex = make(b, nsteps * dt)
        errs.append(max(np.max(np.abs(b.interior(got)[f] - b.interior(ex)[f])) / sc for f, sc in zip(fields, scales)))
    return errs


def test_gravitational_plane_wave(g):
    amp, k = 1e-6, math.pi
    errs = convergence(g, lambda b, t: waves.tt_wave_state(b, amp, k, t), gi.Params(lam=0.0, g2=0.0),
                       [4, 5, 6, 11, 12, 13], [amp, amp, amp, amp * k, amp * k, amp * k], T=0.5)
    assert errs[1] < 1e-3 and 13 < errs[0] / errs[1] < 19, errs


@pytest.mark.parametrize("a0", [0.0, 0.2])
def test_gauge_wave(g, a0):
    eps, k = 1e-6, math.pi
    p = gi.Params(lam=0.0, g2=0.0, shift_F=0.0, a0=a0, b0=0.4)
    errs = convergence(g, lambda b, t: waves.gauge_wave_state(b, eps, k, t, a0), p, [18, 7, 1, 15, 19],
                       [eps, eps * k, eps, eps * k, eps])
    assert errs[1] < 1e-3 and 13 < errs[0] / errs[1] < 19, errs


def test_gamma_driver_gauge_wave(g):
    pytest.importorskip("scipy")
    eps, k, a, F, eta = 1e-6, math.pi, 0.2, 0.75, 1.0
    p = gi.Params(lam=0.0, g2=0.0, shift_F=F, eta=eta, a0=a, b0=0.4)
    errs = convergence(g, lambda b, t: waves.gamma_driver_wave_state(b, eps, k, t, a, F, eta), p,
                       [18, 7, 1, 15, 19, 22], [eps, eps * k, eps, eps * k, eps, eps * k])
    assert errs[1] < 1e-3 and 13 < errs[0] / errs[1] < 19, errs
