"""Pins of the oracle's tangent-linear model (TLM) of the RK4 evolution and of the sphere-averaged
scalar signal (no GPU).

The TLM is the oracle's own core instantiated on dual numbers; the complex-step instance of the
same core is an independent forward-mode construction (no subtraction, exact to rounding for
analytic steps). Both are checked against the plain double oracle (value part, bit for bit) and
against Richardson-extrapolated central differences of the plain oracle (the derivative of the
evolution itself, with no forward-mode arithmetic at all).
"""
import numpy as np
import pytest

import grf_inputs as gi

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", params=["quadratic", "linear_cubic"])
def setup(request):
    box = gi.cube_box(12, -3.0, 3.0)   # dx 0.5, periodic
    if request.param == "quadratic":
        P = gi.Params(lam=0.05, g2=0.02, beta_kind=gi.BETA_QUADRATIC)
    else:  # the cubic Horndeski term in the differentiated evolution (its coupling g3 held fixed)
        P = gi.Params(lam=0.05, g2=0.02, beta_kind=gi.BETA_LINEAR, g3=0.4)
    s0 = gi.random_perturbed_state(box, 3, base=gi.single_puncture(box, amp=0.05), eps=1e-2)
    rng = np.random.default_rng(1)
    ds0 = rng.normal(size=s0.shape) * 1e-2
    return box, P, s0, ds0, (1.7, 0.1, -0.05, 0.07), 0.25 * box.dx, 3


def _run(orc, setup, mode, dp=(0.3, -0.2), scale_ds=1.0):
    box, P, s0, ds0, sphere, dt, n = setup
    s, ds = s0.copy(), scale_ds * ds0
    orc.fill_ghosts(box, s)
    orc.fill_ghosts(box, ds)
    st, L, dL = orc.tlm_rk4(box, P, s, ds, np.array(dp), dt, n, sphere, mode=mode)
    assert st == 0
    return s, ds, L, dL


def test_tlm_value_part_is_the_plain_oracle(orc, setup):
    """Both tangent instances carry the plain evolution in their value part, bit for bit."""
    box, P, s0, ds0, sphere, dt, n = setup
    s = s0.copy()
    orc.fill_ghosts(box, s)
    st, L = orc.rk4_signal(box, P, s, dt, n, sphere)
    assert st == 0
    for mode in ("dual", "cs"):
        sv, _, Lv, _ = _run(orc, setup, mode)
        assert np.array_equal(sv, s) and Lv == L


@pytest.mark.parametrize("dp,scale_ds", [((0.3, -0.2), 1.0), ((1.0, 0.0), 0.0), ((0.0, 1.0), 0.0), ((0.0, 0.0), 1.0)])
def test_tlm_dual_numbers_match_the_complex_step(orc, setup, dp, scale_ds):
    """P11: the dual-number TLM and the complex step (h = 1e-30) agree to 1e-13 relative, on the
    evolved tangent state and on the signal's derivative, for mixed, coupling-only and state-only
    directions. Catches a wrong product or quotient rule, a non-analytic step handled differently,
    and a parameter whose tangent is dropped."""
    _, d1, _, dL1 = _run(orc, setup, "dual", dp, scale_ds)
    _, d2, _, dL2 = _run(orc, setup, "cs", dp, scale_ds)
    assert np.max(np.abs(d1 - d2)) <= 1e-13 * np.max(np.abs(d1))
    assert abs(dL1 - dL2) <= 1e-13 * abs(dL1)


@pytest.mark.parametrize("dp,scale_ds", [((0.3, -0.2), 1.0), ((1.0, 0.0), 0.0), ((0.0, 0.0), 1.0)])
def test_tlm_matches_richardson_differences_of_the_plain_oracle(orc, setup, dp, scale_ds):
    """dL along the direction equals (4 D(h/2) - D(h))/3 with D(h) the central difference of the
    plain oracle's signal (truncation O(h^4)), to the rounding floor of the quotient."""
    box, P, s0, ds0, sphere, dt, n = setup
    _, _, L, dL = _run(orc, setup, "dual", dp, scale_ds)

    def sig(e):
        s = s0 + e * scale_ds * ds0
        orc.fill_ghosts(box, s)
        p = gi.Params(lam=P.lam + e * dp[0], g2=P.g2 + e * dp[1], beta_kind=P.beta_kind, g3=P.g3)
        return orc.rk4_signal(box, p, s, dt, n, sphere)[1]

    h = 1e-3
    D = lambda hh: (sig(hh) - sig(-hh)) / (2.0 * hh)  # noqa: E731
    rich = (4.0 * D(h / 2) - D(h)) / 3.0
    floor = 20.0 * EPS * abs(L) / (h / 2) / abs(dL)
    assert abs(rich - dL) <= max(1e-8, floor) * abs(dL), (rich, dL, floor)


def test_sphere_signal_rule_on_a_static_linear_field(orc):
    """Flat space with a linear scalar phi = a.x + c and Pi = 0 (frozen ghosts), without
    backreaction, does not evolve (box phi = 0, no curvature). Trilinear interpolation is exact on it, and the 26-point rule has
    unit total weight and vanishing odd moments, so each step adds exactly dt * phi(centre)."""
    box = gi.Box(10, 9, 8, 0.4, -1.8, -1.6, -1.4, bc=gi.BC_FROZEN)
    s = gi.flat_state(box)
    a, c = np.array([0.3, -0.2, 0.5]), 0.7
    x, y, z = box.coords()
    s[gi.IDX["phi"]] = c + a[0] * x + a[1] * y + a[2] * z
    centre = np.array([0.05, 0.1, -0.02])
    st, L = orc.rk4_signal(box, gi.Params(lam=0.0, g2=0.0, decoupled=1), s, 0.1, 3, (1.0, *centre))
    assert st == 0
    assert L == pytest.approx(3 * 0.1 * (c + a @ centre), rel=1e-13)
