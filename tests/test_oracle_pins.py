"""Pins of the CPU oracle against facts fixed by the mathematics (no GPU).

Each test names the property it checks and the plausible mistakes it would catch. The
oracle is test infrastructure (oracle/); these tests establish that it is right before
the CUDA path is compared against it.
"""
import math

import numpy as np
import pytest

import grf_inputs as gi

sp = pytest.importorskip("sympy")
import analytic as an  # noqa: E402
import waves  # noqa: E402


def P(**kw):
    p = gi.Params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ----------------------------------------------------------------------------- P1 flat
@pytest.mark.parametrize("kw", [dict(), dict(a0=0.0, b0=0.0), dict(beta_kind=1, lam=0.3, g2=0.2),
                                dict(kappa1=0.5, kappa2=0.3, kappa3=0.5, a0=0.7, b0=1.3)])
def test_flat_space_rhs_is_exactly_zero(orc, kw):
    """Minkowski slice, unit lapse, zero shift and scalar: every RHS value and KO term is 0.0.
    Catches any additive constant or a term that survives on trivial data."""
    b = gi.Box(9, 8, 7, 0.3, -1.0, -1.0, -1.0)
    s = gi.flat_state(b)
    orc.fill_ghosts(b, s)
    r = orc.rhs(b, P(**kw), s)
    assert np.all(r == 0.0)


# ----------------------------------------------------------------------------- P1b damping
@pytest.mark.parametrize("k1,k2,alpha,chi,a0,b0", [(0.1, 0.0, 1.0, 1.0, 0.0, 0.0), (0.5, 0.3, 0.7, 0.6, 0.2, 0.4),
                                                   (0.25, -0.4, 1.3, 0.9, 0.0, 1.1)])
def test_z4_constraint_damping_rates_on_flat_data(orc, k1, k2, alpha, chi, a0, b0):
    """Damped Z4 on a flat slice: constant conformal factor, h = delta, K = A = 0, zero shift,
    a constant lapse, a constant Theta and a constant Z_i. Z_i is carried by Gamma-hat^i =
    Gamma-tilde^i + 2 h^ij Z_j with Gamma-tilde = 0. Every curvature, gradient and Z-derivative
    term vanishes, so only the damping is left. The constraint fields decay at the damped-Z4
    rates
        d_t Theta = -alpha kappa1 (2 + kappa2) Theta,   d_t Z_i = -alpha kappa1 Z_i,
    and the metric and A_ij stay static. With the modified gauge's b(x) the auxiliary metric
    g^ab - b n^a n^b of the Z terms multiplies the time-derivative terms of the nn and ni
    components of the covariant equation by (1 + b), so both rates are divided by (1 + b)
    (the covariant pin below checks the general case). Catches a dropped or anti-damping kappa
    term, kappa2 in the wrong place, a missing lapse factor, and Z read with the wrong metric
    factor."""
    v = np.zeros(27)
    v[0] = chi
    v[1], v[4], v[6] = 1.0, 1.0, 1.0
    theta = 0.3
    ghat = np.array([0.2, -0.1, 0.05])
    v[14] = theta
    v[15:18] = ghat
    v[18] = alpha
    d1 = np.zeros((27, 3))
    d2 = np.zeros((27, 6))
    p = P(kappa1=k1, kappa2=k2, kappa3=0.7, a0=a0, b0=b0, lam=0.2, g2=0.1)
    r, _, st = orc.point_rhs(p, v, d1, d2)
    assert st == 0
    assert r[14] == pytest.approx(-alpha * k1 * (2.0 + k2) * theta / (1.0 + b0), rel=1e-14, abs=1e-15)
    # d_t Gamma-hat^i = 2 h^ij d_t Z_j = -alpha kappa1 Gamma-hat^i / (1 + b) (h static, Gamma-tilde = 0)
    np.testing.assert_allclose(r[15:18], -alpha * k1 * ghat / (1.0 + b0), rtol=1e-14, atol=1e-15)
    assert np.all(r[0:7] == 0.0)     # chi, h_ij static
    # A_ij static; K moves only by the damping terms (-3 alpha kappa1 (1 + kappa2) Theta, and the b(x)
    # term -(3 alpha b/(4 (1 + b))) (-2 kappa1 (2 + kappa2) Theta)); both pass through the oracle's
    # residual-based coupled solve, which leaves rounding far below 1e-15
    assert np.all(np.abs(r[8:14]) < 1e-15)
    kdot = -3.0 * alpha * k1 * (1.0 + k2) * theta + 1.5 * alpha * b0 / (1.0 + b0) * k1 * (2.0 + k2) * theta
    assert r[7] == pytest.approx(kdot, rel=1e-13, abs=1e-15)
    assert np.all(r[19:22] == 0.0) and r[25] == 0.0  # shift, phi
    assert abs(r[26]) < 1e-15  # Pi: zero up to the rounding of the oracle's residual-based solve
    # the same data with the damping switched off: the constraint fields do not move
    r0, _, _ = orc.point_rhs(P(kappa1=0.0, kappa2=k2, kappa3=0.7, a0=a0, b0=b0, lam=0.2, g2=0.1), v, d1, d2)
    assert r0[14] == 0.0 and np.all(r0[15:18] == 0.0)


@pytest.mark.parametrize("k3", [0.0, 0.5, 1.0])
def test_z_part_of_gamma_hat_is_shift_transported_by_kappa3(orc, k3):
    """The same flat slice with a constant Z_i and a shift whose gradient M^i_k = d_k beta^i is
    constant (beta = 0 at the point). The conformal Christoffels, all second derivatives and every
    gradient of the other fields vanish, so the Gamma-hat^i equation keeps only the damping and
    the transport of its Z part: kappa3 = 1 transports 2 h^ij Z_j by the shift exactly as
    Gamma-tilde^i is transported, i.e. as a vector density of weight 2/3 (2/3 G^i tr M - G^k M^i_k);
    kappa3 scales that transport. Catches a wrong kappa3 placement, a transposed M, or a 2/3
    weight error."""
    alpha, k1 = 0.9, 0.2
    v = np.zeros(27)
    v[0] = 0.8
    v[1], v[4], v[6] = 1.0, 1.0, 1.0
    ghat = np.array([0.3, -0.2, 0.1])
    v[15:18] = ghat
    v[18] = alpha
    d1 = np.zeros((27, 3))
    M = np.array([[0.2, -0.1, 0.05], [0.3, 0.1, -0.2], [-0.15, 0.25, 0.4]])  # M[i][k] = d_k beta^i
    for i in range(3):
        d1[19 + i, :] = M[i]
    d2 = np.zeros((27, 6))
    p = P(kappa1=k1, kappa2=0.1, kappa3=k3)
    r, _, st = orc.point_rhs(p, v, d1, d2)
    assert st == 0
    # damping at the modified gauge's rate -alpha kappa1 / (1 + b) (see the flat-slice damping pin)
    expect = -alpha * k1 * ghat / (1.0 + p.b0) + k3 * ((2.0 / 3.0) * ghat * np.trace(M) - M @ ghat)
    np.testing.assert_allclose(r[15:18], expect, rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------------------------- covariant Z4
@pytest.fixture(scope="module")
def z4_point():
    return an.z4_point_data((0.0, 0.37, -0.52, 0.81))


# fields whose time derivative the spacetime fixes (the gauge fields and B^i evolve by choice)
Z4_FIELDS = list(range(0, 18)) + [25, 26]
Z4_CASES = [  # b, kappa1, kappa2, lambda, g2, beta kind[, g3]
    (0.0, 0.0, 0.0, 0.0, 0.0, 0), (0.0, 0.3, 0.4, 0.0, 0.0, 0), (0.4, 0.0, 0.0, 0.0, 0.0, 0),
    (0.4, 0.3, 0.4, 0.0, 0.0, 0), (1.1, 0.2, -0.3, 0.0, 0.0, 0), (0.4, 0.1, 0.0, 0.7, 0.3, 0),
    (0.4, 0.25, 0.5, 0.5, 0.2, 1), (0.0, 0.0, 0.0, 0.0, 0.0, 0, 0.6), (0.4, 0.25, 0.5, 0.5, 0.2, 1, -0.9)]


def _z4_compare(orc, D, case, variant="covariant"):
    b, k1, k2, lam, g2, kind = case[:6]
    g3 = case[6] if len(case) > 6 else 0.0
    want = an.z4_time_derivatives(D, b=b, k1=k1, k2=k2, lam=lam, g2=g2, kind=kind, variant=variant, g3=g3)
    r, _, st = orc.point_rhs(P(kappa1=k1, kappa2=k2, kappa3=1.0, a0=0.2, b0=b, lam=lam, g2=g2, beta_kind=kind,
                               g3=g3), D["v"], D["d1"], D["d2"])
    assert st == 0
    return np.abs(r[Z4_FIELDS] - want[Z4_FIELDS]) / np.maximum(1.0, np.abs(want[Z4_FIELDS]))


@pytest.mark.parametrize("case", Z4_CASES)
def test_ccz4_is_the_3p1_projection_of_covariant_modified_z4(orc, z4_point, case):
    """On a generic spacetime with a generic Z4 vector (Theta, Z_i, the constraints and every
    gradient non-zero; lapse and shift non-trivial) the covariant equations
        G^mn + 2 Phat_a^{b mn} nabla_b Z^a - kappa1 [2 n^(m Z^n) + kappa2 (n.Z) g^mn] = 8 pi T^mn,
        Phat_a^{b mn} = delta_a^(m gh^n)b - 1/2 delta_a^b gh^mn,  gh^mn = g^mn - b n^m n^n,
    together with the 4dST scalar equation, are solved at one point for the 11 second time
    derivatives (of gamma_ij, Z_a and phi) that they fix, in a brute-force 4D coordinate
    computation (numpy Christoffels and Riemann of the 4-metric). The resulting exact time
    derivatives of chi, h_ij, K, A_ij, Theta, Gamma-hat^i, phi and Pi must equal the oracle's
    3+1 right-hand sides. b = 0 with kappa1, kappa2 != 0 pins the damping terms, including
    -3 alpha kappa1 (1 + kappa2) Theta in d_t K; b != 0 pins every b(x) term of the modified
    gauge in d_t K, d_t Theta and d_t Gamma-hat; lambda, g2 != 0 pin the 4dST matter terms
    inside them, and g3 != 0 the cubic Horndeski term g3 X box(phi) (its stress tensor in the
    metric equations and its share of the scalar equation, solved together with them)."""
    err = _z4_compare(orc, z4_point, case)
    assert np.max(err) < 1e-11, dict(zip(Z4_FIELDS, err))


@pytest.mark.parametrize("variant,case", [("b_half", Z4_CASES[3]), ("b_half", Z4_CASES[6]),
                                          ("g3_half", Z4_CASES[7]), ("g3_half", Z4_CASES[8]),
                                          ("gh_first_only", Z4_CASES[3]), ("k2_moved", Z4_CASES[1]),
                                          ("k2_moved", Z4_CASES[4])])
def test_covariant_z4_pin_discriminates(orc, z4_point, variant, case):
    """The same comparison with a planted change in the covariant equation (half the b(x)
    coefficient; g instead of gh in the trace term of Phat; 1 + kappa2 in place of kappa2 in the
    damping; half the cubic coefficient in the stress tensor) must fail by far more than the
    tolerance: the pin above sees each of these terms."""
    err = _z4_compare(orc, z4_point, case, variant)
    assert np.max(err) > 1e-6


# ----------------------------------------------------------------------------- P3 stencils
def _poly(X, Y, Z, coef, deg):
    out = np.zeros_like(X)
    terms = []
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                terms.append((a, b, c))
    for (a, b, c), k in zip(terms, coef):
        out += k * X ** a * Y ** b * Z ** c
    return out, terms


def _poly_deriv(X, Y, Z, coef, terms, d):
    """d: tuple of derivative orders (dx, dy, dz)."""
    out = np.zeros_like(X)
    for (a, b, c), k in zip(terms, coef):
        if a < d[0] or b < d[1] or c < d[2]:
            continue
        fa = math.factorial(a) / math.factorial(a - d[0])
        fb = math.factorial(b) / math.factorial(b - d[1])
        fc = math.factorial(c) / math.factorial(c - d[2])
        out += k * fa * fb * fc * X ** (a - d[0]) * Y ** (b - d[1]) * Z ** (c - d[2])
    return out


def test_stencils_exact_on_quartic_polynomials(orc):
    """First, second and mixed 4th-order stencils are exact on every monomial of total degree
    <= 4. Catches a wrong stencil weight, a wrong 1/(12 dx) or 1/(144 dx^2) scale, or a
    transposed mixed-derivative index."""
    b = gi.Box(7, 6, 5, 0.3, -0.4, 0.2, 0.5, bc=gi.BC_FROZEN)
    X, Y, Z = b.coords()
    rng = np.random.default_rng(1)
    s = np.zeros(b.shape)
    coefs = []
    for f in range(27):
        coef = rng.uniform(-1, 1, 35)
        coefs.append(coef)
        s[f], terms = _poly(X, Y, Z, coef, 4)
    d1, d2 = orc.derivs(b, s)
    Xi, Yi, Zi = (b.interior(a) for a in (X, Y, Z))
    for f in range(27):
        for d in range(3):
            o = [0, 0, 0]
            o[d] = 1
            ex = _poly_deriv(Xi, Yi, Zi, coefs[f], terms, o)
            assert np.max(np.abs(d1[f, d] - ex)) <= 1e-12 * max(1.0, np.max(np.abs(ex)))
        for m, (p, q) in enumerate(an.SYM_PAIRS):
            o = [0, 0, 0]
            o[p] += 1
            o[q] += 1
            ex = _poly_deriv(Xi, Yi, Zi, coefs[f], terms, o)
            assert np.max(np.abs(d2[f, m] - ex)) <= 1e-11 * max(1.0, np.max(np.abs(ex)))


def test_stencils_converge_at_fourth_order(orc):
    """Halving dx on a smooth periodic field divides the first/second/mixed derivative errors
    by ~16 (4th order). Catches a stencil that is only 2nd-order accurate."""
    errs = []
    for n in (16, 32):
        b = gi.cube_box(n, 0.0, 2.0)
        X, Y, Z = b.coords()
        k = math.pi
        s = np.zeros(b.shape)
        s[0] = np.sin(k * X) * np.cos(k * Y) * np.sin(k * Z + 0.3)
        orc.fill_ghosts(b, s)
        d1, d2 = orc.derivs(b, s)
        Xi, Yi, Zi = (b.interior(a) for a in (X, Y, Z))
        ex_x = k * np.cos(k * Xi) * np.cos(k * Yi) * np.sin(k * Zi + 0.3)
        ex_xx = -k * k * np.sin(k * Xi) * np.cos(k * Yi) * np.sin(k * Zi + 0.3)
        ex_xy = -k * k * np.cos(k * Xi) * np.sin(k * Yi) * np.sin(k * Zi + 0.3)
        errs.append([np.max(np.abs(d1[0, 0] - ex_x)), np.max(np.abs(d2[0, 0] - ex_xx)),
                     np.max(np.abs(d2[0, 1] - ex_xy))])
    ratios = np.array(errs[0]) / np.array(errs[1])
    assert np.all(ratios > 14.0) and np.all(ratios < 18.0), ratios


def test_ko_annihilates_quintics_and_damps_nyquist(orc):
    """KO: sigma/(64 dx) sum_d Delta^6_d u is zero on degree-5 polynomials and gives exactly
    -sigma/dx * u per direction on the Nyquist mode. Catches a wrong sign (anti-damping),
    a missing 1/64 or the wrong binomial weights."""
    b = gi.Box(8, 7, 6, 0.25, 0.1, -0.3, 0.2, bc=gi.BC_FROZEN)
    X, Y, Z = b.coords()
    rng = np.random.default_rng(7)
    s = np.zeros(b.shape)
    for f in range(27):
        s[f], _ = _poly(X, Y, Z, rng.uniform(-1, 1, 56), 5)
    r = orc.ko(b, 0.3, s)
    assert np.max(np.abs(b.interior(r))) < 1e-9
    ii = np.arange(b.nx + 6)[None, None, :]
    s = np.zeros(b.shape)
    s[:] = np.where(ii % 2 == 0, 1.0, -1.0)
    r = orc.ko(b, 0.3, s)
    np.testing.assert_allclose(b.interior(r), -0.3 / b.dx * b.interior(s), rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------- 6th order, lopsided advection
# ("Accuracy": 4th- and 6th-order stencils.) A box with 4 ghost layers takes the 6th-order scheme.
NYQ_LOPSIDED = {3: -32.0 / 12.0, 4: -128.0 / 60.0}     # symbol of the lopsided stencil at the Nyquist mode
NYQ_SECOND = {3: -64.0 / 12.0, 4: -1088.0 / 180.0}     # ... of the centred second derivative


def test_sixth_order_stencils_exact_on_sextic_polynomials(orc):
    """With ng = 4 the first, second and mixed stencils are exact on every monomial of total
    degree <= 6. Catches a wrong 6th-order weight, a wrong 1/(60 dx), 1/(180 dx^2) or
    1/(3600 dx^2) scale, or a stencil still of 4th order (not exact on degree 5 and 6)."""
    b = gi.Box(6, 5, 5, 0.3, -0.4, 0.2, 0.5, bc=gi.BC_FROZEN, ng=4)
    X, Y, Z = b.coords()
    rng = np.random.default_rng(11)
    s = np.zeros(b.shape)
    coefs = []
    for f in range(27):
        coef = rng.uniform(-1, 1, 84)
        coefs.append(coef)
        s[f], terms = _poly(X, Y, Z, coef, 6)
    d1, d2 = orc.derivs(b, s)
    Xi, Yi, Zi = (b.interior(a) for a in (X, Y, Z))
    for f in range(27):
        for d in range(3):
            o = [0, 0, 0]
            o[d] = 1
            ex = _poly_deriv(Xi, Yi, Zi, coefs[f], terms, o)
            assert np.max(np.abs(d1[f, d] - ex)) <= 1e-11 * max(1.0, np.max(np.abs(ex)))
        for m, (p, q) in enumerate(an.SYM_PAIRS):
            o = [0, 0, 0]
            o[p] += 1
            o[q] += 1
            ex = _poly_deriv(Xi, Yi, Zi, coefs[f], terms, o)
            assert np.max(np.abs(d2[f, m] - ex)) <= 1e-10 * max(1.0, np.max(np.abs(ex)))


def test_sixth_order_stencils_converge_at_sixth_order(orc):
    """Halving dx on a smooth periodic field divides the 6th-order first/second/mixed derivative
    errors by ~64."""
    errs = []
    for n in (16, 32):
        b = gi.Box(n, n, n, 2.0 / n, 1.0 / n, 1.0 / n, 1.0 / n, ng=4)
        X, Y, Z = b.coords()
        k = math.pi
        s = np.zeros(b.shape)
        s[0] = np.sin(k * X) * np.cos(k * Y) * np.sin(k * Z + 0.3)
        orc.fill_ghosts(b, s)
        d1, d2 = orc.derivs(b, s)
        Xi, Yi, Zi = (b.interior(a) for a in (X, Y, Z))
        ex_x = k * np.cos(k * Xi) * np.cos(k * Yi) * np.sin(k * Zi + 0.3)
        ex_xx = -k * k * np.sin(k * Xi) * np.cos(k * Yi) * np.sin(k * Zi + 0.3)
        ex_xy = -k * k * np.cos(k * Xi) * np.sin(k * Yi) * np.sin(k * Zi + 0.3)
        errs.append([np.max(np.abs(d1[0, 0] - ex_x)), np.max(np.abs(d2[0, 0] - ex_xx)),
                     np.max(np.abs(d2[0, 1] - ex_xy))])
    ratios = np.array(errs[0]) / np.array(errs[1])
    assert np.all(ratios > 56.0) and np.all(ratios < 72.0), ratios


def test_ko8_annihilates_septics_and_damps_nyquist(orc):
    """The 6th-order scheme's dissipation -sigma/(256 dx) sum_d Delta^8_d u is zero on degree-7
    polynomials and gives exactly -sigma/dx * u per direction on the Nyquist mode. Catches the
    anti-damping sign (Delta^8 is positive on that mode), a missing 1/256 or wrong binomials."""
    b = gi.Box(6, 5, 5, 0.25, 0.1, -0.3, 0.2, bc=gi.BC_FROZEN, ng=4)
    X, Y, Z = b.coords()
    rng = np.random.default_rng(8)
    s = np.zeros(b.shape)
    for f in range(27):
        s[f], _ = _poly(X, Y, Z, rng.uniform(-1, 1, 120), 7)
    r = orc.ko(b, 0.3, s)
    assert np.max(np.abs(b.interior(r))) < 1e-8
    for axis in range(3):
        idx = np.indices(b.shape[1:])[2 - axis]
        s = np.zeros(b.shape)
        s[:] = np.where(idx % 2 == 0, 1.0, -1.0)
        r = orc.ko(b, 0.3, s)
        np.testing.assert_allclose(b.interior(r), -0.3 / b.dx * b.interior(s), rtol=0, atol=1e-12)


def _nyquist_scalar(ng, axis, shift):
    """Flat slice, constant shift component `shift` along `axis`, Pi = 0 and phi = 1e-3 (-1)^i
    along that axis (the grid's Nyquist mode), on all points including the ghosts."""
    b = gi.Box(6, 6, 6, 0.2, 0.0, 0.0, 0.0, bc=gi.BC_FROZEN, ng=ng)
    s = gi.flat_state(b)
    idx = np.indices(b.shape[1:])[2 - axis]
    s[25] = 1e-3 * np.where(idx % 2 == 0, 1.0, -1.0)
    s[19 + axis] = shift
    return b, s


@pytest.mark.parametrize("ng", [3, 4])
@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("shift", [0.3, -0.45])
def test_lopsided_advection_damps_the_nyquist_mode(orc, ng, axis, shift):
    """On the Nyquist mode the centred first derivative vanishes, so with centred advection
    d_t phi = 0; the lopsided stencil, biased towards the side the shift points to, damps it:
    d_t phi = -|beta| c / dx phi with c = 8/3 (4th order) or 32/15 (6th order), for either sign
    of the shift. A stencil biased the wrong way gives +|beta| c / dx (growth). d_t Pi is the
    centred second derivative: -16/3 / dx^2 phi (4th order), -272/45 / dx^2 phi (6th order)."""
    b, s = _nyquist_scalar(ng, axis, shift)
    zero = P(lam=0.0, g2=0.0)
    r0 = orc.rhs(b, zero, s, with_ko=False)
    rl = orc.rhs(b, P(lam=0.0, g2=0.0, advection=1), s, with_ko=False)
    phi = b.interior(s)[25]
    assert np.max(np.abs(b.interior(r0)[25])) < 1e-15
    np.testing.assert_allclose(b.interior(rl)[25], NYQ_LOPSIDED[ng] * abs(shift) / b.dx * phi, rtol=1e-12, atol=0)
    for r in (r0, rl):
        np.testing.assert_allclose(b.interior(r)[26], NYQ_SECOND[ng] / b.dx ** 2 * phi, rtol=1e-12, atol=0)
        others = np.delete(b.interior(r), [25, 26], axis=0)   # zero up to the solve's rounding
        assert np.max(np.abs(others)) < 1e-13 * np.max(np.abs(b.interior(r)[26]))


@pytest.mark.parametrize("ng,deg", [(3, 4), (4, 6)])
def test_lopsided_equals_centred_on_polynomial_data(orc, ng, deg):
    """Both stencils are exact on polynomials of degree <= the scheme's order, so on a state whose
    27 fields are such polynomials (a perturbed flat slice with a shift that changes sign inside
    the box, couplings on) the lopsided and centred right-hand sides agree to rounding. Catches a
    wrong lopsided weight, scale or offset, and a wrong chain rule of the shift-contracted
    derivative of K_ij inside the coupled system."""
    b = gi.Box(5, 5, 4, 0.25, -0.5, -0.45, -0.4, bc=gi.BC_FROZEN, ng=ng)
    X, Y, Z = b.coords()
    rng = np.random.default_rng(20 + ng)
    nterm = len(_poly(X, Y, Z, np.zeros(200), deg)[1])
    s = gi.flat_state(b)
    for f in range(27):
        amp = 0.3 if f in (19, 20, 21, 25, 26) else 0.02
        s[f] += _poly(X, Y, Z, amp * rng.uniform(-1, 1, nterm), deg)[0]
    for f in range(19, 22):
        s[f] += 0.4 * (X, Y, Z)[f - 19]   # sign changes across the box
    p = dict(lam=0.3, g2=0.2, beta_kind=1)
    rc = b.interior(orc.rhs(b, P(**p), s, with_ko=False))
    rl = b.interior(orc.rhs(b, P(advection=1, **p), s, with_ko=False))
    scale = np.maximum(np.max(np.abs(rc), axis=(1, 2, 3)), 1e-3)
    err = np.max(np.abs(rl - rc), axis=(1, 2, 3)) / scale
    assert np.max(err) < 1e-11, err
    adv = orc.adv_lopsided(b, s)
    assert np.any(b.interior(s)[19] > 0) and np.any(b.interior(s)[19] < 0)
    assert np.all(np.isfinite(adv))


@pytest.mark.parametrize("ng,ratio", [(3, 16.0), (4, 64.0)])
def test_lopsided_advection_converges_at_the_scheme_order(orc, ng, ratio):
    """beta^k d_k u with the lopsided stencils, on smooth periodic fields and a shift of either
    sign, converges to the exact value with the scheme's order (error ratio ~2^order)."""
    errs = []
    for n in (16, 32):
        b = gi.Box(n, n, n, 2.0 / n, 1.0 / n, 1.0 / n, 1.0 / n, ng=ng)
        X, Y, Z = b.coords()
        k = math.pi
        s = gi.flat_state(b)
        s[0] = 1.0 + 0.1 * np.sin(k * X) * np.cos(k * Y) * np.sin(k * Z + 0.3)
        s[19] = 0.5 * np.sin(k * Y + 0.2)
        s[20] = 0.5 * np.cos(k * Z)
        s[21] = 0.5 * np.sin(k * X - 0.4)
        orc.fill_ghosts(b, s)
        adv = orc.adv_lopsided(b, s)
        Xi, Yi, Zi = (b.interior(a) for a in (X, Y, Z))
        ex = 0.1 * k * (0.5 * np.sin(k * Yi + 0.2) * np.cos(k * Xi) * np.cos(k * Yi) * np.sin(k * Zi + 0.3)
                        - 0.5 * np.cos(k * Zi) * np.sin(k * Xi) * np.sin(k * Yi) * np.sin(k * Zi + 0.3)
                        + 0.5 * np.sin(k * Xi - 0.4) * np.sin(k * Xi) * np.cos(k * Yi) * np.cos(k * Zi + 0.3))
        errs.append(np.max(np.abs(adv[0] - ex)))
    r = errs[0] / errs[1]
    assert 0.8 * ratio < r < 1.25 * ratio, errs


# ----------------------------------------------------------------------------- outer boundaries
# ("Boundary Conditions": extrapolating and Sommerfeld.)
@pytest.mark.parametrize("ng", [3, 4])
def test_extrapolating_ghosts_are_linear_extrapolations(orc, ng):
    """Every ghost of an extrapolating box is exact on affine data, and on u = x^2 + 2 y^2 - z^2
    it misses by exactly -(mx(mx+1) + 2 my(my+1) - mz(mz+1)) dx^2, m the distance (in points)
    beyond the face along each axis: catches a wrong distance, a wrong sign or a non-linear
    formula, and an interior point overwritten."""
    b = gi.Box(6, 5, 7, 0.2, 0.3, -0.4, 0.1, bc=gi.BC_EXTRAPOLATE, ng=ng)
    X, Y, Z = b.coords()
    s = np.zeros(b.shape)
    s[0] = 0.7 + 1.3 * X - 0.4 * Y + 2.1 * Z
    s[1] = X ** 2 + 2 * Y ** 2 - Z ** 2
    s[2:] = 1.0
    ref = s.copy()
    t = s.copy()
    t[:, :ng] = np.nan
    t[:, -ng:] = np.nan
    t[:, :, :ng] = np.nan
    t[:, :, -ng:] = np.nan
    t[..., :ng] = np.nan
    t[..., -ng:] = np.nan
    orc.fill_ghosts(b, t)
    np.testing.assert_allclose(t[0], ref[0], rtol=0, atol=1e-13)
    def beyond(n, N):
        i = np.arange(N)
        return np.where(i < ng, ng - i, np.where(i >= ng + n, i - (ng + n - 1), 0))
    mz, my, mx = np.meshgrid(beyond(b.nz, b.nz + 2 * ng), beyond(b.ny, b.ny + 2 * ng), beyond(b.nx, b.nx + 2 * ng),
                             indexing="ij")
    miss = -(mx * (mx + 1) + 2 * my * (my + 1) - mz * (mz + 1)) * b.dx ** 2
    np.testing.assert_allclose(t[1] - ref[1], miss, rtol=0, atol=1e-12)
    assert np.array_equal(b.interior(t), b.interior(ref))


def _outgoing(b, amp=1e-6, r0=2.5, w=0.3, t=0.0):
    """Flat slice with phi = A f(r - t) / r and Pi = d_t phi, f a Gaussian pulse: an exact
    outgoing solution of the scalar wave equation, and of the Sommerfeld condition."""
    s = gi.flat_state(b)
    X, Y, Z = b.coords()
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    f = np.exp(-((r - t - r0) / w) ** 2)
    fp = -2 * (r - t - r0) / w ** 2 * f
    s[25] = amp * f / r
    s[26] = -amp * fp / r
    return s, r, f, fp


def test_sommerfeld_rhs_is_exact_for_outgoing_waves_to_second_order(orc):
    """At the ghosts of a Sommerfeld box the right-hand side of u = u_inf + A f(r - t)/r is
    -A f'(r - t)/r up to the one-sided differences' error (ratio ~4 per halving); for the static
    u = u_inf + c/r it is 0 to the same order; asymptotic values give exactly 0."""
    errs, errs_static = [], []
    for n in (16, 32):
        b = gi.Box(n, n, n, 1.0 / n, 2.0 + 0.5 / n, 0.5 / n, 1.0 + 0.5 / n, bc=gi.BC_SOMMERFELD)
        s, r, f, fp = _outgoing(b)
        rhs = orc.rhs(b, gi.Params(lam=0.0, g2=0.0), s)
        ghost = np.ones(r.shape, bool)
        ghost[b.ng:-b.ng, b.ng:-b.ng, b.ng:-b.ng] = False
        errs.append(np.max(np.abs(rhs[25][ghost] - (-1e-6 * fp / r)[ghost])) / 1e-6)
        assert np.max(np.abs(rhs[:25][:, ghost])) == 0.0  # the asymptotic values are steady
        s2 = gi.flat_state(b)
        s2[18] = 1.0 + 0.3 / r  # lapse
        rhs2 = orc.rhs(b, gi.Params(lam=0.0, g2=0.0), s2)
        errs_static.append(np.max(np.abs(rhs2[18][ghost])))
    assert 3.3 < errs[0] / errs[1] < 4.8, errs
    assert 3.3 < errs_static[0] / errs_static[1] < 4.8, errs_static


def test_sommerfeld_box_evolves_an_outgoing_wave(orc):
    """A scalar pulse leaving a box that contains the origin (the radiative condition holds on
    outer faces, where x^i/r points out of the box and the inward one-sided differences are
    upwind): with Sommerfeld ghosts evolved by the RK4 stages the interior follows the exact
    solution at 2nd order (ratio ~3.2 at these resolutions, tending to 4), while frozen ghosts
    leave an error 35x larger that does not converge."""
    T, r0, w = 0.5, 2.3, 0.5
    errs, frozen = [], []
    for n in (40, 80):
        dx = 5.0 / n
        for bc, out in ((gi.BC_SOMMERFELD, errs), (gi.BC_FROZEN, frozen)):
            b = gi.Box(n, 4, 4, dx, -2.5 + 0.5 * dx, -1.5 * dx, -1.5 * dx, bc=bc)
            s, *_ = _outgoing(b, r0=r0, w=w)
            dt = 0.25 * dx
            nsteps = int(round(T / dt))
            orc.rk4(b, gi.Params(lam=0.0, g2=0.0), s, dt, nsteps)
            ex, *_ = _outgoing(b, r0=r0, w=w, t=nsteps * dt)
            out.append(np.max(np.abs(b.interior(s)[25] - b.interior(ex)[25])) / 1e-6)
    assert 2.7 < errs[0] / errs[1] < 4.5, errs
    assert frozen[1] > 20 * errs[0] and frozen[0] / frozen[1] < 1.5, (frozen, errs)


def test_octant_with_sommerfeld_faces_reproduces_the_full_box(orc):
    """Mirror planes at the low faces with Sommerfeld high faces (bc 5): an octant of a state with
    the three reflection symmetries, evolved 2 RK4 steps, equals the positive octant of the full
    Sommerfeld box (bc 4) evolved alike, at the interior and at the evolved high-face ghosts.
    Catches an image of a high-face ghost missing, a ghost evolved that should be an image, and a
    one-sided difference where the mirror plane makes the centred one right."""
    n, dx = 6, 0.3
    full = gi.Box(2 * n, 2 * n, 2 * n, dx, -(n - 0.5) * dx, -(n - 0.5) * dx, -(n - 0.5) * dx, bc=gi.BC_SOMMERFELD)
    octb = gi.Box(n, n, n, dx, 0.5 * dx, 0.5 * dx, 0.5 * dx, bc=gi.BC_REFLECT_LOW_SOMMERFELD)
    s_full = gi.mirror_symmetric_state(full)
    s_oct = gi.mirror_symmetric_state(octb)
    p = P(lam=0.2, g2=0.1, beta_kind=1)
    dt = 0.25 * dx
    orc.rk4(full, p, s_full, dt, 2)
    orc.rk4(octb, p, s_oct, dt, 2)
    g = full.ng
    # octant points (ghosted index) i >= g map to full-box index i + n
    ref = s_full[:, g + n:, g + n:, g + n:]
    got = s_oct[:, g:, g:, g:]
    scale = np.maximum(np.max(np.abs(ref), axis=(1, 2, 3)), 1e-12)
    err = np.max(np.abs(got - ref), axis=(1, 2, 3)) / scale
    assert np.max(err) < 1e-12, err
    # the same octant with frozen high faces differs
    s_frz = gi.mirror_symmetric_state(octb)
    frz = gi.Box(n, n, n, dx, 0.5 * dx, 0.5 * dx, 0.5 * dx, bc=gi.BC_REFLECT_LOW)
    orc.rk4(frz, p, s_frz, dt, 2)
    assert np.max(np.abs(s_frz[:, g:, g:, g:] - ref)) > 1e-6


# ----------------------------------------------------------------------------- waveform extraction
# ("Diagnostics": tensor and scalar waveforms, extracted on spheres.)
def test_gauss_legendre_rule_matches_the_library(orc):
    for n in (1, 2, 5, 12, 33):
        x, w = orc.gauss_legendre(n)
        X, W = np.polynomial.legendre.leggauss(n)
        np.testing.assert_allclose(np.sort(x), np.sort(X), rtol=0, atol=1e-14)
        np.testing.assert_allclose(w[np.argsort(x)], W[np.argsort(X)], rtol=1e-13, atol=0)


def test_spin_weighted_harmonics(orc):
    """s = 0 equals the library's Y_lm; s = -2, l = 2 equals its closed forms; both families are
    orthonormal under the extraction's quadrature (catches a wrong normalisation, phase or
    quadrature weight)."""
    sph = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(4)
    for _ in range(5):
        th, ph = rng.uniform(0.05, math.pi - 0.05), rng.uniform(0, 2 * math.pi)
        for l in range(7):
            for m in range(-l, l + 1):
                ref = sph.sph_harm_y(l, m, th, ph)
                assert abs(orc.sylm(0, l, m, th, ph) - ref) < 1e-12
        c = math.cos(th)
        closed = {2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2, 1: math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 + c),
                  0: math.sqrt(15 / (32 * math.pi)) * math.sin(th) ** 2,
                  -1: math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 - c),
                  -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2}
        for m, a in closed.items():
            assert abs(orc.sylm(-2, 2, m, th, ph) - a * np.exp(1j * m * ph)) < 1e-12
    mu, w = orc.gauss_legendre(8)
    nphi = 16
    for s in (0, -2):
        lm = [(l, m) for l in range(abs(s), 7) for m in range(-l, l + 1)]
        Y = np.array([[orc.sylm(s, l, m, math.acos(x), 2 * math.pi * j / nphi) for x in mu for j in range(nphi)]
                      for (l, m) in lm])
        wq = np.repeat(w, nphi) * 2 * math.pi / nphi
        G = (Y * wq) @ Y.conj().T
        np.testing.assert_allclose(G, np.eye(len(lm)), rtol=0, atol=1e-12)


def _solid_harmonic_box(l, m, centre, ng=3):
    sph = pytest.importorskip("scipy.special")
    b = gi.Box(20, 18, 19, 0.2, -1.9, -1.7, -1.8, bc=gi.BC_FROZEN, ng=ng)
    X, Y, Z = b.coords()
    dx, dy, dz = X - centre[0], Y - centre[1], Z - centre[2]
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    th = np.arccos(np.clip(np.where(r > 0, dz / np.where(r > 0, r, 1), 1.0), -1, 1))
    ph = np.arctan2(dy, dx)
    f = r ** l * sph.sph_harm_y(l, m, th, ph)
    return b, np.ascontiguousarray(f.real), np.ascontiguousarray(f.imag)


@pytest.mark.parametrize("lm", [(0, 0), (1, -1), (2, 1), (3, 3), (3, -2)])
def test_extraction_is_exact_on_solid_harmonics(orc, lm):
    """r^l Y_lm (l <= 3) is a polynomial of degree <= 3 along each axis, which the cubic
    interpolation reproduces; the quadrature is exact for the band limit. So the modes are
    exactly R^l at (l, m) and 0 elsewhere; a real field Re(r^l Y_lm) splits into R^l / 2 at
    (l, m) and (-1)^m R^l / 2 at (l, -m)."""
    l, m = lm
    c = (0.13, -0.07, 0.21)
    R = 1.1
    b, fre, fim = _solid_harmonic_box(l, m, c)
    a = orc.extract_modes(b, fre, fim, 0, R, c, 8, 16, 4)
    ref = np.zeros(25, complex)
    ref[l * l + l + m] = R ** l
    np.testing.assert_allclose(a, ref, rtol=0, atol=1e-12)
    a = orc.extract_modes(b, fre, None, 0, R, c, 8, 16, 4)
    ref = np.zeros(25, complex)
    ref[l * l + l + m] += R ** l / 2
    ref[l * l + l - m] += (-1) ** m * R ** l / 2
    np.testing.assert_allclose(a, ref, rtol=0, atol=1e-12)


def test_sphere_interpolation_is_fourth_order(orc):
    """The 4-point Lagrange interpolant at random points: pointwise error ratio ~16 per halving
    of dx on a smooth field, and exact on cubics along each axis."""
    rng = np.random.default_rng(9)
    pts = rng.uniform(-0.9, 0.9, size=(200, 3))
    errs = []
    for dx in (0.1, 0.05):
        n = int(round(3.0 / dx))
        b = gi.Box(n, n, n, dx, -1.5 + 0.5 * dx, -1.5 + 0.5 * dx, -1.5 + 0.5 * dx, bc=gi.BC_FROZEN)
        X, Y, Z = b.coords()
        f = np.sin(2 * X + 0.3) * np.cos(1.5 * Y) * np.exp(0.5 * Z)
        ex = np.sin(2 * pts[:, 0] + 0.3) * np.cos(1.5 * pts[:, 1]) * np.exp(0.5 * pts[:, 2])
        errs.append(np.max(np.abs(orc.interp(b, f, pts) - ex)))
        cub = (X ** 3 - 2 * X) * (Y ** 3 + Y ** 2) * (1 - Z ** 3)
        ex_c = (pts[:, 0] ** 3 - 2 * pts[:, 0]) * (pts[:, 1] ** 3 + pts[:, 1] ** 2) * (1 - pts[:, 2] ** 3)
        np.testing.assert_allclose(orc.interp(b, cub, pts), ex_c, rtol=0, atol=1e-13)
    assert 13 < errs[0] / errs[1] < 19, errs


def test_spin_minus_two_extraction_converges(orc):
    """A field equal to -2Y_22 of the direction from the centre (smooth near the sphere): the
    extracted a_22 tends to 1 and every other mode to 0, at least at the interpolation's 4th
    order (the sphere integral cancels part of the pointwise error, so the ratio can be larger)."""
    errs = []
    for dx in (0.1, 0.05):
        n = int(round(3.2 / dx))
        b = gi.Box(n, n, n, dx, -1.6 + 0.5 * dx, -1.6 + 0.5 * dx, -1.6 + 0.5 * dx, bc=gi.BC_FROZEN)
        X, Y, Z = b.coords()
        r = np.sqrt(X * X + Y * Y + Z * Z)
        c = Z / r
        f = math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2 * np.exp(2j * np.arctan2(Y, X))
        a = orc.extract_modes(b, np.ascontiguousarray(f.real), np.ascontiguousarray(f.imag), -2, 1.0,
                              (0.0, 0.0, 0.0), 10, 20, 4)
        ref = np.zeros(25, complex)
        ref[2 * 2 + 2 + 2] = 1.0
        errs.append(np.max(np.abs(a - ref)))
    assert errs[1] < 1e-4
    assert errs[0] / errs[1] > 12, errs


# ----------------------------------------------------------------------------- P9 solve
def test_full_pivot_solve(orc):
    """The long-double full-pivot elimination solves random systems (residual < 1e-14 relative,
    agreement with LAPACK), handles a pivot-requiring system and reports a singular one."""
    rng = np.random.default_rng(3)
    for n in (6, 7):
        for _ in range(20):
            M = rng.normal(size=(n, n))
            x0 = rng.normal(size=n)
            r = M @ x0
            x, st = orc.solve(M, r)
            assert st == 0
            assert np.max(np.abs(M @ x - r)) <= 1e-13 * np.max(np.abs(r))
            np.testing.assert_allclose(x, np.linalg.solve(M, r), rtol=1e-10, atol=1e-12)
    M = np.eye(7)[::-1].copy()          # zero diagonal: needs pivoting
    x, st = orc.solve(M, np.arange(7.0))
    assert st == 0 and np.allclose(x, np.arange(7.0)[::-1])
    M = np.ones((7, 7))
    x, st = orc.solve(M, np.ones(7))
    assert st == -1


# ----------------------------------------------------------------------------- KS stationarity
KS_POINTS = [(1.3, -0.7, 2.1), (-2.2, 1.9, 0.6), (0.8, 1.1, -1.4)]


@pytest.fixture(scope="module")
def ks_data():
    fields, X = an.kerr_schild_fields(M=1.0)
    return [an.conformal_point(fields, pt, X) for pt in KS_POINTS]


def test_kerr_schild_is_stationary(orc, ks_data):
    """Schwarzschild in Kerr-Schild coordinates, evolved with its own (time-independent) lapse
    and shift, has d_t of chi, h_ij, K, A_ij, Theta and Gamma-hat equal to zero. Every term of
    those six equations is non-zero on this data (K_ij, shift and lapse gradients are all
    non-trivial), so a wrong sign or factor in any of them breaks the cancellation. The
    b-terms multiply the Hamiltonian constraint, which vanishes, so b0 != 0 is used."""
    p = P(lam=0.0, g2=0.0, a0=0.2, b0=0.4)
    idx = [0] + list(range(1, 7)) + [7] + list(range(8, 14)) + [14, 15, 16, 17]
    for (v, d1, d2) in ks_data:
        rhs, diag, st = orc.point_rhs(p, v, d1, d2)
        assert st == 0
        scale = max(1.0, np.max(np.abs(d1)))
        assert np.max(np.abs(rhs[idx])) < 1e-12 * scale * 10, rhs[idx]


def test_kerr_schild_gauss_bonnet_invariant(orc, ks_data):
    """L_GB of Schwarzschild is the Kretschmann scalar 48 M^2 / r^6 (r = Kerr-Schild radius =
    areal radius) on a slice with K_ij != 0 and non-zero shift, and the scalar is sourced as
    d_t Pi = lapse * lambda * L_GB when phi = Pi = 0 (beta = lambda phi). Catches sign errors
    in the Gauss, Codazzi or Ricci-equation blocks, in L_GB, and in the scalar source."""
    lam = 1e-7
    p = P(lam=lam, g2=0.3, a0=0.2, b0=0.4)
    for (v, d1, d2), pt in zip(ks_data, KS_POINTS):
        r = math.sqrt(sum(c * c for c in pt))
        ex = 48.0 / r ** 6
        rhs, diag, st = orc.point_rhs(p, v, d1, d2)
        assert abs(diag[10] - ex) <= 1e-10 * ex
        assert abs(rhs[26] / (v[18] * lam) - ex) <= 1e-6 * ex


@pytest.mark.parametrize("lapse", ["precollapsed", "static", "unit"])
def test_isotropic_schwarzschild_gauss_bonnet_any_lapse(orc, lapse):
    """On the time-symmetric isotropic slice L_GB = 48 M^2/R^6 with R = r(1+M/2r)^2 whatever the
    lapse (it is a spacetime invariant). Catches a lapse-dependent error in the Ricci equation
    (the D_i D_j lapse term) or in the CCZ4 K / A_ij equations feeding d_t K_ij."""
    fields, X = an.isotropic_schwarzschild_fields(lapse=lapse)
    p = P(lam=1e-7, g2=0.0)
    for pt in [(0.9, 0.4, -0.3), (1.5, -1.2, 2.0)]:
        v, d1, d2 = an.conformal_point(fields, pt, X)
        rhs, diag, st = orc.point_rhs(p, v, d1, d2)
        r = math.sqrt(sum(c * c for c in pt))
        R = an.areal_radius_isotropic(r)
        ex = 48.0 / R ** 6
        assert abs(diag[10] - ex) <= 1e-10 * ex


def test_schwarzschild_scalar_source_converges_4th_order(orc):
    """Finite-difference version of the scalar source: d_t Pi / (lapse lambda) at a fixed point,
    computed on grids dx, dx/2, dx/4 with frozen analytic ghosts, converges to 48 M^2/R^6 with
    error ratios ~16 (4th order)."""
    pt = np.array([1.1, 0.7, 0.9])
    r = float(np.linalg.norm(pt))
    ex = 48.0 / an.areal_radius_isotropic(r) ** 6
    lam = 1e-8
    p = P(lam=lam, g2=0.0)
    errs = []
    for dx in (0.1, 0.05, 0.025):
        b = gi.Box(1, 1, 1, dx, pt[0], pt[1], pt[2], bc=gi.BC_FROZEN)
        s = gi.single_puncture(b, amp=0.0)
        rhs = orc.rhs(b, p, s, with_ko=False)
        val = b.interior(rhs)[26].ravel()[0] / (b.interior(s)[18].ravel()[0] * lam)
        errs.append(abs(val - ex))
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20, errs


# ----------------------------------------------------------------------------- 4D brute force
@pytest.fixture(scope="module")
def spacetime():
    T, alpha, beta_u, g, phi = an.generic_spacetime()
    g4 = an.four_metric(alpha, beta_u, g)
    at = an.lambdify_metric_derivs(g4, phi, T)
    phifn = sp.lambdify(T, phi, modules="math")
    return T, alpha, beta_u, g, phi, at, phifn


KAPPA = 0.8  # exponential coupling scale used by the brute-force pins


def _stress_at(at, phifn, pt, lam, g2, kind, g3=0.0):
    g, dg, ddg, dphi, ddphi = at(pt)
    gi4, Gam, Rdn, Ric, Rs = an.geometry4(g, dg, ddg)
    T8, E, LGB, T8gb, T8c = an.stress_and_scalar(g, gi4, Gam, Rdn, Ric, Rs, dphi, ddphi, phifn(*pt), lam, g2,
                                                 kind, KAPPA, g3=g3, parts=True)
    return g, gi4, Gam, T8, E, LGB, dphi, T8gb, T8c


@pytest.mark.parametrize("kind,g3", [(0, 0.0), (1, 0.0), (2, 0.0), (1, 0.6), (0, -0.9)])
def test_3p1_assembly_matches_4d_brute_force(orc, spacetime, kind, g3):
    """The oracle's 3+1 assembly (Gauss/Codazzi/Ricci-equation blocks in the (n, d_i) basis,
    nabla nabla phi projections, T and the scalar equation) reproduces rho, S_i, S_ij, L_GB and
    the scalar-equation residual of a brute-force 4D coordinate computation on a generic
    non-vacuum spacetime with lapse, shift, K_ij, d_t K_ij and a scalar all non-trivial; with
    g3 != 0 the cubic Horndeski term's stress tensor and scalar-equation share are included."""
    T, alpha, beta_u, g, phi, at, phifn = spacetime
    lam, g2 = 0.7, 0.3
    pt = (0.3, 0.4, -0.2, 0.5)
    ab = an.evaluate([alpha] + list(beta_u), T, pt)
    g4v, gi4, Gam, T8, E, LGB, dphi, _, _ = _stress_at(at, phifn, pt, lam, g2, kind, g3)
    a, bu = ab[0], ab[1:4]
    n_up = np.concatenate([[1.0 / a], -bu / a])
    rho8 = n_up @ T8 @ n_up
    S8 = -(T8 @ n_up)[1:]
    Sij8 = T8[1:, 1:]
    phys, u6, w = an.phys_pack_generic(alpha, beta_u, g, phi, T, pt)
    p = P(lam=lam, g2=g2, beta_kind=kind, beta_kappa=KAPPA, g3=g3)
    out = orc.phys_sources(p, phys, u6, w)
    scale = max(1.0, abs(rho8), np.max(np.abs(Sij8)))
    assert abs(out[0] - rho8) < 1e-10 * scale
    np.testing.assert_allclose(out[1:4], S8, atol=1e-10 * scale)
    np.testing.assert_allclose(out[4:10], [Sij8[i, j] for i, j in an.SYM_PAIRS], atol=1e-10 * scale)
    assert abs(out[10] - LGB) < 1e-10 * max(1.0, abs(LGB))
    assert abs(out[11] - E) < 1e-10 * max(1.0, abs(E))


def _tetrad_psi4_brute_force(g4, gi4, Rdn, Ric, Rs, alpha, beta_u, xyz):
    """Psi_4 = C(n, mbar, n, mbar) from the coordinate-basis 4D Riemann tensor: the Weyl tensor
    by its decomposition, the null tetrad from the slice normal and the gamma-orthonormalised
    (r, theta, phi) coordinate directions about the origin."""
    C = (Rdn - 0.5 * (np.einsum("ac,bd->abcd", g4, Ric) - np.einsum("ad,bc->abcd", g4, Ric)
                      - np.einsum("bc,ad->abcd", g4, Ric) + np.einsum("bd,ac->abcd", g4, Ric))
         + Rs / 6 * (np.einsum("ac,bd->abcd", g4, g4) - np.einsum("ad,bc->abcd", g4, g4)))
    gam = g4[1:, 1:]
    x, y, z = xyz
    e = [np.array([x, y, z]), np.array([x * z, y * z, -(x * x + y * y)]), np.array([-y, x, 0.0])]
    for a in range(3):
        for b in range(a):
            e[a] = e[a] - (e[a] @ gam @ e[b]) * e[b]
        e[a] = e[a] / math.sqrt(e[a] @ gam @ e[a])
    n_up = np.concatenate([[1.0 / alpha], -np.asarray(beta_u) / alpha])
    sp4 = [np.concatenate([[0.0], v]) for v in e]
    nv = (n_up - sp4[0]) / math.sqrt(2)
    mbar = (sp4[1] - 1j * sp4[2]) / math.sqrt(2)
    return np.einsum("abcd,a,b,c,d->", C, nv, mbar, nv, mbar)


def test_psi4_matches_4d_brute_force(orc, spacetime):
    """The Weyl scalar Psi_4 from the oracle's 3+1 assembly equals a brute-force 4D coordinate
    computation (Riemann from the metric, the Weyl decomposition, the tetrad built independently)
    on a generic non-vacuum spacetime: catches a wrong Riemann block, Weyl term, tetrad vector,
    normalisation or the sign of the imaginary part."""
    T, alpha, beta_u, g, phi, at, phifn = spacetime
    for pt in [(0.3, 0.4, -0.2, 0.5), (0.1, -0.6, 0.7, 0.2)]:
        g4v, dg, ddg, dphi, ddphi = at(pt)
        gi4, Gam, Rdn, Ric, Rs = an.geometry4(g4v, dg, ddg)
        ab = an.evaluate([alpha] + list(beta_u), T, pt)
        ref = _tetrad_psi4_brute_force(g4v, gi4, Rdn, Ric, Rs, ab[0], ab[1:4], pt[1:])
        phys, u6, w = an.phys_pack_generic(alpha, beta_u, g, phi, T, pt)
        got = orc.phys_psi4(P(lam=0.7, g2=0.3), phys, u6, w, np.array(pt[1:]))
        assert abs(ref) > 1e-3
        assert abs(got - ref) < 1e-10 * max(1.0, abs(ref)), (got, ref)


def test_psi4_vanishes_for_schwarzschild_with_the_radial_tetrad(orc, ks_data):
    """Schwarzschild is of Petrov type D with its principal null directions in the t-r plane:
    with the triad about the hole, Psi_4 = 0 (the evolution equations supply d_t K_ij = 0). About
    another centre the same data give Psi_4 of order 1e-4 .. 1e-2."""
    for (v, d1, d2), pt in zip(ks_data, KS_POINTS):
        p = P(lam=0.0, g2=0.0)
        assert abs(orc.point_psi4(p, v, d1, d2, np.array(pt))) < 1e-11
        off = np.array(pt) + np.array([1.0, -0.8, 0.6])
        assert abs(orc.point_psi4(p, v, d1, d2, off)) > 1e-4


@pytest.mark.parametrize("kind,g3", [(0, 0.0), (1, 0.0), (2, 0.0), (1, 0.6), (0, -0.9)])
def test_effective_stress_tensor_obeys_bianchi(spacetime, kind, g3):
    """Contracted Bianchi identity, off shell: nabla^m (8 pi T_mn) = (1/2) E d_n phi for the
    4dST effective stress tensor (with the cubic Horndeski term g3 X box(phi) where g3 != 0), on
    a generic spacetime. This fixes the Gauss-Bonnet coefficient (-4 P nabla nabla beta in
    8 pi T) relative to the first-order terms and to the scalar equation: a coefficient of -2,
    +4 or -8 fails by O(L_GB beta' d phi); likewise the cubic stress tensor relative to the
    cubic scalar-equation terms (box(phi)^2 - nabla nabla phi . nabla nabla phi - R(d phi, d phi))."""
    T, alpha, beta_u, g, phi, at, phifn = spacetime
    lam, g2 = 0.7, 0.3
    pt = np.array([0.3, 0.4, -0.2, 0.5])
    g4v, gi4, Gam, T8, E, LGB, dphi, T8gb, T8c = _stress_at(at, phifn, tuple(pt), lam, g2, kind, g3)
    h = 2e-3
    wts = {-3: -1 / 60, -2: 3 / 20, -1: -3 / 4, 1: 3 / 4, 2: -3 / 20, 3: 1 / 60}

    def divergence(gb_factor, cubic_factor=1.0):
        dT = np.zeros((4, 4, 4))  # dT[r][m][n]
        for r in range(4):
            for o, wgt in wts.items():
                q = pt.copy()
                q[r] += o * h
                res = _stress_at(at, phifn, tuple(q), lam, g2, kind, g3)
                dT[r] += wgt * (res[3] + (gb_factor - 1.0) * res[7] + (cubic_factor - 1.0) * res[8]) / h
        Tc = T8 + (gb_factor - 1.0) * T8gb + (cubic_factor - 1.0) * T8c
        cov = dT - np.einsum("lrm,ln->rmn", Gam, Tc) - np.einsum("lrn,ml->rmn", Gam, Tc)
        return np.einsum("rm,rmn->n", gi4, cov), np.max(np.abs(cov))

    rhs = 0.5 * E * dphi
    div, scale = divergence(1.0)
    tol = 1e-9 * max(1.0, scale)
    np.testing.assert_allclose(div, rhs, atol=tol)
    # discrimination: the same identity fails by far more than the tolerance when the
    # Gauss-Bonnet term carries half, or minus, its coefficient (or the cubic term half of its)
    wrongs = [(0.5, 1.0), (-1.0, 1.0)] + ([(1.0, 0.5)] if g3 else [])
    for gbf, cf in wrongs:
        div_w, _ = divergence(gbf, cf)
        assert np.max(np.abs(div_w - rhs)) > 1e3 * tol


# ----------------------------------------------------------------------------- ADM consistency
@pytest.fixture(scope="module")
def conformal_generic():
    """Generic conformal state with Theta = 0 and Gamma-hat = Gamma-tilde (Z = 0) and a scalar.
    The physical reference quantities (gamma = h/chi, its Christoffels and Ricci tensor, D_i D_j
    lapse) are computed by the numpy brute-force geometry from exact derivatives."""
    t, x, y, z = an.symbols()
    X = (x, y, z)
    chi = 0.6 + 0.1 * sp.sin(0.5 * x + 0.3 * y) * sp.cos(0.4 * z)
    h, hi = an.rotated_diag([1 + 0.1 * sp.sin(0.3 * y + 0.2 * z), 1 - 0.08 * sp.cos(0.5 * x + 0.2 * y),
                             1 + 0.07 * sp.sin(0.6 * y + 0.1 * x - 0.3 * z)])
    K = 0.2 * sp.cos(0.3 * x + 0.6 * y - 0.2 * z)
    Araw = {(0, 0): 0.1 * sp.sin(x), (0, 1): 0.05 * sp.cos(y + z), (0, 2): -0.07 * sp.sin(0.5 * z),
            (1, 1): 0.08 * sp.cos(0.3 * x + y), (1, 2): 0.04 * sp.sin(0.7 * x - z), (2, 2): -0.06 * sp.cos(0.4 * y)}
    Am = sp.Matrix(3, 3, lambda i, j: Araw[(min(i, j), max(i, j))])
    trA = sum(hi[i, j] * Am[i, j] for i in range(3) for j in range(3))
    A = Am - h * trA / 3
    Gt1 = an.christoffel_first(h, X)
    Gam = [sum(hi[j, k] * sum(hi[i, l] * Gt1[l][j][k] for l in range(3)) for j in range(3) for k in range(3))
           for i in range(3)]
    alpha = 0.8 + 0.1 * sp.sin(0.4 * x - 0.5 * y + 0.3 * z)
    beta = [0.1 * sp.sin(0.3 * y), 0.05 * sp.cos(0.5 * z + x), -0.08 * sp.sin(0.2 * x + 0.4 * y)]
    B = [0.02, -0.01, 0.03]
    phi = 0.2 * sp.sin(0.5 * x + 0.2 * y) * sp.cos(0.3 * z)
    Pi = 0.15 * sp.cos(0.4 * x - 0.3 * y + 0.2 * z)
    fields = [chi] + [h[i, j] for i, j in an.SYM_PAIRS] + [K] + [A[i, j] for i, j in an.SYM_PAIRS] + [0] \
             + Gam + [alpha] + beta + B + [phi, Pi]
    pt = (0.37, -0.52, 0.81)
    v, d1, d2 = an.conformal_point(fields, pt, X)
    g = h / chi
    Kij = (A + h * K / 3) / chi
    exprs = ([g[i, j] for i in range(3) for j in range(3)]
             + [sp.diff(g[i, j], X[k]) for k in range(3) for i in range(3) for j in range(3)]
             + [sp.diff(g[i, j], X[k], X[l]) for k in range(3) for l in range(3) for i in range(3) for j in range(3)]
             + [Kij[i, j] for i in range(3) for j in range(3)]
             + [sp.diff(Kij[i, j], X[k]) for k in range(3) for i in range(3) for j in range(3)]
             + [alpha] + [sp.diff(alpha, X[k]) for k in range(3)]
             + [sp.diff(alpha, X[k], X[l]) for k in range(3) for l in range(3)]
             + beta + [sp.diff(beta[i], X[j]) for j in range(3) for i in range(3)])
    vals = an.evaluate(exprs, X, pt)
    o = [0]

    def take(n, shape):
        a = vals[o[0]:o[0] + n].reshape(shape)
        o[0] += n
        return a
    gv, dg, ddg = take(9, (3, 3)), take(27, (3, 3, 3)), take(81, (3, 3, 3, 3))
    Kv, dK = take(9, (3, 3)), take(27, (3, 3, 3))
    al, dal, ddal = float(take(1, (1,))[0]), take(3, (3,)), take(9, (3, 3))
    bv, dbv = take(3, (3,)), take(9, (3, 3))
    gi3, Gam3, Rdn, Ric, Rs = an.geometry4(gv, dg, ddg)
    phys = dict(g=gv, K=Kv, dK=dK, Ric=Ric, DDa=ddal - np.einsum("kij,k->ij", Gam3, dal), Gam=Gam3, dg=dg,
                alpha=al, beta=bv, dbeta=dbv)
    return v, d1, d2, phys


@pytest.mark.parametrize("couplings", [(0.0, 0.0), (0.4, 0.3)])
def test_ccz4_reduces_to_adm(orc, conformal_generic, couplings):
    """With Theta = 0, Z = 0 and b = 0 the CCZ4 equations for chi, h_ij, K, A_ij imply exactly the
    ADM equations:
        d_t gamma_ij = -2 lapse K_ij + D_i beta_j + D_j beta_i,
        d_t K_ij = -D_i D_j lapse + lapse (R_ij + K K_ij - 2 K_ik K^k_j) + L_beta K_ij
                   - lapse (8 pi S_ij - 1/2 gamma_ij (8 pi S - 8 pi rho)),
    with the solved (coupled) S_ij. The ADM side is computed here from the physical metric
    with an independent (sympy) Ricci tensor. Catches errors in any term of the four
    conformal equations or in the matter coupling of K and A_ij."""
    v, d1, d2, ph = conformal_generic
    lam, g2 = couplings
    p = P(lam=lam, g2=g2, b0=0.0, a0=0.3)
    rhs, diag, st = orc.point_rhs(p, v, d1, d2)
    assert st == 0
    chi, K = v[0], v[7]
    h = np.zeros((3, 3)); A = np.zeros((3, 3)); hd = np.zeros((3, 3)); Ad = np.zeros((3, 3))
    for m, (i, j) in enumerate(an.SYM_PAIRS):
        h[i, j] = h[j, i] = v[1 + m]
        A[i, j] = A[j, i] = v[8 + m]
        hd[i, j] = hd[j, i] = rhs[1 + m]
        Ad[i, j] = Ad[j, i] = rhs[8 + m]
    chid, Kd = rhs[0], rhs[7]
    g, Kij, al = ph["g"], ph["K"], ph["alpha"]
    gi3 = np.linalg.inv(g)
    # d_t gamma_ij from the conformal right-hand sides
    gd = hd / chi - h * chid / chi ** 2
    beta_l = g @ ph["beta"]
    dbeta_l = np.einsum("kij,j->ki", ph["dg"], ph["beta"]) + np.einsum("ij,kj->ki", g, ph["dbeta"])
    Dbeta = dbeta_l - np.einsum("lki,l->ki", ph["Gam"], beta_l)   # D_k beta_i
    np.testing.assert_allclose(gd, -2 * al * Kij + Dbeta + Dbeta.T, atol=1e-12)
    # d_t K_ij from the conformal right-hand sides
    ud = (Ad + hd * K / 3 + h * Kd / 3) / chi - Kij * chid / chi
    Sij8 = np.zeros((3, 3))
    for m, (i, j) in enumerate(an.SYM_PAIRS):
        Sij8[i, j] = Sij8[j, i] = diag[4 + m]
    rho8 = diag[0]
    S8 = np.einsum("ij,ij->", gi3, Sij8)
    Ktr = np.einsum("ij,ij->", gi3, Kij)
    KK = Kij @ gi3 @ Kij
    LbK = (np.einsum("k,kij->ij", ph["beta"], ph["dK"]) + np.einsum("kj,ik->ij", Kij, ph["dbeta"])
           + np.einsum("ik,jk->ij", Kij, ph["dbeta"]))
    adm = -ph["DDa"] + al * (ph["Ric"] + Ktr * Kij - 2 * KK) + LbK - al * (Sij8 - 0.5 * g * (S8 - rho8))
    np.testing.assert_allclose(ud, adm, atol=1e-11)
    # the solved d_t K_ij is the one that enters the coupled system
    np.testing.assert_allclose([ud[i, j] for i, j in an.SYM_PAIRS], diag[11:17], atol=1e-11)


def test_zero_coupling_scalar_is_klein_gordon(orc, conformal_generic):
    """With lambda = g2 = 0 the solved d_t Pi equals the 3+1 Klein-Gordon equation
    d_t Pi = beta^k d_k Pi + lapse (D^i D_i phi + K Pi) + gamma^ij d_i lapse d_j phi,
    and 8 pi rho = (Pi^2 + |D phi|^2)/4, 8 pi S_i = -Pi d_i phi / 2 (action R + X over 16 pi).
    Catches sign errors in the nabla_i nabla_j phi = D_i D_j phi + K_ij Pi projection and in
    the n-n block of the scalar equation."""
    v, d1, d2, ph = conformal_generic
    p = P(lam=0.0, g2=0.0)
    rhs, diag, st = orc.point_rhs(p, v, d1, d2)
    g, Kij, al = ph["g"], ph["K"], ph["alpha"]
    gi3 = np.linalg.inv(g)
    Pi, dPi, dphi = v[26], d1[26], d1[25]
    ddphi = np.zeros((3, 3))
    for m, (i, j) in enumerate(an.SYM_PAIRS):
        ddphi[i, j] = ddphi[j, i] = d2[25, m]
    DDphi = ddphi - np.einsum("kij,k->ij", ph["Gam"], dphi)
    Ktr = np.einsum("ij,ij->", gi3, Kij)
    kg = ph["beta"] @ dPi + al * (np.einsum("ij,ij->", gi3, DDphi) + Ktr * Pi) + d1[18] @ gi3 @ dphi
    assert abs(rhs[26] - kg) < 1e-12
    assert abs(diag[0] - 0.25 * (Pi ** 2 + dphi @ gi3 @ dphi)) < 1e-13
    np.testing.assert_allclose(diag[1:4], -0.5 * Pi * dphi, atol=1e-13)


def test_solve_matrix_is_identity_at_zero_coupling(orc, conformal_generic):
    """The coupled system's Jacobian reduces to the trivial one (-1 on the d_t K_ij rows, +1 on
    the d_t Pi row) when the couplings vanish, and departs from it when they do not."""
    v, d1, d2, ph = conformal_generic
    _, diag0, _ = orc.point_rhs(P(lam=0.0, g2=0.0), v, d1, d2)
    np.testing.assert_allclose(diag0[38:45], [-1, -1, -1, -1, -1, -1, 1], atol=1e-13)
    _, diag1, _ = orc.point_rhs(P(lam=0.5, g2=0.4), v, d1, d2)
    assert np.max(np.abs(diag1[38:45] - np.array([-1, -1, -1, -1, -1, -1, 1]))) > 1e-3
    assert diag1[18] < 1e-12  # residual of the coupled equations after the solve


@pytest.mark.parametrize("kind,g3", [(0, 0.0), (1, 0.0), (1, 0.6)])
def test_decoupled_metric_is_vacuum_and_blind_to_the_scalar(orc, conformal_generic, kind, g3):
    """4dST without backreaction onto the metric ("Key features"): with decoupled = 1 the metric
    and gauge right-hand sides (fields 0..24) do not see the scalar at all. For any scalar data
    they equal the full theory's with the scalar switched off (phi = Pi = 0 with zero derivatives,
    where T_ab vanishes for both couplings: vacuum CCZ4 in the same gauge). With backreaction the
    same scalar data does move the metric, and the decoupled scalar still evolves. Catches a
    stress-energy term left in a metric equation, or a mode switch that does nothing.
    The vacuum reference also switches the couplings off: with beta = lambda phi a zero scalar is
    still sourced by L_GB (d_t Pi != 0), and its Gauss-Bonnet stress does not vanish. With the
    cubic term (g3 != 0) its stress tensor is left out too, while the scalar equation keeps it:
    the decoupled d_t Pi differs from the one without it."""
    v, d1, d2, ph = conformal_generic
    gauge = dict(a0=0.3, b0=0.5)
    kw = dict(lam=0.4, g2=0.3, beta_kind=kind, g3=g3, **gauge)
    r_dec, diag_dec, st = orc.point_rhs(P(decoupled=1, **kw), v, d1, d2)
    assert st == 0
    v0, d10, d20 = v.copy(), d1.copy(), d2.copy()
    v0[25:27] = 0.0
    d10[25:27] = 0.0
    d20[25:27] = 0.0
    r_vac, diag_vac, _ = orc.point_rhs(P(lam=0.0, g2=0.0, **gauge), v0, d10, d20)
    assert np.all(diag_vac[0:10] == 0.0)          # no stress-energy without a scalar
    np.testing.assert_allclose(r_dec[:25], r_vac[:25], rtol=1e-12, atol=1e-13)
    assert np.all(diag_dec[0:10] == 0.0)          # decoupled: rho, S_i, S_ij left out
    r_full, _, _ = orc.point_rhs(P(**kw), v, d1, d2)
    assert np.max(np.abs(r_full[:25] - r_vac[:25])) > 1e-4
    assert abs(r_dec[26]) > 1e-4 and abs(r_dec[26] - r_full[26]) > 1e-8
    assert diag_dec[18] < 1e-12                   # residual of the scalar equation after the solve
    if g3:
        r_nocub, _, _ = orc.point_rhs(P(decoupled=1, **dict(kw, g3=0.0)), v, d1, d2)
        np.testing.assert_array_equal(r_dec[:25], r_nocub[:25])
        assert abs(r_dec[26] - r_nocub[26]) > 1e-4


def test_decoupled_scalar_at_zero_coupling_is_klein_gordon(orc, conformal_generic):
    """Without couplings the scalar equation does not involve d_t K_ij, so the decoupled d_t Pi
    equals the full theory's, which the Klein-Gordon pin fixes."""
    v, d1, d2, ph = conformal_generic
    r_full, _, _ = orc.point_rhs(P(lam=0.0, g2=0.0), v, d1, d2)
    r_dec, _, _ = orc.point_rhs(P(lam=0.0, g2=0.0, decoupled=1), v, d1, d2)
    assert abs(r_dec[26] - r_full[26]) < 1e-13


def _full_and_octant(n=10, dx=0.25):
    full = gi.Box(2 * n, 2 * n, 2 * n, dx, -(n - 0.5) * dx, -(n - 0.5) * dx, -(n - 0.5) * dx, bc=gi.BC_FROZEN)
    octant = gi.Box(n, n, n, dx, 0.5 * dx, 0.5 * dx, 0.5 * dx, bc=gi.BC_REFLECT_LOW)
    return full, octant


def test_mirror_planes_reproduce_the_symmetric_full_box(orc):
    """A state symmetric under the x, y and z reflections is evolved twice for 2 RK4 steps.
    - on a full box with frozen ghosts (the analytic data);
    - on its positive octant, whose three low faces are mirror planes (ghosts rebuilt from the
      interior with each component's parity after every stage) and whose high faces keep the
      same analytic ghosts.
    The two agree on the octant to rounding. The same octant with its low ghosts frozen instead
    does not (the mirror ghosts must follow the evolution). Catches a wrong parity for any
    component, a mirror offset by one point, and ghosts not refreshed between stages."""
    n = 10
    full_box, oct_box = _full_and_octant(n)
    p = P(lam=0.2, g2=0.1, beta_kind=1)
    dt = 0.25 * full_box.dx
    full = gi.mirror_symmetric_state(full_box)
    octant = gi.mirror_symmetric_state(oct_box)
    frozen = octant.copy()
    orc.rk4(full_box, p, full, dt, 2)
    orc.rk4(oct_box, p, octant, dt, 2)
    frozen_box = gi.Box(n, n, n, oct_box.dx, oct_box.x0, oct_box.y0, oct_box.z0, bc=gi.BC_FROZEN)
    orc.rk4(frozen_box, p, frozen, dt, 2)
    ref = full[:, n + 3:2 * n + 3, n + 3:2 * n + 3, n + 3:2 * n + 3]
    got = oct_box.interior(octant)
    scale = np.maximum(np.max(np.abs(ref), axis=(1, 2, 3)), 1e-12)
    err = np.max(np.abs(got - ref), axis=(1, 2, 3)) / scale
    assert np.max(err) < 1e-12, err
    err_frozen = np.max(np.abs(oct_box.interior(frozen) - ref), axis=(1, 2, 3)) / scale
    assert np.max(err_frozen) > 1e-6


@pytest.mark.parametrize("couplings", [(0.0, 0.0), (0.4, 0.3)])
@pytest.mark.parametrize("kind", [0, 1])
def test_energy_densities_of_the_three_scalar_terms(orc, conformal_generic, couplings, kind):
    """The energy density is split by the terms of the action R + X + g2 X^2 + beta(phi) L_GB
    ("Diagnostics"), in the 8 pi rho units of the right-hand sides:
        X term:    (Pi^2 + |D phi|^2) / 4 for any couplings (the minimally coupled scalar);
        X^2 term:  g2 (X Pi^2 - X^2 / 2) with X = (Pi^2 - |D phi|^2) / 2;
        GB term:   zero when lambda = 0;
    and the three add up to the 8 pi rho that enters the equations. Catches a term assigned to
    the wrong part, a sign of X, or a missing g2."""
    v, d1, d2, ph = conformal_generic
    lam, g2 = couplings
    p = P(lam=lam, g2=g2, beta_kind=kind)
    parts = orc.point_energy(p, v, d1, d2)
    _, diag, _ = orc.point_rhs(p, v, d1, d2)
    gi3 = np.linalg.inv(ph["g"])
    Pi, dphi = v[26], d1[25]
    grad2 = dphi @ gi3 @ dphi
    X = 0.5 * (Pi ** 2 - grad2)
    assert abs(parts[0] - 0.25 * (Pi ** 2 + grad2)) < 1e-14
    assert abs(parts[1] - g2 * (X * Pi ** 2 - 0.5 * X ** 2)) < 1e-14
    if lam == 0.0:
        assert parts[2] == 0.0
    else:
        assert abs(parts[2]) > 1e-6
    assert abs(parts.sum() - diag[0]) < 1e-13


def test_exponential_coupling_tends_to_the_quadratic_one(orc, conformal_generic):
    """beta = lam/(2 kappa) (1 - e^{-kappa phi^2}) -> lam phi^2 / 2 as kappa -> 0: the right-hand side
    with kappa = 1e-7 equals the quadratic coupling's to O(kappa phi^2), while kappa = 0.8 differs;
    the brute-force pins above check the exponential kind's beta', beta'' at finite kappa."""
    v, d1, d2, ph = conformal_generic
    quad, _, _ = orc.point_rhs(P(lam=0.4, g2=0.2, beta_kind=1), v, d1, d2)
    small, _, _ = orc.point_rhs(P(lam=0.4, g2=0.2, beta_kind=2, beta_kappa=1e-7), v, d1, d2)
    big, _, _ = orc.point_rhs(P(lam=0.4, g2=0.2, beta_kind=2, beta_kappa=0.8), v, d1, d2)
    scale = np.maximum(np.abs(quad), 1e-6)
    assert np.max(np.abs(small - quad) / scale) < 1e-6
    assert np.max(np.abs(big - quad) / scale) > 1e-5


# ----------------------------------------------------------------------------- constraints
def test_constraints_converge_to_zero_on_kerr_schild(orc):
    """H and M_i of the exact Kerr-Schild data, computed with 4th-order differences on boxes
    away from the singularity, converge to zero at 4th order (ratio ~16 per halving).
    Catches wrong factors in H = R + K^2 - K_ij K^ij or M_i = D_j K^j_i - D_i K."""
    fields, X = an.kerr_schild_fields(M=1.0)
    fn = sp.lambdify(X, fields, modules="numpy")
    errs = []
    for dx in (0.1, 0.05):
        n = int(round(0.4 / dx))
        b = gi.Box(n, n, n, dx, 1.5, 1.2, 1.3, bc=gi.BC_FROZEN)
        Xg, Yg, Zg = b.coords()
        s = np.zeros(b.shape)
        vals = fn(Xg, Yg, Zg)
        for f in range(27):
            s[f] = np.broadcast_to(np.asarray(vals[f], dtype=np.float64), Xg.shape)
        c = orc.constraints(b, P(lam=0.0, g2=0.0), s)
        # compare at the common physical points (every second point of the finer grid)
        if dx == 0.1:
            errs.append(np.max(np.abs(c)))
        else:
            errs.append(np.max(np.abs(c)))
    assert errs[0] < 1e-4
    assert 12 < errs[0] / errs[1] < 20, errs


# ----------------------------------------------------------------------------- P4 plane wave
def test_scalar_plane_wave_converges_4th_order(orc):
    """A small scalar plane wave on flat space (amplitude 1e-6, so back-reaction is O(1e-12))
    evolved with the full RK4 + 4th-order FD + KO converges to the exact solution
    phi = A sin(k(x - t)) at 4th order. Catches errors in the RK4 weights/stage times, in the
    scalar advection/lapse terms and in the stencils."""
    amp, L, T = 1e-6, 2.0, 0.5
    k = 2 * math.pi / L
    errs = []
    for n in (16, 32):
        b = gi.Box(n, 4, 4, L / n, 0.5 * L / n, 0.0, 0.0)
        s = gi.scalar_plane_wave(b, amp, (k, 0.0, 0.0))
        dt = 0.25 * b.dx
        nsteps = int(round(T / dt))
        orc.rk4(b, gi.Params(), s, dt, nsteps)
        ex = gi.scalar_plane_wave(b, amp, (k, 0.0, 0.0), t=nsteps * dt)
        errs.append(np.max(np.abs(b.interior(s)[25] - b.interior(ex)[25])) / amp)
    assert errs[1] < 1e-3
    assert 13 < errs[0] / errs[1] < 19, errs


def test_psi4_of_an_outgoing_plane_wave(orc):
    """For a weak outgoing wave the Weyl scalar is Psi_4 = -(h+'' - i hx''), with h+ = h_theta theta
    and hx = h_theta phi in the triad about the origin (the standard relation between Psi_4 and
    the wave's strain). At (X0, 0, 0) the triad is (x, -z, y), so h+ = -a, hx = -b and
    Psi_4 = a'' - i b''. An ingoing wave gives Psi_4 = 0 to first order (it is carried by Psi_0):
    this fixes the choice of the ingoing null vector n, the normalisation of the tetrad and the sign
    of the imaginary part against physics rather than against a second code's definition."""
    amp, k, X0 = 1e-6, 0.9, 2.3
    p = P(lam=0.0, g2=0.0)
    (v, d1, d2), add, bdd = an.tt_plane_wave_point(+1, amp, 0.7 * amp, k, X0)
    got = orc.point_psi4(p, v, d1, d2, np.array([X0, 0.0, 0.0]))
    want = add - 1j * bdd
    assert abs(want) > 0.3 * amp * k * k
    assert abs(got - want) < 1e-5 * abs(want), (got, want)
    (v, d1, d2), add, bdd = an.tt_plane_wave_point(-1, amp, 0.7 * amp, k, X0)
    got = orc.point_psi4(p, v, d1, d2, np.array([X0, 0.0, 0.0]))
    assert abs(got) < 1e-5 * abs(add - 1j * bdd), got


def test_gravitational_plane_wave_converges_4th_order(orc):
    """The metric sector's counterpart of the scalar plane wave: a weak transverse-traceless
    gravitational wave (amplitude 1e-6, both polarisations) on a periodic box, evolved by the full
    CCZ4 RK4 with 1+log slicing and the Gamma-driver, travels at the speed of light with its shape:
    h_22, h_23, h_33 and A_22, A_23, A_33 converge to the exact wave at 4th order. Catches errors in
    the Ricci tensor of the conformal metric, the A_ij and h_ij equations and their coupling."""
    amp, L, T = 1e-6, 2.0, 0.5
    k = 2 * math.pi / L
    errs = []
    for n in (16, 32):
        b = gi.Box(n, 4, 4, L / n, 0.5 * L / n, 0.0, 0.0)
        s = waves.tt_wave_state(b, amp, k, 0.0)
        dt = 0.25 * b.dx
        nsteps = int(round(T / dt))
        orc.rk4(b, gi.Params(lam=0.0, g2=0.0), s, dt, nsteps)
        ex = waves.tt_wave_state(b, amp, k, nsteps * dt)
        fields = [4, 5, 6, 11, 12, 13]
        scale = [amp, amp, amp, amp * k, amp * k, amp * k]
        errs.append(max(np.max(np.abs(b.interior(s)[f] - b.interior(ex)[f])) / sc for f, sc in zip(fields, scale)))
    assert errs[1] < 1e-3, errs
    assert 13 < errs[0] / errs[1] < 19, errs


@pytest.mark.parametrize("a0", [0.0, 0.2])
def test_gauge_wave_of_the_modified_puncture_gauge(orc, a0):
    """A pure gauge perturbation of the lapse on flat space (amplitude 1e-6, Gamma-driver off by
    F = 0) oscillates as the standing wave of the slicing, at speed sqrt(2) in the standard gauge
    (a = 0) and sqrt(2 / (1 + a)) in the modified one, where the lapse gradient also drives the
    shift: the lapse, K, the conformal metric, Gamma-hat and the shift converge at 4th order to the
    exact linear solution. Fixes the coefficient 2 and the sign of the slicing, the a-terms of the
    lapse and shift conditions as read, the D_i D_j alpha terms of the A_ij and K equations and the
    shift terms of the metric's evolution; the b terms multiply constraints, which vanish here."""
    eps, L, T = 1e-6, 2.0, 0.6
    k = 2 * math.pi / L
    p = gi.Params(lam=0.0, g2=0.0, shift_F=0.0, a0=a0, b0=0.4)
    errs = []
    for n in (16, 32):
        b = gi.Box(n, 4, 4, L / n, 0.5 * L / n, 0.0, 0.0)
        s = waves.gauge_wave_state(b, eps, k, 0.0, a0)
        dt = 0.25 * b.dx
        nsteps = int(round(T / dt))
        orc.rk4(b, p, s, dt, nsteps)
        ex = waves.gauge_wave_state(b, eps, k, nsteps * dt, a0)
        fields = [18, 7, 1, 15, 19]
        scale = [eps, eps * k, eps, eps * k, eps]
        errs.append(max(np.max(np.abs(b.interior(s)[f] - b.interior(ex)[f])) / sc for f, sc in zip(fields, scale)))
    assert errs[1] < 1e-3, errs
    assert 13 < errs[0] / errs[1] < 19, errs


def test_gamma_driver_gauge_wave(orc):
    """The same flat-space gauge perturbation with the Gamma-driver on (F = 0.75, eta = 1) and the
    modified gauge's a = 0.2: the lapse, K, the metric, Gamma-hat, the shift and B converge at 4th
    order to the exact linear mode, the matrix exponential of the linearised gauge system. Fixes
    the Gamma-driver as read: F / (1 + a) on B, d_t B = d_t Gamma-hat - eta B, and the shift's second
    derivatives in the Gamma-hat equation."""
    eps, L, T = 1e-6, 2.0, 0.6
    k = 2 * math.pi / L
    a, F, eta = 0.2, 0.75, 1.0
    p = gi.Params(lam=0.0, g2=0.0, shift_F=F, eta=eta, a0=a, b0=0.4)
    errs = []
    for n in (16, 32):
        b = gi.Box(n, 4, 4, L / n, 0.5 * L / n, 0.0, 0.0)
        s = waves.gamma_driver_wave_state(b, eps, k, 0.0, a, F, eta)
        dt = 0.25 * b.dx
        nsteps = int(round(T / dt))
        orc.rk4(b, p, s, dt, nsteps)
        ex = waves.gamma_driver_wave_state(b, eps, k, nsteps * dt, a, F, eta)
        moved = np.max(np.abs(b.interior(ex)[19])) / eps
        fields = [18, 7, 1, 15, 19, 22]
        scale = [eps, eps * k, eps, eps * k, eps, eps * k]
        errs.append(max(np.max(np.abs(b.interior(s)[f] - b.interior(ex)[f])) / sc for f, sc in zip(fields, scale)))
    assert moved > 0.05  # the shift is driven to a sizeable fraction of the lapse perturbation
    assert errs[1] < 1e-3, errs
    assert 13 < errs[0] / errs[1] < 19, errs


def test_gravitational_plane_wave_converges_6th_order_on_4_ghost_boxes(orc):
    """The same gravitational wave on 4-ghost boxes (6th-order differences, Delta^8 dissipation)
    with a time step small enough (dx / 16) that RK4's error stays below the spatial one: from 8 to
    16 points per wavelength the error falls by ~64 (measured 61), against ~16 on 3-ghost boxes.
    Catches a 6th-order stencil that is only 4th-order accurate in the metric sector."""
    amp, L, T = 1e-8, 2.0, 0.5
    k = 2 * math.pi / L
    errs = []
    for n in (8, 16):
        b = gi.Box(n, 4, 4, L / n, 0.5 * L / n, 0.0, 0.0, ng=4)
        s = waves.tt_wave_state(b, amp, k, 0.0)
        dt = b.dx / 16
        nsteps = int(round(T / dt))
        orc.rk4(b, gi.Params(lam=0.0, g2=0.0), s, dt, nsteps)
        ex = waves.tt_wave_state(b, amp, k, nsteps * dt)
        fields = [4, 5, 6, 11, 12, 13]
        scale = [amp, amp, amp, amp * k, amp * k, amp * k]
        errs.append(max(np.max(np.abs(b.interior(s)[f] - b.interior(ex)[f])) / sc for f, sc in zip(fields, scale)))
    assert errs[1] < 1e-5, errs
    assert 45 < errs[0] / errs[1] < 80, errs


# ----------------------------------------------------------------------------- hyperbolicity
@pytest.fixture(scope="module")
def schwarzschild_points():
    fields, X = an.isotropic_schwarzschild_fields(M=1.0, lapse="precollapsed")
    rs = np.linspace(0.3, 3.0, 28)
    d = np.array([0.6, -0.3, 0.74])
    d = d / np.linalg.norm(d)
    pts = [tuple(r * d) for r in rs]
    return rs, an.conformal_point(fields, pts, X)


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_coupled_system_determinant_on_schwarzschild(orc, schwarzschild_points, lam):
    """Schwarzschild (K = 0, vacuum) with phi = 0 and beta = lambda phi: Phi = nabla nabla beta = 0,
    so the 6x6 block of the coupled system is the identity and only the Gauss-Bonnet coupling
    lambda L(G_S) of the scalar equation to d_t K_ij remains:
        det M = 1 - 32 lambda^2 G_S^ij L(G_S)_ij = 1 - 32 lambda^2 R_ij R^ij = 1 - 192 lambda^2 M^2 / R^6,
    R the areal radius (R_ij = diag(-2, 1, 1) M / R^3 in an orthonormal frame). The oracle's
    determinant comes from its covariant residual; the closed form is independent of it. The
    quadratic coupling has beta'(0) = 0 and det M = 1.
    The same structure fixes the smallest pivot ratio: with the 6x6 block the identity and the
    scalar row's couplings below 1 in magnitude, partial pivoting exchanges no rows, the pivots are
    1, ..., 1 and the Schur complement det M, and the ratio is min(1, |det M|) / max |M_ij|."""
    rs, data = schwarzschild_points
    p = P(lam=lam, g2=0.3, beta_kind=gi.BETA_LINEAR)
    closed = 0
    for r, (v, d1, d2) in zip(rs, data):
        R = an.areal_radius_isotropic(r, 1.0)
        h = orc.point_hyperbolicity(p, v, d1, d2)
        det = h[0]
        assert det == pytest.approx(1.0 - 192.0 * lam ** 2 / R ** 6, rel=1e-12, abs=1e-13)
        detq = orc.point_hyperbolicity(P(lam=lam, g2=0.3, beta_kind=gi.BETA_QUADRATIC), v, d1, d2)[0]
        assert detq == pytest.approx(1.0, abs=1e-14)
        M = orc.point_system(p, v, d1, d2)
        np.testing.assert_allclose(M[:6, :6], np.eye(6), rtol=0, atol=1e-14)
        assert M[6, 6] == 1.0
        if np.max(np.abs(M[6, :6])) < 1.0:
            assert h[3] == pytest.approx(min(1.0, abs(det)) / np.max(np.abs(M)), rel=1e-12)
            closed += 1
    assert closed >= 10


def test_loss_of_solvability_radius_on_schwarzschild(orc, schwarzschild_points):
    """With lambda = M^2 the determinant crosses zero outside the horizon, at R^6 = 192 lambda^2 M^2:
    bisection on the oracle's determinant along a radial line finds that areal radius."""
    fields, X = an.isotropic_schwarzschild_fields(M=1.0, lapse="precollapsed")
    d = np.array([0.6, -0.3, 0.74])
    d = d / np.linalg.norm(d)
    p = P(lam=1.0, g2=0.0, beta_kind=gi.BETA_LINEAR)

    def det(r):
        v, d1, d2 = an.conformal_point(fields, tuple(r * d), X)
        return orc.point_hyperbolicity(p, v, d1, d2)[0]

    lo, hi = 0.6, 1.6  # isotropic radii with areal radius 2.12 .. 2.74
    assert det(lo) < 0.0 < det(hi)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if det(mid) < 0.0 else (lo, mid)
    assert an.areal_radius_isotropic(0.5 * (lo + hi), 1.0) == pytest.approx(192.0 ** (1.0 / 6.0), rel=1e-9)


def test_hyperbolicity_diagnostics_without_coupling(orc, conformal_generic):
    """lambda = g2 = 0: the coupled system is the identity (all pivots 1) and g_eff = g."""
    v, d1, d2, ph = conformal_generic
    h = orc.point_hyperbolicity(P(lam=0.0, g2=0.0), v, d1, d2)
    np.testing.assert_allclose(h, [1.0, 1.0, 1.0, 1.0], rtol=0, atol=1e-14)


@pytest.mark.parametrize("g2", [0.3, -0.8])
def test_effective_metric_of_the_scalar_equation(orc, conformal_generic, g2):
    """On a generic non-vacuum point (Pi and grad phi non-zero), without backreaction so that the
    scalar equation alone fixes d_t Pi:
      * its linearisation in the second derivatives of phi, by differences of the oracle's d_t Pi
        (exact: d_t Pi is affine in them), is alpha g_eff^ij / D with the principal symbol
        g_eff^ab = (1 + 2 g2 X) g^ab - 2 g2 nabla^a phi nabla^b phi (the X^2 term of the action)
        and D = -g_eff^nn, the oracle's third diagnostic;
      * D is the coefficient of d_t Pi in the oracle's residual (the solve's w-w entry);
      * det(g_eff)/det(g) is (1 + 2 g2 X)^3 (1 + 6 g2 X), the matrix determinant lemma."""
    v, d1, d2, ph = conformal_generic
    p = P(lam=0.4, g2=g2, decoupled=1)
    h = orc.point_hyperbolicity(p, v, d1, d2)
    gi3 = np.linalg.inv(ph["g"])
    al = ph["alpha"]
    Pi = v[26]
    dphi = d1[25]
    X = 0.5 * (Pi * Pi - dphi @ gi3 @ dphi)
    geff = (1 + 2 * g2 * X) * gi3 - 2 * g2 * np.outer(gi3 @ dphi, gi3 @ dphi)
    D = 1 + 2 * g2 * X + 2 * g2 * Pi * Pi
    assert h[2] == pytest.approx(D, rel=1e-13)
    assert h[1] == pytest.approx((1 + 2 * g2 * X) ** 3 * (1 + 6 * g2 * X), rel=1e-12)
    _, diag, _ = orc.point_rhs(p, v, d1, d2)
    assert diag[44] == pytest.approx(D, rel=1e-12)
    base = orc.point_rhs(p, v, d1, d2)[0][26]
    for m, (i, j) in enumerate(an.SYM_PAIRS):
        dd = d2.copy()
        dd[25, m] += 1e-3
        got = (orc.point_rhs(p, v, d1, dd)[0][26] - base) / 1e-3
        want = al * geff[i, j] / D * (1.0 if i == j else 2.0)
        assert got == pytest.approx(want, rel=1e-8, abs=1e-11), (i, j)


@pytest.mark.parametrize("g3,lam,g2", [(0.6, 0.0, 0.0), (-0.9, 0.5, 0.2)])
def test_cubic_effective_metric_against_brute_force(orc, z4_point, g3, lam, g2):
    """With the cubic term the scalar equation's principal symbol g_eff^ab = dE/d(nabla_a nabla_b phi)
    depends on the second derivatives of phi themselves: 2 g3 (box(phi) g^ab - nabla^a nabla^b phi)
    joins the X and X^2 terms. The covariant Z4 solution at the generic point gives the 4D second
    derivatives of the metric and of phi; central differences of the brute-force E (quadratic in
    nabla nabla phi, so exact) give g_eff there, and its invariants det(g_eff)/det(g) and
    -g_eff(n, n) must equal the oracle's second and third diagnostics (which evaluate the symbol at
    the oracle's own solution of the 7x7 system)."""
    D = z4_point
    kw = dict(b=0.4, k1=0.25, k2=0.5, lam=lam, g2=g2, kind=1, g3=g3)
    unk = an.z4_unknowns(D, **kw)
    ddg = D["ddg"].copy()
    for m, (i, j) in enumerate(an.SYM_PAIRS):
        ddg[0, 0, i + 1, j + 1] += unk[m]
        if i != j:
            ddg[0, 0, j + 1, i + 1] += unk[m]
    ddphi = D["ddphi"].copy()
    ddphi[0, 0] += unk[10]
    g = D["g4"]
    gi4, Gam, Rdn, Ric, Rs = an.geometry4(g, D["dg"], ddg)

    def E_of(dd):
        return an.stress_and_scalar(g, gi4, Gam, Rdn, Ric, Rs, D["dphi"], dd, D["phi"], lam, g2, 1, g3=g3)[1]
    geff = np.zeros((4, 4))
    eps = 1e-3
    for a in range(4):
        for b in range(a, 4):
            e = np.zeros((4, 4))
            e[a, b] += 0.5 * eps
            e[b, a] += 0.5 * eps
            geff[a, b] = geff[b, a] = (E_of(ddphi + e) - E_of(ddphi - e)) / (2 * eps)
    al = 1.0 / math.sqrt(-gi4[0, 0])
    ratio = np.linalg.det(geff) / np.linalg.det(gi4)
    dnn = -al * al * geff[0, 0]
    h = orc.point_hyperbolicity(P(kappa1=0.25, kappa2=0.5, kappa3=1.0, a0=0.2, b0=0.4, lam=lam, g2=g2,
                                  beta_kind=1, g3=g3), D["v"], D["d1"], D["d2"])
    assert abs(ratio - 1.0) > 1e-3 and abs(dnn - 1.0) > 1e-3  # the cubic term changes both
    assert h[1] == pytest.approx(ratio, rel=1e-9)
    assert h[2] == pytest.approx(dnn, rel=1e-9)
