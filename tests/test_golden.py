"""The oracle against the stored fixtures of tests/golden/: closed forms the mathematics fixes
(closed_forms.json, pins) and a regression snapshot of oracle outputs (oracle_regression.json,
written by tests/golden/make_oracle_regression.py from the oracle alone)."""
import json
import math
import os

import numpy as np
import pytest

import grf_inputs as gi

HERE = os.path.dirname(os.path.abspath(__file__))
CLOSED = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))
REGRESSION = json.load(open(os.path.join(HERE, "golden", "oracle_regression.json")))


def _nyquist_rhs(orc, ng, advection):
    b = gi.Box(6, 6, 6, 0.2, 0.0, 0.0, 0.0, bc=gi.BC_FROZEN, ng=ng)
    s = gi.flat_state(b)
    idx = np.indices(b.shape[1:])[2]
    s[25] = 1e-3 * np.where(idx % 2 == 0, 1.0, -1.0)
    s[19] = 0.5
    r = orc.rhs(b, gi.Params(lam=0.0, g2=0.0, advection=advection), s, with_ko=False)
    return b, s, r


@pytest.mark.parametrize("ng,key", [(3, "4th"), (4, "6th")])
def test_nyquist_symbols(orc, ng, key):
    ny = CLOSED["nyquist_symbol"]
    b, s, r = _nyquist_rhs(orc, ng, 1)
    phi = b.interior(s)[25]
    np.testing.assert_allclose(b.interior(r)[25], ny["lopsided_" + key]["value"] * 0.5 / b.dx * phi, rtol=1e-12)
    np.testing.assert_allclose(b.interior(r)[26], ny["second_" + key]["value"] / b.dx ** 2 * phi, rtol=1e-12)
    ko = orc.ko(b, 0.3, s)
    np.testing.assert_allclose(b.interior(ko)[25], ny["kreiss_oliger_per_direction"]["value"] * 0.3 / b.dx * phi,
                               rtol=1e-12)


def test_gauss_legendre_three_points(orc):
    x, w = orc.gauss_legendre(3)
    o = np.argsort(x)
    np.testing.assert_allclose(x[o], CLOSED["gauss_legendre_3"]["nodes"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w[o], CLOSED["gauss_legendre_3"]["weights"], rtol=1e-14)


def test_spin_weighted_harmonic_values(orc):
    h = CLOSED["spin_weighted_harmonics"]
    for key, (re, im) in h["values"].items():
        s, l, m = (int(t[1:]) if t[0] in "lm" else int(t[1:]) for t in key.split("_"))
        got = orc.sylm(s, l, m, h["theta"], h["phi"])
        assert abs(got - complex(re, im)) < 1e-14, key


def test_schwarzschild_gauss_bonnet_value(orc):
    import analytic as an
    g = CLOSED["schwarzschild_gauss_bonnet"]
    fields, X = an.isotropic_schwarzschild_fields(M=g["M"], lapse="precollapsed")
    r = g["r_isotropic"] / math.sqrt(3.0)
    v, d1, d2 = an.conformal_point(fields, (r, r, r), X)
    _, diag, st = orc.point_rhs(gi.Params(lam=0.0, g2=0.0), v, d1, d2)
    assert st == 0
    assert abs(diag[10] - g["value"]) < 1e-12 * g["value"]


def test_oracle_regression_snapshot(orc):
    """Regression, not a pin: the oracle's outputs on the snapshot's seeded inputs are unchanged."""
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_oracle_regression as mk
    now = mk.snapshot()
    for key in ("point_rhs", "point_rho8_S8_LGB", "point_constraints", "point_energy", "point_psi4",
                "box_rhs_interior_sum_abs_per_field"):
        ref = np.asarray(REGRESSION[key])
        np.testing.assert_allclose(np.asarray(now[key]), ref, rtol=1e-12, atol=1e-14 * np.max(np.abs(ref)), err_msg=key)
    for part in ("re", "im"):
        ref = np.asarray(REGRESSION["modes_phi_l3"][part])
        np.testing.assert_allclose(now["modes_phi_l3"][part], ref, rtol=1e-12, atol=1e-15)
