"""CPU check of the CUDA kernels' pointwise formulas (the kernel source instantiated for the
host in FP64) against the oracle's pointwise RHS on generic points. This is a fast
development check; the GPU parity tests compare the real kernels through the C ABI."""
import numpy as np
import pytest

import grf_inputs as gi

D1_FIELDS = list(range(22)) + [25, 26]
D2_FIELDS = [0, 1, 2, 3, 4, 5, 6, 18, 19, 20, 21, 25]


def slots(d1, d2):
    return d1[D1_FIELDS].reshape(-1), d2[D2_FIELDS].reshape(-1)


@pytest.fixture(scope="module")
def flops():
    from paper_2309_06225_gb300 import flops as fl
    return fl


@pytest.mark.parametrize("g3", [0.0, 0.45])
@pytest.mark.parametrize("decoupled", [0, 1])
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_kernel_pointwise_rhs_matches_oracle(orc, flops, seed, kind, decoupled, g3):
    import paper_2309_06225_gb300 as grf
    rng = np.random.default_rng(100 + seed)
    v = rng.uniform(-0.2, 0.2, 27)
    v[0] = rng.uniform(0.3, 1.0)                 # chi
    for m, d in zip(range(1, 7), [1, 0, 0, 1, 0, 1]):
        v[m] = d + rng.uniform(-0.15, 0.15)      # h_ij near delta
    v[18] = rng.uniform(0.4, 1.0)                # lapse
    d1 = rng.normal(size=(27, 3)) * 0.3
    d2 = rng.normal(size=(27, 6)) * 0.3
    p = gi.Params(lam=rng.uniform(0.0, 0.6), g2=rng.uniform(0.0, 0.4), beta_kind=kind, a0=0.3, b0=0.7,
                  kappa2=0.2, kappa3=0.6, decoupled=decoupled, beta_kappa=rng.uniform(0.5, 3.0), g3=g3)
    ref, diag, st = orc.point_rhs(p, v, d1, d2)
    assert st == 0
    s1, s2 = slots(d1, d2)
    got, extra, st2 = flops.host_point_rhs(grf.params_like(p), v, s1, s2)
    assert st2 == 0
    scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
    err = np.abs(got - ref) / scale
    assert np.max(err) < 1e-11, (np.argmax(err), gi.FIELD_NAMES[int(np.argmax(err))], np.max(err))
    # constraint by-products against the oracle's physical-form constraints
    con = orc.point_constraints(p, v, d1, d2)
    # the oracle's physical forms assume nothing about tr(A); compare on the trace-free part
    np.testing.assert_allclose(extra, con, rtol=1e-9, atol=1e-9 * np.max(np.abs(con)))


@pytest.mark.parametrize("g3", [0.0, 0.45, -0.6])
@pytest.mark.parametrize("decoupled", [0, 1])
@pytest.mark.parametrize("seed", range(3))
def test_kernel_hyperbolicity_matches_oracle(orc, flops, seed, decoupled, g3):
    """The kernel's hyperbolicity diagnostics (det M from its closed-form assembly, det g_eff /
    det g by the determinant lemma or, with the cubic term, by the Schur complement at the solved
    d_t Pi, and -g_eff^nn) against the oracle's full-pivot determinants on generic points."""
    import paper_2309_06225_gb300 as grf
    rng = np.random.default_rng(300 + seed)
    v = rng.uniform(-0.2, 0.2, 27)
    v[0] = rng.uniform(0.3, 1.0)
    for m, d in zip(range(1, 7), [1, 0, 0, 1, 0, 1]):
        v[m] = d + rng.uniform(-0.15, 0.15)
    v[18] = rng.uniform(0.4, 1.0)
    d1 = rng.normal(size=(27, 3)) * 0.3
    d2 = rng.normal(size=(27, 6)) * 0.3
    p = gi.Params(lam=rng.uniform(0.1, 0.6), g2=rng.uniform(0.0, 0.4), beta_kind=seed % 2, decoupled=decoupled,
                  g3=g3)
    ref = orc.point_hyperbolicity(p, v, d1, d2)
    s1, s2 = slots(d1, d2)
    got, st = flops.host_point_hyp(grf.params_like(p), v, s1, s2)
    assert st == 0
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_kernel_psi4_matches_oracle(orc, flops, seed):
    """The kernel's Psi_4 (the Riemann tensor on the null tetrad from the Gauss, Codazzi and
    Ricci-equation blocks) equals the oracle's contraction of the full Weyl tensor on generic
    non-vacuum points, couplings on."""
    import paper_2309_06225_gb300 as grf
    rng = np.random.default_rng(200 + seed)
    v = rng.uniform(-0.2, 0.2, 27)
    v[0] = rng.uniform(0.3, 1.0)
    for m, d in zip(range(1, 7), [1, 0, 0, 1, 0, 1]):
        v[m] = d + rng.uniform(-0.15, 0.15)
    v[18] = rng.uniform(0.4, 1.0)
    d1 = rng.normal(size=(27, 3)) * 0.3
    d2 = rng.normal(size=(27, 6)) * 0.3
    p = gi.Params(lam=rng.uniform(0.0, 0.6), g2=rng.uniform(0.0, 0.4), beta_kind=seed % 2)
    xyz = rng.uniform(-2, 2, 3)
    ref = orc.point_psi4(p, v, d1, d2, xyz)
    s1, s2 = slots(d1, d2)
    got, st = flops.host_point_psi4(grf.params_like(p), v, s1, s2, xyz)
    assert st == 0 and abs(ref) > 1e-3
    assert abs(got - ref) < 1e-11 * max(1.0, abs(ref)), (got, ref)


def test_kernel_psi4_of_an_outgoing_plane_wave(flops):
    """The kernel's Psi_4 on a weak outgoing gravitational plane wave along x, at (X0, 0, 0):
    a'' - i b'' (the standard -(h+'' - i hx'') in the triad (x, -z, y)); zero to first order for
    the ingoing wave."""
    pytest.importorskip("sympy")
    import analytic as an
    import paper_2309_06225_gb300 as grf
    amp, k, X0 = 1e-6, 0.9, 2.3
    p = grf.params_like(gi.Params(lam=0.0, g2=0.0))
    for direction in (+1, -1):
        (v, d1, d2), add, bdd = an.tt_plane_wave_point(direction, amp, 0.7 * amp, k, X0)
        s1, s2 = slots(d1, d2)
        got, st = flops.host_point_psi4(p, v, s1, s2, np.array([X0, 0.0, 0.0]))
        assert st == 0
        want = add - 1j * bdd if direction > 0 else 0.0
        assert abs(got - want) < 1e-5 * abs(add - 1j * bdd), (direction, got, want)


def test_operation_count_is_stable(flops):
    """The per-point FP64 operation count of the kernels (the roofline numerator) is a fixed
    property of the formulation: independent of the point data."""
    import paper_2309_06225_gb300 as grf
    p = grf.params_like(gi.Params())
    a = flops.point_ops(p).sum(axis=0)
    rng = np.random.default_rng(3)
    b = flops.point_ops(p, rng.uniform(0.5, 1, 27), rng.normal(size=72), rng.normal(size=72)).sum(axis=0)
    assert np.array_equal(a[:4], b[:4])
    assert 4000 < flops.flops_per_point_stage(p) < 20000
