"""GPU (CUDA path through the C ABI) versus the CPU oracle, element by element.

Tolerances (per field, relative to that field's maximum over the interior): one RHS
evaluation <= 1e-11; one RK4 step <= 1e-11 and ten RK4 steps <= 1e-9 (the stated parity bar
for the FP64 evolution). Integer/byte work (ghost fill) is bit-exact.
"""
import math

import numpy as np
import pytest

import grf_inputs as gi
from parity import describe, field_errors

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


def P(**kw):
    p = gi.Params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def gpu_rhs(g, box, params, s):
    b = g.box_like(box)
    st = g.to_device(s, b)
    r = g.alloc_state(b)
    g.grf_rhs(b, g.params_like(params), st, r)
    assert g.grf_check_status() == 0
    return g.to_host(r, b)


def gpu_rk4(g, box, params, s, dt, n):
    b = g.box_like(box)
    st = g.to_device(s, b)
    g.grf_rk4_step(b, g.params_like(params), st, dt, n)
    assert g.grf_check_status() == 0
    return g.to_host(st, b)


def test_ghost_fill_is_bit_exact(g, orc):
    box = gi.Box(13, 17, 11, 0.2, 0.0, 0.0, 0.0)
    s = np.random.default_rng(0).normal(size=box.shape)
    b = g.box_like(box)
    t = g.to_device(s, b)
    g.grf_fill_ghosts(b, t)
    ref = orc.fill_ghosts(box, s.copy())
    assert np.array_equal(g.to_host(t, b), ref)


def test_ko_parity(g, orc):
    box = gi.Box(13, 9, 11, 0.2, 0.0, 0.0, 0.0, bc=gi.BC_FROZEN)
    s = np.random.default_rng(1).normal(size=box.shape)
    b = g.box_like(box)
    t = g.to_device(s, b)
    r = g.alloc_state(b)
    g.grf_ko_dissipation(b, 0.3, t, r)
    ref = orc.ko(box, 0.3, s)
    errs = field_errors(g.to_host(r, b), ref, box)
    assert np.max(errs) < 1e-13, describe(errs)


RHS_CASES = {
    "puncture32": lambda: (gi.cube_box(32, -4.0, 4.0), P(), "puncture", 0),
    "ragged_perturbed_linear": lambda: (gi.Box(13, 17, 11, 0.3, -1.9, -2.3, -1.6), P(lam=0.3, g2=0.2), "perturbed", 1),
    "ragged_perturbed_quadratic": lambda: (gi.Box(11, 9, 14, 0.3, -1.7, -1.3, -2.0),
                                           P(lam=0.4, g2=0.3, beta_kind=1, a0=0.5, b0=0.9, kappa2=0.2), "perturbed", 2),
    "frozen_small": lambda: (gi.Box(7, 5, 9, 0.25, 0.9, 0.6, -1.2, bc=gi.BC_FROZEN), P(lam=0.2, g2=0.1), "perturbed", 3),
    "minimal_periodic": lambda: (gi.Box(3, 3, 3, 0.4, -0.5, -0.5, -0.5), P(lam=0.1, g2=0.1), "perturbed", 4),
    "single_point_frozen": lambda: (gi.Box(1, 1, 1, 0.3, 1.1, 0.7, 0.9, bc=gi.BC_FROZEN), P(lam=0.5, g2=0.5), "perturbed", 5),
    # the unperturbed puncture at one point (K = A = Theta = Gamma-hat = shift = 0: many RHS terms
    # vanish, the rest come from the conformal factor, the lapse and the scalar alone)
    "single_point_frozen_puncture": lambda: (gi.Box(1, 1, 1, 0.1, 1.1, 0.7, 0.9, bc=gi.BC_FROZEN), P(lam=0.5, g2=0.5),
                                             "puncture", 5),
    "zero_coupling_standard_gauge": lambda: (gi.Box(12, 10, 8, 0.3, -1.5, -1.4, -1.1), P(lam=0.0, g2=0.0, a0=0.0, b0=0.0),
                                             "perturbed", 6),
}


def make_state(box, kind, seed):
    if kind == "puncture":
        base = gi.single_puncture(box)
        return base
    base = gi.single_puncture(box, amp=0.05)
    s = gi.random_perturbed_state(box, seed, base=base, eps=3e-2)
    # give Pi, K, Theta, shift and B non-trivial values of order one percent
    return s


@pytest.mark.parametrize("case", list(RHS_CASES))
def test_rhs_parity(g, orc, case):
    box, params, kind, seed = RHS_CASES[case]()
    s = make_state(box, kind, seed)
    if box.bc == gi.BC_PERIODIC:
        orc.fill_ghosts(box, s)
    ref = orc.rhs(box, params, s)
    out = gpu_rhs(g, box, params, s)
    errs = field_errors(out, ref, box, state=s, sigma=params.sigma_ko)
    if kind == "puncture":
        # On constraint-satisfying data d_t Theta is the Hamiltonian-constraint residual
        # alpha (H - 16 pi rho)/(2 (1 + b)): a truncation residue of Ricci terms of order one, so
        # its rounding error is eps times those terms, not eps times its own (tiny) value. It is
        # compared on the scale of d_t K, which carries the same terms.
        ci, gi_ = box.interior(ref), box.interior(out)
        th = gi.IDX["Theta"]
        den = max(np.max(np.abs(ci[gi.IDX["K"]])), np.max(np.abs(ci[th])))
        errs[th] = np.max(np.abs(gi_[th] - ci[th])) / den
    assert np.max(errs) < 1e-11, describe(errs)


def test_rk4_parity_single_puncture_32(g, orc):
    """The 32^3 single-puncture workload: 1 step <= 1e-11 and 10 steps <= 1e-9 per field."""
    cfg = gi.config_single_puncture_32()
    box, params, dt = cfg["box"], cfg["params"], cfg["dt"]
    s0 = cfg["make_state"]()
    cpu = s0.copy()
    orc.fill_ghosts(box, cpu)
    orc.rk4(box, params, cpu, dt, 1)
    gpu = gpu_rk4(g, box, params, s0, dt, 1)
    e1 = field_errors(gpu, cpu, box)
    assert np.max(e1) < 1e-11, describe(e1)
    orc.rk4(box, params, cpu, dt, 9)
    gpu = gpu_rk4(g, box, params, s0, dt, 10)
    e10 = field_errors(gpu, cpu, box)
    assert np.max(e10) < 1e-9, describe(e10)


@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN])
def test_rk4_parity_ragged_perturbed(g, orc, bc):
    box = gi.Box(14, 11, 9, 0.3, -2.0, -1.6, -1.3, bc=bc)
    params = P(lam=0.3, g2=0.2, beta_kind=1)
    s0 = make_state(box, "perturbed", 11)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, 3)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 3)
    errs = field_errors(gpu, cpu, box)
    assert np.max(errs) < 1e-10, describe(errs)


@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN])
def test_rk4_parity_folded_launch(g, orc, bc):
    """48 x 40 x 36: the x-extent is not a multiple of 32 and the grid is large enough, so the
    stage runs as the folded kernel (each warp covers 2 rows of 16 points, per-thread gather).
    One RK4 step <= 1e-11 per field against the oracle; the host-to-host step on the same box
    gives the same bits."""
    import torch
    box = gi.Box(48, 40, 36, 0.25, -5.8, -4.9, -4.4, bc=bc)
    params = P(lam=0.2, g2=0.1, beta_kind=1)
    s0 = make_state(box, "perturbed", 17)
    assert np.all(np.isfinite(s0))
    cpu = s0.copy()
    if bc == gi.BC_PERIODIC:
        orc.fill_ghosts(box, cpu)
    orc.rk4(box, params, cpu, 0.25 * box.dx, 1)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 1)
    errs = field_errors(gpu, cpu, box)
    assert np.max(errs) < 1e-11, describe(errs)
    b = g.box_like(box)
    hin = torch.zeros(g.state_shape(b), dtype=torch.float64, pin_memory=True)
    hin[..., :box.nx + 6] = torch.from_numpy(np.ascontiguousarray(s0))
    hout = torch.empty_like(hin).pin_memory()
    g.grf_rk4_step_host(b, g.params_like(params), hin, hout, g.alloc_state(b), 0.25 * box.dx, 1)
    torch.cuda.synchronize()
    assert np.array_equal(hout.numpy()[..., :box.nx + 6], gpu)


@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN])
def test_decoupled_mode_parity(g, orc, bc):
    """4dST without backreaction: the RHS and 3 RK4 steps against the oracle's decoupled mode;
    the metric fields after the steps equal those of a vacuum evolution (couplings off, no
    scalar) to 1e-12."""
    box = gi.Box(14, 11, 9, 0.3, -2.0, -1.6, -1.3, bc=bc)
    params = P(lam=0.3, g2=0.2, beta_kind=1, decoupled=1)
    s0 = make_state(box, "perturbed", 23)
    s = s0.copy()
    if bc == gi.BC_PERIODIC:
        orc.fill_ghosts(box, s)
    ref = orc.rhs(box, params, s)
    out = gpu_rhs(g, box, params, s)
    errs = field_errors(out, ref, box, state=s, sigma=params.sigma_ko)
    assert np.max(errs) < 1e-11, describe(errs)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, 3)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 3)
    errs = field_errors(gpu, cpu, box)
    assert np.max(errs) < 1e-10, describe(errs)
    vac0 = s0.copy()
    vac0[25:27] = 0.0
    vac = gpu_rk4(g, box, P(lam=0.0, g2=0.0, beta_kind=1), vac0, 0.25 * box.dx, 3)
    errs = field_errors(gpu[:25], vac[:25], box)
    assert np.max(errs) < 1e-12, describe(errs)


def test_mirror_planes_parity(g, orc):
    """Mirror planes at the three low faces (GRF_BC_REFLECT_LOW) on a generic state: the ghost
    fill bit for bit against the oracle's, the RHS and 3 RK4 steps against the oracle's mirror
    boxes, and the host-to-host step's bits against the device step."""
    import torch
    box = gi.Box(17, 14, 12, 0.3, 0.15, 0.15, 0.15, bc=gi.BC_REFLECT_LOW)
    params = P(lam=0.3, g2=0.2, beta_kind=1)
    s0 = gi.random_perturbed_state(box, 29, base=gi.mirror_symmetric_state(box), eps=2e-2)
    assert np.all(np.isfinite(s0))
    b = g.box_like(box)
    t = g.to_device(s0, b)
    g.grf_fill_ghosts(b, t)
    filled = s0.copy()
    orc.fill_ghosts(box, filled)
    assert np.array_equal(g.to_host(t, b), filled)
    ref = orc.rhs(box, params, filled)
    out = gpu_rhs(g, box, params, s0)
    errs = field_errors(out, ref, box, state=filled, sigma=params.sigma_ko)
    assert np.max(errs) < 1e-11, describe(errs)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, 3)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 3)
    errs = field_errors(gpu, cpu, box)
    assert np.max(errs) < 1e-10, describe(errs)
    hin = torch.zeros(g.state_shape(b), dtype=torch.float64, pin_memory=True)
    hin[..., :box.nx + 6] = torch.from_numpy(np.ascontiguousarray(s0))
    hout = torch.empty_like(hin).pin_memory()
    g.grf_rk4_step_host(b, g.params_like(params), hin, hout, g.alloc_state(b), 0.25 * box.dx, 3)
    torch.cuda.synchronize()
    assert np.array_equal(hout.numpy()[..., :box.nx + 6], gpu)


def test_constraints_parity(g, orc):
    box = gi.Box(13, 12, 10, 0.3, -1.9, -1.7, -1.4)
    params = P(lam=0.3, g2=0.2)
    s = make_state(box, "perturbed", 21)
    orc.enforce(box, params, s)
    orc.fill_ghosts(box, s)
    ref = orc.constraints(box, params, s)
    b = g.box_like(box)
    t = g.to_device(s, b)
    out = g.alloc_state(b, 4)
    norms = g.grf_constraints(b, g.params_like(params), t, out)
    got = g.to_host(out, b)
    gg = box.interior(got[:4])
    for m in range(4):
        den = np.max(np.abs(ref[m]))
        assert np.max(np.abs(gg[m] - ref[m])) <= 1e-11 * den, m
        np.testing.assert_allclose(norms[2 * m], math.sqrt(np.mean(ref[m] ** 2)), rtol=1e-11)
        np.testing.assert_allclose(norms[2 * m + 1], np.max(np.abs(ref[m])), rtol=1e-11)


@pytest.mark.parametrize("bc,decoupled", [(gi.BC_PERIODIC, 0), (gi.BC_FROZEN, 1)])
def test_energy_densities_parity(g, orc, bc, decoupled):
    """The three energy densities (X, g2 X^2 and Gauss-Bonnet terms) against the oracle's split
    of its covariant stress tensor, each to 1e-11 of its own maximum; the split does not depend
    on whether the scalar backreacts. Ghosts of the device state are refilled by the call."""
    box = gi.Box(15, 11, 13, 0.3, -2.1, -1.5, -1.8, bc=bc)
    params = P(lam=0.3, g2=0.2, beta_kind=1, decoupled=decoupled)
    s = make_state(box, "perturbed", 31)
    orc.enforce(box, params, s)
    filled = s.copy()
    orc.fill_ghosts(box, filled)
    ref = orc.energy_densities(box, params, filled)
    b = g.box_like(box)
    t = g.to_device(s, b)
    out = g.alloc_state(b, 3)
    g.grf_energy_densities(b, g.params_like(params), t, out)
    assert g.grf_check_status() == 0
    got = box.interior(g.to_host(out, b)[:3])
    for m in range(3):
        den = np.max(np.abs(ref[m]))
        assert den > 0, m
        assert np.max(np.abs(got[m] - ref[m])) <= 1e-11 * den, m


@pytest.mark.parametrize("g3,decoupled", [(0.0, 0), (0.1, 0), (0.0, 1)])
def test_bl_pair_256_sampled_outputs(g, orc, g3, decoupled):
    """Full-size 256^3 Brill-Lindquist workload, one RK4 step in the production launch
    configuration; sampled points are recomputed by the oracle on 19^3 frozen-ghost sub-boxes
    centred on them (one RK4 step has a domain of dependence of 12 points, so the centre of
    such a sub-box is exact). Each field agrees to 1e-11 of its scale, or to 64 times the
    oracle's own rounding noise at the point where that is larger. g3 = 0.1 is the cubic
    workload's launch (`bench.py --g3 0.1`: the general instantiation with the cubic branch),
    decoupled = 1 that of `bench.py --decoupled` (the stage kernel without backreaction)."""
    cfg = gi.config_bl_pair_256()
    box, params, dt = cfg["box"], cfg["params"], cfg["dt"]
    params.g3 = g3
    params.decoupled = decoupled
    s0 = cfg["make_state"]()
    gpu = gpu_rk4(g, box, params, s0, dt, 1)
    assert np.all(np.isfinite(box.interior(gpu)))
    orc.fill_ghosts(box, s0)
    rng = np.random.default_rng(5)
    samples = [(128, 128, 128 + 24), (3, 200, 77)] + [tuple(int(x) for x in rng.integers(0, 256, 3)) for _ in range(2)]
    # the 8 grid points around each puncture (z = +-3): where the fields sourced by the lapse and
    # the curvature peak, so the oracle's values there give each field's scale over the box
    samples += [(i, j, k) for k in (103, 104, 151, 152) for j in (127, 128) for i in (127, 128)]
    R = 9
    refs, noise, gots = [], [], []
    for (i, j, k) in samples:
        sub = gi.Box(2 * R + 1, 2 * R + 1, 2 * R + 1, box.dx, 0.0, 0.0, 0.0, bc=gi.BC_FROZEN)
        idx = [(np.arange(2 * R + 7) + c - R - 3) % 256 + 3 for c in (k, j, i)]
        ss0 = np.ascontiguousarray(s0[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]])
        ss = ss0.copy()
        orc.rk4(sub, params, ss, dt, 1)
        ref = ss[:, R + 3, R + 3, R + 3]
        # the oracle's own rounding noise at this point: the spread of its result when every
        # input is perturbed by about one unit in the last place
        spread = np.zeros(ref.shape)
        for seed in (1, 2):
            sp = ss0 * (1.0 + 2.0 ** -52 * np.random.default_rng(seed).standard_normal(ss0.shape))
            orc.rk4(sub, params, sp, dt, 1)
            spread = np.maximum(spread, np.abs(sp[:, R + 3, R + 3, R + 3] - ref))
        refs.append(ref)
        noise.append(spread)
        gots.append(gpu[:, k + 3, j + 3, i + 3])
    refs, noise, gots = np.array(refs), np.array(noise), np.array(gots)
    # per-field scale from the inputs and the oracle only: the field's maximum over the whole
    # initial box, or over the oracle's sampled results (which include the points next to the
    # punctures) for fields that start at zero
    scale = np.maximum(np.maximum(np.max(np.abs(box.interior(s0)), axis=(1, 2, 3)), np.max(np.abs(refs), axis=0)),
                       1e-12)
    # A field that one step sources by cancelling terms (the A_ij, of order 1e-7 here while the
    # terms that make them are of order 1) carries rounding above 1e-11 of its own scale; there
    # the bound is 64 times the oracle's rounding noise at the point instead
    for n, (i, j, k) in enumerate(samples):
        err = np.abs(gots[n] - refs[n]) / np.maximum(1e-11 * scale, 64.0 * noise[n])
        assert np.max(err) < 1.0, (i, j, k, describe(err))


def test_error_codes(g):
    import torch
    box = gi.cube_box(8, -1.0, 1.0)
    b = g.box_like(box)
    t = g.alloc_state(b)
    p = g.params_like(P())
    small = g.alloc_workspace(1024)
    with pytest.raises(g.GrfError) as e:
        g.grf_rk4_step(b, p, t, 0.1, 1, ws=small)
    assert e.value.code == g.GRF_EWORKSPACE
    bad = g.box_like(box)
    bad.nx = 2  # periodic boxes need >= 3 points per axis
    with pytest.raises(g.GrfError) as e:
        g.grf_rhs(bad, p, t, t)
    assert e.value.code == g.GRF_EINVAL
    pb = g.params_like(P(beta_kind=7))
    with pytest.raises(g.GrfError):
        g.grf_rhs(b, pb, t, g.alloc_state(b))
    s = gi.single_puncture(box)
    t = g.to_device(s, b)
    assert g.grf_check_finite(b, t) == 0
    t[5, 5, 5, 5] = float("nan")
    assert g.grf_check_finite(b, t) == g.GRF_ENONFINITE
    torch.cuda.synchronize()


@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN])
def test_exponential_coupling_parity(g, orc, bc):
    """The exponential Gauss-Bonnet coupling (GRF_BETA_EXPONENTIAL): RHS and 3 RK4 steps against the
    oracle on a state whose scalar is large enough for e^{-kappa phi^2} to matter."""
    box = gi.Box(13, 11, 10, 0.3, -1.95, -1.65, -1.5, bc=bc)
    params = P(lam=0.3, g2=0.2, beta_kind=gi.BETA_EXPONENTIAL, beta_kappa=2.0)
    s0 = make_state(box, "perturbed", 37)
    s0[25] += 0.6 * np.exp(-sum(c ** 2 for c in box.coords()) / 4.0)
    s = s0.copy()
    if bc == gi.BC_PERIODIC:
        orc.fill_ghosts(box, s)
    ref = orc.rhs(box, params, s)
    out = gpu_rhs(g, box, params, s)
    errs = field_errors(out, ref, box, state=s, sigma=params.sigma_ko)
    assert np.max(errs) < 1e-11, describe(errs)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, 3)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 3)
    errs = field_errors(gpu, cpu, box)
    assert np.max(errs) < 1e-10, describe(errs)


@pytest.mark.parametrize("case", ["ragged_perturbed_linear", "ragged_perturbed_quadratic", "single_point_frozen"])
def test_hyperbolicity_parity(g, orc, case):
    """grf_hyperbolicity (det M of the coupled system from the kernel's closed-form assembly and
    its own LU; the effective-metric determinant by the determinant lemma; -g_eff^nn) against the
    oracle (its residual's Jacobian and long-double full-pivot determinants) to 1e-11."""
    box, params, kind, seed = RHS_CASES[case]()
    s = make_state(box, kind, seed)
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
    assert np.min(ref[0]) != 1.0  # the couplings make the system non-trivial
