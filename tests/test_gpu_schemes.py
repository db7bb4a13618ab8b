"""The 6th-order scheme (4 ghost layers) and lopsided advection on the GPU against the oracle
("Accuracy": 4th- and 6th-order finite differences; GRChombo's lopsided advection stencils).

Tolerances as in test_gpu_parity.py: one RHS evaluation <= 1e-11 of each field's maximum, three
RK4 steps <= 1e-10, ghost fills bit-exact.
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


def state_for(box, seed):
    """A generic state: the puncture plus seeded sinusoids in every field (the shift takes both
    signs); mirror boxes start from the mirror-symmetric state."""
    if box.bc == gi.BC_REFLECT_LOW:
        return gi.random_perturbed_state(box, seed, base=gi.mirror_symmetric_state(box), eps=2e-2)
    return gi.random_perturbed_state(box, seed, base=gi.single_puncture(box, amp=0.05), eps=3e-2)


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
    return s0, out, gpu


@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN, gi.BC_REFLECT_LOW])
def test_lopsided_advection_parity(g, orc, bc):
    """4th-order scheme with lopsided advection: RHS and 3 RK4 steps against the oracle, and
    the RHS visibly different from the centred one (the switch takes effect)."""
    box = gi.Box(14, 11, 9, 0.3, -2.0, -1.6, -1.3, bc=bc)
    if bc == gi.BC_REFLECT_LOW:
        box = gi.Box(14, 11, 9, 0.3, 0.15, 0.15, 0.15, bc=bc)
    params = P(lam=0.3, g2=0.2, beta_kind=1, advection=1)
    s0, lop, _ = check_rhs_and_rk4(g, orc, box, params, 41)
    cen = gpu_rhs(g, box, P(lam=0.3, g2=0.2, beta_kind=1), s0)
    assert np.max(np.abs(box.interior(lop) - box.interior(cen))) > 1e-6


def test_lopsided_advection_decoupled_parity(g, orc):
    """Lopsided advection without backreaction (the decoupled mode read at run time)."""
    box = gi.Box(12, 13, 10, 0.3, -1.8, -1.9, -1.5, bc=gi.BC_FROZEN)
    check_rhs_and_rk4(g, orc, box, P(lam=0.3, g2=0.2, beta_kind=1, advection=1, decoupled=1), 43, nsteps=2)


@pytest.mark.parametrize("advection", [0, 1])
@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN, gi.BC_REFLECT_LOW])
def test_sixth_order_parity(g, orc, bc, advection):
    """6th-order scheme (4 ghost layers): ghost fill bit-exact, RHS and 3 RK4 steps against the
    oracle, with centred and lopsided advection and every boundary type."""
    if bc == gi.BC_REFLECT_LOW:
        box = gi.Box(13, 11, 10, 0.3, 0.15, 0.15, 0.15, bc=bc, ng=4)
    else:
        box = gi.Box(13, 11, 10, 0.3, -1.9, -1.6, -1.5, bc=bc, ng=4)
    b = g.box_like(box)
    assert b.ng == 4
    s0 = state_for(box, 47)
    t = g.to_device(s0, b)
    g.grf_fill_ghosts(b, t)
    filled = s0.copy()
    orc.fill_ghosts(box, filled)
    assert np.array_equal(g.to_host(t, b), filled)
    check_rhs_and_rk4(g, orc, box, P(lam=0.3, g2=0.2, beta_kind=1, advection=advection), 47)


def test_sixth_order_ragged_multi_tile_rk4(g, orc):
    """A box spanning several 32 x 4 tiles with ragged edges in x and y, periodic, 6th order,
    lopsided advection, one RK4 step; and the no-allocation entry point gives the same bits."""
    box = gi.Box(37, 10, 6, 0.3, -5.5, -1.5, -0.9, ng=4)
    params = P(lam=0.2, g2=0.1, advection=1)
    s0 = state_for(box, 53)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, 1)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 1)
    errs = field_errors(gpu, cpu, box)
    assert np.max(errs) < 1e-11, describe(errs)
    b = g.box_like(box)
    t = g.to_device(s0, b)
    g.grf_rk4_step_noalloc(b, g.params_like(params), t, 0.25 * box.dx, 1)
    assert np.array_equal(g.to_host(t, b), gpu)


def test_sixth_order_ko_constraints_and_densities(g, orc):
    """The standalone 6th-order calls: dissipation (-sigma/(256 dx) Delta^8), constraints with
    their norms and the energy densities, against the oracle."""
    box = gi.Box(15, 12, 11, 0.3, -2.2, -1.8, -1.6, ng=4)
    params = P(lam=0.3, g2=0.2, beta_kind=1)
    s = state_for(box, 59)
    orc.enforce(box, params, s)
    orc.fill_ghosts(box, s)
    b = g.box_like(box)
    t = g.to_device(s, b)
    r = g.alloc_state(b)
    g.grf_ko_dissipation(b, 0.3, t, r)
    # smooth fields: Delta^8 is far below its 210 u_0 and 56 t_1 terms, whose rounding (~1e-16
    # sigma/dx |u|) sets the scale; the RHS bar with its dissipation floor applies
    errs = field_errors(g.to_host(r, b), orc.ko(box, 0.3, s), box, state=s, sigma=0.3)
    assert np.max(errs) < 1e-11, describe(errs)
    noise = np.random.default_rng(2).normal(size=box.shape)  # O(1) differences
    tn = g.to_device(noise, b)
    rn = g.alloc_state(b)
    g.grf_ko_dissipation(b, 0.3, tn, rn)
    errs = field_errors(g.to_host(rn, b), orc.ko(box, 0.3, noise), box)
    assert np.max(errs) < 1e-13, describe(errs)
    ref = orc.constraints(box, params, s)
    out = g.alloc_state(b, 4)
    norms = g.grf_constraints(b, g.params_like(params), t, out)
    got = box.interior(g.to_host(out, b)[:4])
    for m in range(4):
        den = np.max(np.abs(ref[m]))
        assert np.max(np.abs(got[m] - ref[m])) <= 1e-11 * den, m
        np.testing.assert_allclose(norms[2 * m], math.sqrt(np.mean(ref[m] ** 2)), rtol=1e-11)
        np.testing.assert_allclose(norms[2 * m + 1], np.max(np.abs(ref[m])), rtol=1e-11)
    dref = orc.energy_densities(box, params, s)
    d3 = g.alloc_state(b, 3)
    g.grf_energy_densities(b, g.params_like(params), t, d3)
    dgot = box.interior(g.to_host(d3, b)[:3])
    for m in range(3):
        assert np.max(np.abs(dgot[m] - dref[m])) <= 1e-11 * np.max(np.abs(dref[m])), m


def test_sixth_order_converges_faster_on_a_plane_wave(g):
    """The scalar plane wave on flat space, RHS only: the 6th-order scheme's error falls ~64x per
    halving of dx, the 4th-order one's ~16x (dissipation off, centred advection)."""
    amp, L = 1e-6, 2.0
    k = 2 * math.pi / L
    for ng, lo, hi in ((3, 13.0, 19.0), (4, 50.0, 72.0)):
        errs = []
        for n in (16, 32):
            box = gi.Box(n, 4, 4, L / n, 0.5 * L / n, 0.0, 0.0, ng=ng)
            s = gi.scalar_plane_wave(box, amp, (k, 0.0, 0.0))
            out = gpu_rhs(g, box, P(lam=0.0, g2=0.0, sigma_ko=0.0), s)
            X = box.interior(box.coords()[0])
            exact_dPi = -amp * k * k * np.sin(k * X)  # d_t Pi = lapse * Laplacian(phi) on flat space
            errs.append(np.max(np.abs(box.interior(out)[26] - exact_dPi)) / (amp * k * k))
        assert lo < errs[0] / errs[1] < hi, (ng, errs)


def _all_points_errors(gpu, cpu):
    """Per field max|gpu - cpu| over every point of the ghosted box / that field's maximum."""
    nf = cpu.shape[0]
    return np.array([np.max(np.abs(gpu[f] - cpu[f])) / max(np.max(np.abs(cpu[f])), 1e-12) for f in range(nf)])


@pytest.mark.parametrize("ng", [3, 4])
def test_extrapolating_boundaries_parity(g, orc, ng):
    """Extrapolating boxes ("Boundary Conditions"): the ghost fill bit for bit against the
    oracle's (the roundings are pinned on both sides), the RHS and 3 RK4 steps within the parity
    bar, for both schemes."""
    box = gi.Box(14, 11, 9, 0.3, -1.95, -1.5, -1.2, bc=gi.BC_EXTRAPOLATE, ng=ng)
    b = g.box_like(box)
    s0 = state_for(box, 61)
    t = g.to_device(s0, b)
    g.grf_fill_ghosts(b, t)
    filled = s0.copy()
    orc.fill_ghosts(box, filled)
    assert np.array_equal(g.to_host(t, b), filled)
    s, _, gpu = check_rhs_and_rk4(g, orc, box, P(lam=0.3, g2=0.2, beta_kind=1), 61)
    cpu = s0.copy()
    orc.rk4(box, P(lam=0.3, g2=0.2, beta_kind=1), cpu, 0.25 * box.dx, 3)
    errs = _all_points_errors(gpu, cpu)  # the returned ghosts are extrapolated from the new interior
    assert np.max(errs) < 1e-10, describe(errs)


@pytest.mark.parametrize("ng", [3, 4])
def test_sommerfeld_boundaries_parity(g, orc, ng):
    """Sommerfeld boxes around the origin: the RHS at interior and ghost points, and 3 RK4 steps
    with the ghosts evolved, at every point against the oracle."""
    n = (14, 11, 9)
    box = gi.Box(*n, 0.3, *(-(m - 1) * 0.15 for m in n), bc=gi.BC_SOMMERFELD, ng=ng)
    params = P(lam=0.3, g2=0.2, beta_kind=1)
    s0 = state_for(box, 67)
    ref = orc.rhs(box, params, s0)
    out = gpu_rhs(g, box, params, s0)
    errs = field_errors(out, ref, box, state=s0, sigma=params.sigma_ko)
    assert np.max(errs) < 1e-11, describe(errs)
    ghost = np.ones(s0.shape[1:], bool)
    ghost[ng:-ng, ng:-ng, ng:-ng] = False
    errs = _all_points_errors(out[:, ghost], ref[:, ghost])
    assert np.max(errs) < 1e-12, describe(errs)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, 3)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 3)
    errs = _all_points_errors(gpu, cpu)
    assert np.max(errs) < 1e-10, describe(errs)
    assert not np.array_equal(gpu[:, ghost], s0[:, ghost])  # the ghosts evolved


@pytest.mark.parametrize("ng", [3, 4])
def test_mirror_planes_with_sommerfeld_faces_parity(g, orc, ng):
    """Mirror planes at the low faces and Sommerfeld high faces (GRF_BC_REFLECT_LOW_SOMMERFELD): the
    ghost fill bit for bit, the RHS at the interior and the evolved high-face ghosts, and 3 RK4
    steps at every point against the oracle."""
    box = gi.Box(13, 11, 10, 0.3, 0.15, 0.15, 0.15, bc=gi.BC_REFLECT_LOW_SOMMERFELD, ng=ng)
    params = P(lam=0.3, g2=0.2, beta_kind=1)
    s0 = gi.random_perturbed_state(box, 83, base=gi.mirror_symmetric_state(box), eps=2e-2)
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
    som = np.zeros(s0.shape[1:], bool)
    som[ng:, ng:, ng:] = True
    som[ng:-ng, ng:-ng, ng:-ng] = False
    errs = _all_points_errors(out[:, som], ref[:, som])
    assert np.max(errs) < 1e-12, describe(errs)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, 3)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 3)
    errs = _all_points_errors(gpu, cpu)
    assert np.max(errs) < 1e-10, describe(errs)


@pytest.mark.parametrize("ng,advection", [(3, 1), (4, 0), (4, 1)])
def test_bl_pair_256_sampled_outputs_schemes(g, orc, ng, advection):
    """The 256^3 workload (bench.py --order / --advection) in its production launch, one RK4 step;
    sampled points recomputed by the oracle on frozen-ghost sub-boxes whose ghosts lie beyond the
    step's domain of dependence (4 stages x the stencil reach: 12 points with 3 ghost layers, 16
    with 4), so their centres are exact."""
    import dataclasses
    cfg = gi.config_bl_pair_256()
    box = dataclasses.replace(cfg["box"], ng=ng)
    params = P(**{k: v for k, v in cfg["params"].to_dict().items()})
    params.advection = advection
    s0 = gi.brill_lindquist_pair(box)
    gpu = gpu_rk4(g, box, params, s0, cfg["dt"], 1)
    assert np.all(np.isfinite(box.interior(gpu)))
    orc.fill_ghosts(box, s0)
    R = 16 - ng
    n = box.nx
    rng = np.random.default_rng(7 + ng + advection)
    samples = [(128, 128, 128 + 24)] + [tuple(int(x) for x in rng.integers(0, n, 3)) for _ in range(2)]
    scale = np.maximum(np.max(np.abs(box.interior(gpu)), axis=(1, 2, 3)), 1e-12)
    for (i, j, k) in samples:
        sub = gi.Box(2 * R + 1, 2 * R + 1, 2 * R + 1, box.dx, 0.0, 0.0, 0.0, bc=gi.BC_FROZEN, ng=ng)
        idx = [(np.arange(2 * R + 1 + 2 * ng) + c - R - ng) % n + ng for c in (k, j, i)]
        ss = np.ascontiguousarray(s0[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]])
        orc.rk4(sub, params, ss, cfg["dt"], 1)
        ref = ss[:, R + ng, R + ng, R + ng]
        got = gpu[:, k + ng, j + ng, i + ng]
        err = np.abs(got - ref) / scale
        assert np.max(err) < 1e-11, (i, j, k, describe(err))


@pytest.mark.parametrize("bc,ng", [(gi.BC_SOMMERFELD, 3), (gi.BC_EXTRAPOLATE, 4), (gi.BC_REFLECT_LOW_SOMMERFELD, 3)])
def test_outer_boundaries_multi_tile(g, orc, bc, ng):
    """Outer boundaries on a box spanning two 32-wide tiles with ragged x and y edges, 2 RK4 steps,
    every point against the oracle."""
    if bc == gi.BC_REFLECT_LOW_SOMMERFELD:
        box = gi.Box(37, 10, 6, 0.3, 0.15, 0.15, 0.15, bc=bc, ng=ng)
        s0 = gi.random_perturbed_state(box, 89, base=gi.mirror_symmetric_state(box), eps=2e-2)
    else:
        box = gi.Box(37, 10, 6, 0.3, -5.4, -1.35, -0.75, bc=bc, ng=ng)
        s0 = state_for(box, 89)
    params = P(lam=0.2, g2=0.1, beta_kind=1)
    cpu = s0.copy()
    orc.rk4(box, params, cpu, 0.25 * box.dx, 2)
    gpu = gpu_rk4(g, box, params, s0, 0.25 * box.dx, 2)
    errs = _all_points_errors(gpu, cpu)
    assert np.max(errs) < 1e-10, describe(errs)


def test_sixth_order_decoupled_parity(g, orc):
    """The 6th-order kernels read the decoupled mode at run time: RHS and 2 RK4 steps without
    backreaction against the oracle."""
    box = gi.Box(12, 11, 10, 0.3, -1.65, -1.5, -1.35, bc=gi.BC_PERIODIC, ng=4)
    check_rhs_and_rk4(g, orc, box, P(lam=0.3, g2=0.2, beta_kind=1, decoupled=1, advection=1), 97, nsteps=2)
