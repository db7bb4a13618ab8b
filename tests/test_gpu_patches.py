"""One box (periodic, or with frozen ghosts) evolved as patches with a halo exchange after every RK4 stage
(grf_patches_rk4, grf_halo_exchange, grf_patch_copy) on the GPU.

The exchange and the copies move values only, so they are checked bit for bit against the
periodic images of the whole box. Each patch's stage runs the batched stage kernel on the same
values the whole-box stage reads, so the patches' interiors after nsteps steps must equal,
bit for bit, grf_rk4_step on the whole box (itself checked against the oracle in
test_gpu_parity.py); one case is also compared with the oracle directly.
"""
import ctypes as C

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


def offsets(n, p):
    return [(a * n) // p for a in range(p + 1)]


def periodic_block(whole, box, lo, n):
    """The ghosted block of the periodic box that a patch with interior [lo, lo + n) holds."""
    idx = [np.arange(l - 3, l + m + 3) % N for l, m, N in zip(lo, n, (box.nx, box.ny, box.nz))]
    return whole[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]


def split(g, box, s, p):
    """The patches of a host state of the whole box, interiors copied on the device, ghosts exchanged."""
    b = g.box_like(box)
    L = g.patch_level(b, *p)
    whole = g.to_device(s, b)
    patches = g.patch_states(L)
    g.grf_patch_copy(L, whole, patches, 0)
    g.grf_halo_exchange(L, patches)
    return L, patches


@pytest.mark.parametrize("n,p", [((29, 22, 17), (3, 2, 2)), ((16, 16, 16), (1, 1, 1)), ((9, 8, 12), (3, 4, 4)),
                                 ((40, 6, 6), (16, 2, 1)), ((16, 16, 5), (16, 16, 1)), ((3, 3, 3), (3, 3, 3))])
def test_exchange_writes_the_periodic_images(g, n, p):
    """Every patch, ghosts included, equals the block of the periodic box it stands for (patches
    narrower than the 3 ghost layers read their ghosts from patches two or more away)."""
    box = gi.Box(*n, 0.2, 0.0, 0.0, 0.0)
    s = np.random.default_rng(1).normal(size=box.shape)
    whole = s[:, 3:-3, 3:-3, 3:-3]
    L, patches = split(g, box, s, p)
    ox, oy, oz = offsets(n[0], p[0]), offsets(n[1], p[1]), offsets(n[2], p[2])
    for c in range(p[2]):
        for b in range(p[1]):
            for a in range(p[0]):
                q = a + p[0] * (b + p[1] * c)
                pb = g.grf_patch_box(L, q)
                lo, m = (ox[a], oy[b], oz[c]), (pb.nx, pb.ny, pb.nz)
                assert np.array_equal(g.to_host(patches[q], pb), periodic_block(whole, box, lo, m)), q


@pytest.mark.parametrize("n,p", [((29, 22, 17), (3, 2, 2)), ((9, 8, 2), (3, 4, 2)), ((7, 5, 4), (1, 1, 1))])
def test_exchange_in_a_frozen_box(g, n, p):
    """Frozen box: each patch equals the block of the ghosted box it covers; ghosts inside the box
    come from the neighbouring patches, those outside it are the box's own ghosts, left as copied."""
    box = gi.Box(*n, 0.2, 0.0, 0.0, 0.0, bc=gi.BC_FROZEN)
    s = np.random.default_rng(3).normal(size=box.shape)
    L, patches = split(g, box, s, p)
    ox, oy, oz = offsets(n[0], p[0]), offsets(n[1], p[1]), offsets(n[2], p[2])
    for c in range(p[2]):
        for b in range(p[1]):
            for a in range(p[0]):
                q = a + p[0] * (b + p[1] * c)
                pb = g.grf_patch_box(L, q)
                want = s[:, oz[c]:oz[c] + pb.nz + 6, oy[b]:oy[b] + pb.ny + 6, ox[a]:ox[a] + pb.nx + 6]
                assert np.array_equal(g.to_host(patches[q], pb), want), q


def test_patch_copy_round_trip(g):
    box = gi.Box(21, 13, 10, 0.2, 0.0, 0.0, 0.0)
    s = np.random.default_rng(2).normal(size=box.shape)
    b = g.box_like(box)
    L, patches = split(g, box, s, (2, 3, 2))
    back = g.alloc_state(b)
    back.zero_()
    g.grf_patch_copy(L, back, patches, 1)
    got = g.to_host(back, b)
    assert np.array_equal(got[:, 3:-3, 3:-3, 3:-3], s[:, 3:-3, 3:-3, 3:-3])
    assert not np.any(got[:, :3]) and not np.any(got[:, :, :, -3:])  # the box's ghosts are left alone


def whole_and_patches(g, box, params, s, p, dt, nsteps, exchange=None):
    b, gp = g.box_like(box), g.params_like(params)
    t = g.to_device(s, b)
    g.grf_rk4_step(b, gp, t, dt, nsteps)
    assert g.grf_check_status() == 0
    ref = g.to_host(t, b)
    L, patches = split(g, box, s, p)
    g.grf_patches_rk4(L, gp, patches, dt, nsteps, exchange=exchange)
    out = g.alloc_state(b)
    g.grf_patch_copy(L, out, patches, 1)
    return ref, g.to_host(out, b)


@pytest.mark.parametrize("p", [(2, 2, 2), (1, 1, 1), (4, 1, 3), (3, 2, 5), (16, 1, 1), (8, 16, 2)])
def test_patches_equal_the_whole_box_bit_for_bit(g, p):
    """32^3 single puncture: 32-wide patches take the block gather, 16- and 8-wide ones the folded
    per-thread gather, ragged ones (10 / 11 points) partial rows; patches of 2 points along an axis
    read their ghosts from patches up to two away; 256 patches is the most a level takes."""
    cfg = gi.config_single_puncture_32()
    box, params, dt = cfg["box"], cfg["params"], cfg["dt"]
    s = cfg["make_state"]()
    ref, got = whole_and_patches(g, box, params, s, p, dt, 2)
    assert np.array_equal(got[:, 3:-3, 3:-3, 3:-3], ref[:, 3:-3, 3:-3, 3:-3])


@pytest.mark.parametrize("params", [gi.Params(lam=0.05, g2=0.02, advection=1),
                                    gi.Params(lam=0.3, g2=0.1, beta_kind=2, beta_kappa=1.5),
                                    gi.Params(lam=0.2, g2=0.1, decoupled=1)])
def test_patches_other_schemes_bit_for_bit(g, params):
    """Lopsided advection, the exponential coupling and the decoupled mode on a ragged box."""
    box = gi.Box(26, 19, 14, 0.3, -3.9, -2.85, -2.1)
    s = gi.random_perturbed_state(box, 5, base=gi.single_puncture(box, amp=0.05), eps=2e-2)
    ref, got = whole_and_patches(g, box, params, s, (2, 3, 2), 0.25 * box.dx, 2)
    assert np.array_equal(got[:, 3:-3, 3:-3, 3:-3], ref[:, 3:-3, 3:-3, 3:-3])


@pytest.mark.parametrize("p", [(2, 3, 2), (3, 1, 4), (1, 1, 1)])
def test_patches_of_a_frozen_box_bit_for_bit(g, p):
    """A box with frozen ghosts (single-puncture data in them): the patches on its faces keep
    those ghosts through the stages, the inner faces are exchanged."""
    box = gi.Box(26, 19, 14, 0.3, -3.9, -2.85, -2.1, bc=gi.BC_FROZEN)
    s = gi.random_perturbed_state(box, 6, base=gi.single_puncture(box, amp=0.05), eps=2e-2)
    ref, got = whole_and_patches(g, box, gi.Params(lam=0.1, g2=0.05, beta_kind=1), s, p, 0.25 * box.dx, 3)
    assert np.array_equal(got[:, 3:-3, 3:-3, 3:-3], ref[:, 3:-3, 3:-3, 3:-3])


def test_patches_256_bit_for_bit_at_full_size(g):
    """The split-box bench workload at full size: the 256^3 Brill-Lindquist box as 2 x 2 x 2 patches
    of 128^3, one step, against the whole box's step, bit for bit (compared on the device)."""
    import torch
    cfg = gi.config_bl_pair_256()
    box, params, dt = cfg["box"], cfg["params"], cfg["dt"]
    b, p = g.box_like(box), g.params_like(params)
    whole = g.to_device(cfg["make_state"](), b)
    level = g.patch_level(b, 2, 2, 2)
    patches = g.patch_states(level)
    g.grf_patch_copy(level, whole, patches, 0)
    g.grf_patches_rk4(level, p, patches, dt, 1)
    g.grf_rk4_step(b, p, whole, dt, 1)
    out = torch.zeros_like(whole)
    g.grf_patch_copy(level, out, patches, 1)
    torch.cuda.synchronize()
    n = 3 + box.nx
    assert torch.equal(out[:, 3:-3, 3:-3, 3:n], whole[:, 3:-3, 3:-3, 3:n])
    del patches, out, whole
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN])
def test_constraints_over_patches(g, bc):
    """H and M_i of every patch equal the whole box's at the same points, bit for bit; the norms
    combined from the patches equal the whole box's (maxima exactly, L2 to the summation order)."""
    box = gi.Box(26, 19, 14, 0.3, -3.9, -2.85, -2.1, bc=bc)
    s = gi.random_perturbed_state(box, 7, base=gi.single_puncture(box, amp=0.05), eps=1e-2)
    params = g.params_like(gi.Params(lam=0.1, g2=0.05, beta_kind=1))
    b = g.box_like(box)
    whole = g.to_device(s, b)
    out_w = g.alloc_state(b, 4)
    nw = g.grf_constraints(b, params, whole, out_w)
    p = (2, 3, 2)
    L, patches = split(g, box, s, p)
    outs = [g.alloc_state(g.grf_patch_box(L, q), 4) for q in range(len(patches))]
    npch = g.grf_patches_constraints(L, params, patches, outs)
    ox, oy, oz = offsets(box.nx, p[0]), offsets(box.ny, p[1]), offsets(box.nz, p[2])
    w = g.to_host(out_w, b)
    for c in range(p[2]):
        for bb in range(p[1]):
            for a in range(p[0]):
                q = a + p[0] * (bb + p[1] * c)
                pb = g.grf_patch_box(L, q)
                got = g.to_host(outs[q], pb)[:, 3:-3, 3:-3, 3:-3]
                want = w[:, 3 + oz[c]:3 + oz[c] + pb.nz, 3 + oy[bb]:3 + oy[bb] + pb.ny, 3 + ox[a]:3 + ox[a] + pb.nx]
                assert np.array_equal(got, want), q
    assert np.array_equal(npch[1::2], nw[1::2])
    np.testing.assert_allclose(npch[0::2], nw[0::2], rtol=1e-13, atol=0)


def test_patches_parity_with_the_oracle(g, orc):
    box = gi.Box(24, 20, 18, 0.3, -3.6, -3.0, -2.7)
    params = gi.Params(lam=0.1, g2=0.05, beta_kind=1)
    s = gi.random_perturbed_state(box, 9, base=gi.single_puncture(box, amp=0.05), eps=1e-2)
    b = g.box_like(box)
    L, patches = split(g, box, s, (3, 2, 2))
    dt = 0.25 * box.dx
    g.grf_patches_rk4(L, g.params_like(params), patches, dt, 2)
    out = g.alloc_state(b)
    g.grf_patch_copy(L, out, patches, 1)
    cpu = s.copy()
    orc.fill_ghosts(box, cpu)
    orc.rk4(box, params, cpu, dt, 2)
    errs = field_errors(g.to_host(out, b), cpu, box)
    assert np.max(errs) < 1e-11, describe(errs)


def test_exchange_is_pluggable(g):
    """A caller's exchange (here one that counts its calls and forwards to the built-in one) takes
    the built-in one's place: called once before the first step and once after every stage, with
    the same result bits."""
    cfg = gi.config_single_puncture_32()
    box, params, dt = cfg["box"], cfg["params"], cfg["dt"]
    s = cfg["make_state"]()
    calls = []

    def exchange(level, ptrs, stream):
        calls.append(stream)
        return g.lib().grf_halo_exchange(level, ptrs, stream)

    nsteps = 3
    ref, got = whole_and_patches(g, box, params, s, (2, 1, 2), dt, nsteps, exchange=exchange)
    assert len(calls) == 1 + 4 * nsteps
    assert np.array_equal(got[:, 3:-3, 3:-3, 3:-3], ref[:, 3:-3, 3:-3, 3:-3])


def test_failing_exchange_ends_the_step(g):
    """An exchange that reports an error (a lost peer, say) ends grf_patches_rk4 with its code after
    the stage already in flight; no kernel waits on it."""
    cfg = gi.config_single_puncture_32()
    box, params, dt = cfg["box"], cfg["params"], cfg["dt"]
    s = cfg["make_state"]()
    calls = []

    def exchange(level, ptrs, stream):
        calls.append(1)
        return g.GRF_ETIMEOUT if len(calls) == 3 else g.lib().grf_halo_exchange(level, ptrs, stream)

    L, patches = split(g, box, s, (2, 2, 1))
    with pytest.raises(g.GrfError) as e:
        g.grf_patches_rk4(L, g.params_like(params), patches, dt, 2, exchange=exchange)
    assert e.value.code == g.GRF_ETIMEOUT and len(calls) == 3
    import torch
    torch.cuda.synchronize()  # the context is still usable
    g.grf_halo_exchange(L, patches)
    torch.cuda.synchronize()


def test_exchange_that_raises(g):
    """A Python exchange that raises ends the step after the stage in flight, and the exception
    reaches the caller."""
    cfg = gi.config_single_puncture_32()
    box, params, dt = cfg["box"], cfg["params"], cfg["dt"]
    L, patches = split(g, box, cfg["make_state"](), (1, 2, 2))

    def exchange(level, ptrs, stream):
        raise KeyError("peer lost")

    with pytest.raises(KeyError):
        g.grf_patches_rk4(L, g.params_like(params), patches, dt, 1, exchange=exchange)
    import torch
    torch.cuda.synchronize()


@pytest.mark.parametrize("n,p,bc", [((12, 12, 12), (2, 2, 2), gi.BC_PERIODIC), ((8, 8, 8), (4, 4, 4), gi.BC_PERIODIC),
                                    ((10, 7, 9), (3, 1, 2), gi.BC_PERIODIC), ((9, 8, 7), (2, 3, 1), gi.BC_FROZEN)])
def test_device_exchange_equals_the_plan(g, n, p, bc):
    """The built-in device exchange and the exchange plan (grf_halo_plan, applied on the host)
    write the same ghost points with the same values, bit for bit."""
    from paper_2309_06225_gb300 import halo
    box = gi.Box(*n, 0.3, -1.0, -1.0, -1.0, bc=bc)
    level = g.patch_level(g.box_like(box), *p)
    rng = np.random.default_rng(3)
    host = []
    for q in range(p[0] * p[1] * p[2]):
        pb = g.grf_patch_box(level, q)
        host.append(rng.normal(size=(27, pb.nz + 6, pb.ny + 6, pb.pitch)))
    import torch
    dev = [torch.from_numpy(a.copy()).cuda() for a in host]
    g.grf_halo_exchange(level, dev)
    torch.cuda.synchronize()
    halo.apply_plan(g.grf_halo_plan(level), host)
    for q in range(len(host)):
        assert np.array_equal(dev[q].cpu().numpy(), host[q]), q
