"""grf_rk4_step_host: the RK4 step from host memory to host memory with the copies overlapped
with the first and last stage (slabs of z-planes on a library copy stream). Its result must be
bit-identical to copying the state to the device, grf_rk4_step, and copying it back: the same
kernels compute every point from the same inputs, only the order in which slabs are launched
differs."""
import numpy as np
import pytest

import grf_inputs as gi

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


def host_state(g, box, s0, pinned=True, poison_ghosts=False):
    """Padded host array (state_shape) holding s0; periodic ghosts optionally set to NaN (they
    must not be read)."""
    import torch
    b = g.box_like(box)
    s = np.array(s0, dtype=np.float64)
    if poison_ghosts:
        s[:, :3] = np.nan
        s[:, box.nz + 3:] = np.nan
        s[:, :, :3] = np.nan
        s[:, :, box.ny + 3:] = np.nan
        s[..., :3] = np.nan
        s[..., box.nx + 3:] = np.nan
    t = torch.zeros(g.state_shape(b), dtype=torch.float64, pin_memory=pinned)
    t[..., :box.nx + 6] = torch.from_numpy(s)
    return t


def same_state(box, a, b):
    """Equal on the ghosted extent (the row padding beyond nx + 6 is not part of the state)."""
    import torch
    return torch.equal(a[..., :box.nx + 6], b[..., :box.nx + 6])


def reference(g, b, params, hin, dt, nsteps):
    dev = hin.cuda()
    g.grf_rk4_step(b, params, dev, dt, nsteps)
    return dev.cpu()


def initial(box, seed):
    return gi.random_perturbed_state(box, seed, base=gi.single_puncture(box, amp=0.05), eps=2e-2)


CASES = {
    # name: (box, nsteps)
    "periodic_ragged_10_slabs": (gi.Box(20, 14, 37, 0.3, -2.8, -2.0, -5.4), 1),
    "frozen_14_slabs_2_steps": (gi.Box(13, 9, 70, 0.3, -1.9, -1.3, -10.2, bc=gi.BC_FROZEN), 2),
    "periodic_minimal_one_slab": (gi.Box(3, 3, 3, 0.4, -0.5, -0.5, -0.5), 2),
    "frozen_single_plane": (gi.Box(5, 4, 1, 0.3, 0.9, 0.6, -1.2, bc=gi.BC_FROZEN), 1),
    "periodic_two_slabs_3_steps": (gi.Box(12, 10, 8, 0.3, -1.7, -1.4, -1.1), 3),
    "periodic_lopsided_8_slabs": (gi.Box(17, 12, 33, 0.3, -2.5, -1.7, -4.8), 2),
}
LOPSIDED = {"periodic_lopsided_8_slabs"}


@pytest.mark.parametrize("case", sorted(CASES))
def test_host_step_bit_identical_to_device_step(g, case):
    import torch
    box, nsteps = CASES[case]
    b = g.box_like(box)
    params = g.params_like(gi.Params(lam=0.2, g2=0.1, beta_kind=gi.BETA_QUADRATIC,
                                     advection=1 if case in LOPSIDED else 0))
    periodic = box.bc == gi.BC_PERIODIC
    hin = host_state(g, box, initial(box, 5), poison_ghosts=periodic)
    dt = 0.25 * box.dx
    ref = reference(g, b, params, hin, dt, nsteps)
    hout = torch.full_like(hin, float("nan")).pin_memory()
    state = torch.full(g.state_shape(b), float("nan"), dtype=torch.float64, device="cuda")
    g.grf_rk4_step_host(b, params, hin, hout, state, dt, nsteps)
    torch.cuda.synchronize()
    assert same_state(box, hout, ref), case
    assert same_state(box, state.cpu(), ref), case
    assert g.grf_check_status() == 0


def test_host_step_in_place_back_to_back_on_a_side_stream(g):
    """Two calls queued without a synchronisation in between, host_in == host_out, on a
    non-default stream: the second call's copies must see the first call's result."""
    import torch
    box = gi.Box(16, 12, 29, 0.3, -2.2, -1.6, -4.2)
    b = g.box_like(box)
    params = g.params_like(gi.Params(lam=0.3, g2=0.05))
    h = host_state(g, box, initial(box, 9))
    dt = 0.25 * box.dx
    ref = reference(g, b, params, h, dt, 2)
    state = g.alloc_state(b)
    ws = g.alloc_workspace(g.grf_workspace_bytes(b, g.GRF_OP_RK4))
    side = torch.cuda.Stream()
    g.grf_rk4_step_host(b, params, h, h, state, dt, 1, ws=ws, stream=side)
    g.grf_rk4_step_host(b, params, h, h, state, dt, 1, ws=ws, stream=side)
    side.synchronize()
    assert same_state(box, h, ref)


def test_host_step_pageable_numpy_buffers(g):
    import torch
    box = gi.Box(11, 13, 21, 0.3, -1.6, -1.9, -3.1, bc=gi.BC_FROZEN)
    b = g.box_like(box)
    params = g.params_like(gi.Params(lam=0.1, g2=0.2))
    hin = host_state(g, box, initial(box, 3), pinned=False).numpy()
    hout = np.full_like(hin, np.nan)
    ref = reference(g, b, params, torch.from_numpy(hin), 0.25 * box.dx, 1)
    g.grf_rk4_step_host(b, params, hin, hout, g.alloc_state(b), 0.25 * box.dx, 1)
    torch.cuda.synchronize()
    assert np.array_equal(hout[..., :box.nx + 6], ref.numpy()[..., :box.nx + 6])


def test_host_step_zero_steps_is_a_round_trip(g):
    import torch
    box = gi.Box(7, 6, 9, 0.3, 0.1, 0.2, 0.3)
    b = g.box_like(box)
    hin = host_state(g, box, initial(box, 4))
    hout = torch.zeros_like(hin).pin_memory()
    state = g.alloc_state(b)
    g.grf_rk4_step_host(b, g.params_like(gi.Params()), hin, hout, state, 0.1, 0)
    torch.cuda.synchronize()
    assert same_state(box, hout, hin) and same_state(box, state.cpu(), hin)


def test_host_step_sixteen_slabs_128(g):
    """128^3: 16 slabs of 8 planes (the largest slab count) on the Brill-Lindquist pair."""
    import torch
    cfg = gi.config_bl_pair_256(128)
    box = cfg["box"]
    b = g.box_like(box)
    p = g.params_like(cfg["params"])
    hin = host_state(g, box, cfg["make_state"]())
    dt = cfg["dt"]
    ref = reference(g, b, p, hin, dt, 1)
    hout = torch.empty_like(hin).pin_memory()
    g.grf_rk4_step_host(b, p, hin, hout, g.alloc_state(b), dt, 1)
    torch.cuda.synchronize()
    assert same_state(box, hout, ref)


def test_host_step_pinned_input_pageable_output(g):
    """Page-locked host_in (copied in by the SMs) with a pageable host_out (copied out by
    cudaMemcpyAsync): both copy paths in one call."""
    import torch
    box = gi.Box(18, 10, 23, 0.3, -2.6, -1.4, -3.3)
    b = g.box_like(box)
    params = g.params_like(gi.Params(lam=0.15, g2=0.05, beta_kind=gi.BETA_QUADRATIC))
    hin = host_state(g, box, initial(box, 11))
    hout = np.full(tuple(hin.shape), np.nan)
    ref = reference(g, b, params, hin, 0.25 * box.dx, 2)
    g.grf_rk4_step_host(b, params, hin, hout, g.alloc_state(b), 0.25 * box.dx, 2)
    torch.cuda.synchronize()
    assert np.array_equal(hout[..., :box.nx + 6], ref.numpy()[..., :box.nx + 6])


OTHER_BOXES = {
    # boxes outside the slab pipeline: whole-state copies around the device step
    "sixth_order_periodic": (gi.Box(14, 11, 12, 0.3, -2.0, -1.6, -1.8, ng=4), dict()),
    "sommerfeld": (gi.Box(14, 12, 11, 0.3, -1.95, -1.65, -1.5, bc=gi.BC_SOMMERFELD), dict()),
    "extrapolating_lopsided": (gi.Box(13, 12, 10, 0.3, -1.8, -1.65, -1.35, bc=gi.BC_EXTRAPOLATE), dict(advection=1)),
    "mirror_sommerfeld_sixth": (gi.Box(12, 11, 10, 0.3, 0.15, 0.15, 0.15, bc=gi.BC_REFLECT_LOW_SOMMERFELD, ng=4),
                                dict()),
}


@pytest.mark.parametrize("case", sorted(OTHER_BOXES))
def test_host_step_other_boxes_bit_identical(g, case):
    import torch
    box, extra = OTHER_BOXES[case]
    b = g.box_like(box)
    params = g.params_like(gi.Params(lam=0.2, g2=0.1, beta_kind=gi.BETA_QUADRATIC, **extra))
    base = gi.mirror_symmetric_state(box) if box.bc == gi.BC_REFLECT_LOW_SOMMERFELD else None
    s0 = gi.random_perturbed_state(box, 13, base=base if base is not None else gi.single_puncture(box, amp=0.05),
                                   eps=2e-2)
    hin = torch.zeros(g.state_shape(b), dtype=torch.float64, pin_memory=True)
    hin[..., :box.nx + 2 * box.ng] = torch.from_numpy(s0)
    dt = 0.25 * box.dx
    dev = hin.cuda()
    g.grf_rk4_step(b, params, dev, dt, 2)
    ref = dev.cpu()
    hout = torch.full_like(hin, float("nan")).pin_memory()
    g.grf_rk4_step_host(b, params, hin, hout, g.alloc_state(b), dt, 2)
    torch.cuda.synchronize()
    w = box.nx + 2 * box.ng
    assert torch.equal(hout[..., :w], ref[..., :w]), case
