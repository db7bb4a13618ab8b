"""Batched RK4 over uneven boxes (grf_batched_rk4) on the GPU.

Every box of a batch runs the same device code as the single-box path, so the batched result
must equal, bit for bit, each box advanced alone with grf_rk4_step (which is itself checked
against the oracle in test_gpu_parity.py). One box is also compared with the oracle directly.
"""
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


def small_batch():
    """Uneven boxes: ragged sizes, both boundary types, different couplings and time steps."""
    boxes = [gi.Box(13, 9, 7, 0.25, -1.6, -1.1, -0.9, bc=gi.BC_FROZEN),
             gi.Box(8, 8, 8, 0.3, -1.05, -1.05, -1.05, bc=gi.BC_PERIODIC),
             gi.Box(24, 5, 11, 0.125, 0.3, -0.4, 0.2, bc=gi.BC_FROZEN),
             gi.Box(1, 1, 1, 0.1, 1.1, 0.7, 0.9, bc=gi.BC_FROZEN),
             gi.Box(16, 16, 8, 0.5, -3.75, -3.75, -1.75, bc=gi.BC_PERIODIC)]
    params = [gi.Params(lam=0.05, g2=0.02), gi.Params(lam=0.3, g2=0.1, beta_kind=1), gi.Params(lam=0.0, g2=0.0)]
    pidx = [0, 1, 2, 0, 1]
    states = [gi.random_perturbed_state(b, 40 + i, base=gi.single_puncture(b, amp=0.05), eps=2e-2)
              for i, b in enumerate(boxes)]
    assert all(np.all(np.isfinite(s)) for s in states)  # no grid point on the puncture
    dts = [0.25 * b.dx for b in boxes]
    return boxes, params, pidx, states, dts


@pytest.mark.parametrize("variant,tile", [(1, (32, 4, 1)), (2, (32, 4, 1)), (3, (16, 4, 2)), (1, (64, 2, 1)),
                                          (2, (16, 8, 1))])
def test_batched_equals_single_box_path(g, variant, tile):
    import torch
    boxes, params, pidx, states, dts = small_batch()
    gb = [g.box_like(b) for b in boxes]
    gp = g.params_array([g.params_like(p) for p in params])
    nsteps = 2
    ref = []
    for b, s, pi, dt in zip(gb, states, pidx, dts):
        t = g.to_device(s, b)
        g.grf_rk4_step(b, gp[pi], t, dt, nsteps)
        ref.append(g.to_host(t, b))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dev = [g.to_device(s, b) for s, b in zip(states, gb)]
        items = g.batch_items(gb, dev, pidx, dts)
        g.grf_batched_rk4(items, gp, nsteps, g.batch_config(variant, tile), stream=stream)
    stream.synchronize()
    for b, d, r in zip(gb, dev, ref):
        got = g.to_host(d, b)
        assert np.array_equal(got, r)


@pytest.mark.parametrize("variant,tile", [(1, (32, 4, 1)), (2, (32, 4, 1)), (3, (16, 4, 2))])
def test_batched_lopsided_advection_equals_single_box_path(g, variant, tile):
    """Boxes with lopsided advection (and one without backreaction) mixed with centred ones with the
    exponential coupling: each box's bits equal its single-box evolution, in every launch variant
    and gather mode."""
    import torch
    boxes, params, pidx, states, dts = small_batch()
    params = [gi.Params(lam=0.05, g2=0.02, advection=1), gi.Params(lam=0.3, g2=0.1, beta_kind=2, beta_kappa=1.5),
              gi.Params(lam=0.2, g2=0.1, advection=1, decoupled=1)]
    gb = [g.box_like(b) for b in boxes]
    gp = g.params_array([g.params_like(p) for p in params])
    nsteps = 2
    ref = []
    for b, s, pi, dt in zip(gb, states, pidx, dts):
        t = g.to_device(s, b)
        g.grf_rk4_step(b, gp[pi], t, dt, nsteps)
        ref.append(g.to_host(t, b))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dev = [g.to_device(s, b) for s, b in zip(states, gb)]
        items = g.batch_items(gb, dev, pidx, dts)
        g.grf_batched_rk4(items, gp, nsteps, g.batch_config(variant, tile), stream=stream)
    stream.synchronize()
    for b, d, r in zip(gb, dev, ref):
        assert np.array_equal(g.to_host(d, b), r)


def test_batched_graph_replay_and_oracle(g, orc):
    """Stepping the same batch twice replays the cached CUDA graph; the result after 2 x 1 steps
    equals 2 steps of the oracle for one of the boxes (within the parity tolerance)."""
    import torch
    boxes, params, pidx, states, dts = small_batch()
    gb = [g.box_like(b) for b in boxes]
    gp = g.params_array([g.params_like(p) for p in params])
    stream = torch.cuda.Stream()
    cfg = g.batch_config(g.GRF_BATCH_GRAPH, (32, 4, 1))
    with torch.cuda.stream(stream):
        dev = [g.to_device(s, b) for s, b in zip(states, gb)]
        items = g.batch_items(gb, dev, pidx, dts)
        ws = g.alloc_workspace(g.grf_batched_workspace_bytes(items, cfg))
        g.grf_batched_rk4(items, gp, 1, cfg, ws=ws, stream=stream)
        g.grf_batched_rk4(items, gp, 1, cfg, ws=ws, stream=stream)
    stream.synchronize()
    k = 0
    cpu = states[k].copy()
    orc.rk4(boxes[k], params[pidx[k]], cpu, dts[k], 2)
    errs = field_errors(g.to_host(dev[k], gb[k]), cpu, boxes[k])
    assert np.max(errs) < 1e-10, describe(errs)


@pytest.mark.parametrize("name", ["amr_boxes_96", "coupling_sweep_32"])
def test_full_size_batches_in_the_bench_launch(g, orc, name):
    """The batched bench workloads at full size (96 AMR-like boxes, 6.27M points; 32 x 64^3), in
    the launch the autotuner picks for them (graph of 32 x 4 x 1 tiles): after one step every box
    equals, bit for bit, the box stepped alone by grf_rk4_step, and the smallest, a middle and the
    largest box match one oracle step."""
    import torch
    import bench
    boxes, params, pidx, dts = bench.batched_workload(name)
    gb = [g.box_like(b) for b in boxes]
    gp = g.params_array([g.params_like(p) for p in params])
    init = [gi.single_puncture(b) for b in boxes]
    dev = [g.to_device(s, b) for s, b in zip(init, gb)]
    cfg = g.batch_config(g.GRF_BATCH_GRAPH, (32, 4, 1))
    items = g.batch_items(gb, dev, pidx, dts)
    g.grf_batched_rk4(items, gp, 1, cfg)
    torch.cuda.synchronize()
    for b2, s, d, pi, dt in zip(gb, init, dev, pidx, dts):
        t = g.to_device(s, b2)
        g.grf_rk4_step(b2, gp[pi], t, dt, 1)
        n = 3 + b2.nx
        assert torch.equal(t[:, 3:-3, 3:-3, 3:n], d[:, 3:-3, 3:-3, 3:n])
    sizes = [b.npoints for b in boxes]
    order = sorted(range(len(boxes)), key=lambda i: sizes[i])
    for k in (order[0], order[len(order) // 2], order[-1]):
        cpu = init[k].copy()
        orc.rk4(boxes[k], params[pidx[k]], cpu, dts[k], 1)
        errs = field_errors(g.to_host(dev[k], gb[k]), cpu, boxes[k])
        assert np.max(errs) < 1e-11, (k, describe(errs))


def test_persistent_barrier_timeout_is_reported_and_context_survives(g):
    """A grid barrier given a 1-cycle spin limit runs out (the other blocks have not arrived):
    the call returns GRF_ETIMEOUT instead of hanging, and the device stays usable."""
    import torch
    boxes, params, pidx, states, dts = small_batch()
    gb = [g.box_like(b) for b in boxes]
    gp = g.params_array([g.params_like(p) for p in params])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dev = [g.to_device(s, b) for s, b in zip(states, gb)]
        items = g.batch_items(gb, dev, pidx, dts)
        cfg = g.batch_config(g.GRF_BATCH_PERSISTENT, (32, 4, 1), barrier_timeout_cycles=1)
        with pytest.raises(g.GrfError) as e:
            g.grf_batched_rk4(items, gp, 3, cfg, stream=stream)
        assert e.value.code == g.GRF_ETIMEOUT
        # the context is still usable
        dev2 = [g.to_device(s, b) for s, b in zip(states, gb)]
        items2 = g.batch_items(gb, dev2, pidx, dts)
        g.grf_batched_rk4(items2, gp, 1, g.batch_config(g.GRF_BATCH_PERSISTENT, (32, 4, 1)), stream=stream)
    stream.synchronize()


def test_autotuner_picks_a_valid_config_and_caches(g, tmp_path):
    import torch
    from paper_2309_06225_gb300 import autotune
    boxes, params, pidx, states, dts = small_batch()
    gb = [g.box_like(b) for b in boxes]
    gp = g.params_array([g.params_like(p) for p in params])
    dev = [g.to_device(s, b) for s, b in zip(states, gb)]
    before = [d.clone() for d in dev]
    path = str(tmp_path / "tune.json")
    cfg, timings = autotune.tune(gb, dev, pidx, dts, gp, cache_path=path)
    assert len(timings) == len(autotune.CANDIDATES) and all(t > 0 for t in timings.values())
    for a, b in zip(dev, before):
        assert torch.equal(a, b)  # the tuner works on scratch copies
    cfg2, _ = autotune.tune(gb, dev, pidx, dts, gp, cache_path=path)
    assert (cfg2.variant, cfg2.tile_x, cfg2.tile_y, cfg2.tile_z) == (cfg.variant, cfg.tile_x, cfg.tile_y, cfg.tile_z)


def test_amr_like_and_sweep_generators_shapes():
    boxes = gi.amr_like_boxes()
    assert len(boxes) == 96
    pts = sum(b.npoints for b in boxes)
    assert 2e6 < pts < 2e7
    bx, ps = gi.coupling_sweep_boxes()
    assert len(bx) == 32 and all(b.nx == 64 for b in bx)
    assert all(0 <= p.lam <= 0.1 and 0 <= p.g2 <= 0.05 for p in ps)


@pytest.mark.parametrize("n,tile", [(8, (32, 4, 1)), (16, (32, 4, 1)), (12, (16, 4, 2))])
def test_persistent_launch_small_box_many_steps_equals_single_box_path(g, n, tile):
    """One small periodic box (its whole working set fits in the SMs' L1) advanced 20 steps in one
    persistent launch: every stage reads states that other blocks wrote before the previous grid
    barrier, so stale non-coherent cache lines would show as differing bits. The result must equal
    grf_rk4_step's, bit for bit."""
    import torch
    box = gi.cube_box(n, -1.5, 1.5)
    params = gi.Params(lam=0.2, g2=0.1, beta_kind=1)
    s0 = gi.random_perturbed_state(box, 7, base=gi.single_puncture(box, amp=0.05), eps=2e-2)
    b = g.box_like(box)
    p = g.params_like(params)
    dt = 0.25 * box.dx
    nsteps = 20
    ref = g.to_device(s0, b)
    g.grf_rk4_step(b, p, ref, dt, nsteps)
    gp = g.params_array([p])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dev = [g.to_device(s0, b)]
        items = g.batch_items([b], dev, [0], [dt])
        g.grf_batched_rk4(items, gp, nsteps, g.batch_config(g.GRF_BATCH_PERSISTENT, tile), stream=stream)
    stream.synchronize()
    assert np.array_equal(g.to_host(dev[0], b), g.to_host(ref, b))
