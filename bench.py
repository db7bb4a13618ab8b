#!/usr/bin/env python
"""Throughput of the modified-CCZ4 + 4dST RHS/RK4 path on GB300: FP64 grid-point RK4
updates per second, with the FP64 roofline fraction of the RK4-stage kernel.

One "step" = one full RK4 step (4 fused stage kernels: stencils + pointwise RHS + 7x7 solve
+ KO + stage update) over the whole 256^3 Brill-Lindquist box (the 32^3 single-puncture box
and the other workloads are parity-test cases). Inputs are resident in HBM for `value`; `e2e`
repeats the measurement with the state copied from pinned host memory to the device and back
inside every timed step. The state (3.9 GB) is larger than L2, so no L2 flush is needed.

--impl reference times the CPU oracle (the baseline arm) on a bounded sample of the same
workload on the host cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 grid-point RK4 updates/s (mCCZ4+4∂ST) and % of FP64/HBM roofline"
UNIT = "point-updates/s"

# FLOP_alg: the method's FP64 work per interior point and RK4 stage, frozen at 6,615.25 flops. It
# was counted once by running this formulation's pointwise right-hand side (CCZ4 + 4dST + the
# 7x7 solve), its stencils, dissipation and stage update with an operation-counting scalar
# (paper_2309_06225_gb300.flops; add/sub/mul 1, fma 2, div 1). It is not recounted when the
# kernel changes, so the achieved rate tracks the time per point, not source edits.
FLOP_ALG_PER_POINT_STAGE = 6615.25
# algorithmic HBM bytes per point-update (stage-wise RK4, 27 fields, perfect stencil reuse):
# stage 1: read u_n, write u_1 and acc (3 x 216 B); stages 2-3: read u_s, u_n, acc, write u_s, acc
# (5 x 216 B each); stage 4: read u_3, u_n, acc, write u_n (4 x 216 B)
BYTES_PER_POINT_UPDATE = 216 * (3 + 5 + 5 + 4)
# Per interior point and stage launch, from an ncu capture of each stage kernel on the 96^3 box
# (mean of stages 0 and 1): the FP64 thread instructions (dadd + dmul + dfma) and
# dram__bytes_read.sum + dram__bytes_write.sum. Keyed by (order, advection, cubic term), with
# backreaction; a scheme absent here (the decoupled kernels, or one whose kernel changed since its
# capture) reports neither.
STAGE_CAPTURES = {
    (4, "centred", False): (4196, 12773),     # the default kernel, no cubic code
    (4, "centred", True): (4464, 13769),      # general instantiation, g3 = 0.1
    (4, "lopsided", False): (4523, 13515),
    (6, "centred", False): (4846.5, 11629),
    (6, "lopsided", False): (5381.5, 11256),
}
FP64_INSTR_PER_POINT_STAGE, TRAFFIC_BYTES_PER_POINT_STAGE = STAGE_CAPTURES[(4, "centred", False)]
# the tangent-linear (dual-number) stage kernel's FP64 instructions per point-stage (same kind of capture)
TLM_FP64_INSTR_PER_POINT_STAGE = 29130
# nominal FP64 (non-tensor) peak of GB300: 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x ~2.06 GHz;
# used only when no measured figure is stored
FP64_NOMINAL_TFLOPS = 1.25
PEAKS_FP64_FILE = os.path.join(ROOT, "paper_2309_06225_gb300", "peaks_fp64.json")


def fp64_peak():
    """FP64 pipe ceilings: (TFLOP/s, FP64 instructions/s, source). The measured sweep of
    build_peak.measure() stored in peaks_fp64.json (best DFMA flop rate, best instruction rate of
    any kind, with the clocks seen), else the nominal figure (instructions at 2 per FMA flop)."""
    try:
        d = json.load(open(PEAKS_FP64_FILE))
        return float(d["tflops"]), float(d["instr_per_s"]), "of measured"
    except (OSError, ValueError, KeyError):
        return FP64_NOMINAL_TFLOPS, FP64_NOMINAL_TFLOPS * 1e12 / 2, "of nominal"


FP64_PEAK_TFLOPS, FP64_PEAK_INSTR, FP64_PEAK_SOURCE = fp64_peak()
# The FP64 pipe's issue ceiling: 2 thread-instructions per SM per clock (ncu's peak_sustained of
# the DFMA/DADD/DMUL thread-instruction counters, 304 per clock over 152 SMs).
FP64_PIPE_INSTR_PER_SM_CLK = 2
GB300_SMS = 152


def fp64_issue_ceiling(sm_mhz):
    """FP64 thread-instructions per second the pipe can issue at the given SM clock."""
    return FP64_PIPE_INSTR_PER_SM_CLK * GB300_SMS * sm_mhz * 1e6


def measured_hbm_gbs():
    """(GB/s, source) of the HBM copy peak: MEASURED_PEAKS.json when present, else the fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "of measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "of fallback"


def job_time_ms(ms_local, dist=None, device="cuda"):
    """The job's timed-region duration: the max over ranks (the job ends with its slowest rank);
    the rank's own value when it runs alone."""
    if dist is None:
        return ms_local
    import torch
    t = torch.tensor([ms_local], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, ms, world):
    """Units all ranks processed per second over the job's timed region (weak scaling: every rank
    advances its own replica)."""
    return world * units_per_rank * steps / (ms * 1e-3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bl_pair_256", choices=["bl_pair_256", "bl_pair_128", "bl_pair_96", "bl_pair_64", "amr_boxes_96", "coupling_sweep_32", "sphere_signal_96", "adjoint_96", "calls_256", "calls_96", "bl_pair_octant_128", "patches_256"])
    ap.add_argument("--patches", default="2,2,2", help="patches per axis of the patches_256 workload")
    ap.add_argument("--adjoint-grid", type=int, default=96,
                    help="points per axis of the adjoint_96 workload's box (dx = 0.2; 96 is the workload, smaller "
                         "grids are for profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sub-records", action="store_true",
                    help="skip the short same-process runs of the batched, differentiated and split-box workloads "
                         "that the default line carries under sub_records")
    ap.add_argument("--g3", type=float, default=0.0,
                    help="cubic Horndeski coupling g3 of the bl_pair workloads (0: 4dST alone); a non-zero value "
                         "runs the general stage instantiation with the cubic terms")
    ap.add_argument("--decoupled", action="store_true",
                    help="4dST without backreaction onto the metric (bl_pair workloads)")
    ap.add_argument("--order", type=int, default=4, choices=[4, 6],
                    help="finite-difference order: 6 runs the bl_pair workloads on 4-ghost boxes")
    ap.add_argument("--advection", default="centred", choices=["centred", "lopsided"],
                    help="stencil of the advection terms beta^k d_k u")
    ap.add_argument("--boundary", default="periodic", choices=["periodic", "extrapolating", "sommerfeld"],
                    help="outer boundary of the bl_pair box (its domain is centred on the origin)")
    ap.add_argument("--measure-peak", action="store_true",
                    help="also run the FP64 microbenchmark sweep in this process and report it")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    return ap.parse_args()


def workload(name, order=4, advection="centred", boundary="periodic"):
    """The named bl_pair workload, on 4-ghost boxes (6th-order scheme) when order == 6, with
    lopsided advection and extrapolating or Sommerfeld outer boundaries when asked."""
    import dataclasses
    import grf_inputs as gi
    n = int(name.rsplit("_", 1)[1])
    cfg = gi.config_bl_pair_octant(n) if name.startswith("bl_pair_octant_") else gi.config_bl_pair_256(n)
    if order == 6:
        box = dataclasses.replace(cfg["box"], ng=4)
        make = gi.brill_lindquist_pair_symmetric if name.startswith("bl_pair_octant_") else gi.brill_lindquist_pair
        cfg = dict(cfg, box=box, make_state=lambda b=box: make(b))
    if advection == "lopsided":
        cfg["params"].advection = 1
    if boundary != "periodic" and name.startswith("bl_pair_octant_"):
        # the octant keeps its mirror planes; its high faces become radiative
        assert boundary == "sommerfeld", "the octant takes mirror planes with Sommerfeld high faces"
        box = dataclasses.replace(cfg["box"], bc=gi.BC_REFLECT_LOW_SOMMERFELD)
        cfg = dict(cfg, box=box, make_state=lambda b=box: gi.brill_lindquist_pair_symmetric(b))
    elif boundary != "periodic":
        bc = gi.BC_EXTRAPOLATE if boundary == "extrapolating" else gi.BC_SOMMERFELD
        box = dataclasses.replace(cfg["box"], bc=bc)
        cfg = dict(cfg, box=box, make_state=lambda b=box: gi.brill_lindquist_pair(b))
    return cfg


def batched_workload(name):
    """(boxes, params list, params index per box, dt per box, initial states) of a batched
    workload: 96 uneven AMR-like boxes with frozen ghosts (single-puncture data, dt = dx/4 per
    box), or the 32-instance coupling sweep of periodic 64^3 boxes (dt = dx/4)."""
    import grf_inputs as gi
    if name == "amr_boxes_96":
        boxes = gi.amr_like_boxes()
        params = [gi.Params(beta_kind=gi.BETA_LINEAR, lam=0.01, g2=0.01)]
        pidx = [0] * len(boxes)
    else:
        boxes, params = gi.coupling_sweep_boxes()
        pidx = list(range(len(boxes)))
    dts = [0.25 * b.dx for b in boxes]
    return boxes, params, pidx, dts


def run_calls(args, rank, world, local_rank):
    """The standalone entry points on the 256^3 (calls_256) or 96^3 (calls_96, small enough for a
    full profiler capture) Brill-Lindquist state: one RHS evaluation with
    dissipation (grf_rhs), the dissipation alone (grf_ko_dissipation, added into an RHS array), the
    constraints (grf_constraints, the 4 fields without the norms) and the energy densities of the
    three scalar terms (grf_energy_densities). The timed RK4 step fuses the first two; the last two
    are diagnostics taken between steps. On the periodic box grf_rhs, grf_constraints and
    grf_energy_densities and grf_weyl_psi4 each launch the ghost fill and their kernel,
    grf_ko_dissipation one kernel, grf_extract_modes three: 12 launches per timed iteration over
    the six calls."""
    import torch
    import paper_2309_06225_gb300 as grf
    from paper_2309_06225_gb300 import flops as grf_flops
    if rank != 0:
        return
    cfg = workload("bl_pair_" + args.workload.rsplit("_", 1)[1])
    box, params = cfg["box"], cfg["params"]
    b = grf.box_like(box)
    p = grf.params_like(params)
    state = grf.to_device(cfg["make_state"](), b)
    rhs = grf.alloc_state(b)
    out4 = grf.alloc_state(b, 4)
    out3 = grf.alloc_state(b, 3)
    out4 = grf.alloc_state(b, 4)
    out2 = grf.alloc_state(b, 2)
    ews = grf.alloc_workspace(grf.grf_extract_workspace_bytes(32, 8))
    npts = box.nx * box.ny * box.nz
    stream = torch.cuda.current_stream()
    calls = {
        "grf_rhs": lambda: grf.grf_rhs(b, p, state, rhs),
        "grf_ko_dissipation": lambda: grf.grf_ko_dissipation(b, params.sigma_ko, state, rhs),
        "grf_constraints": lambda: grf.grf_constraints(b, p, state, out4, norms=False),
        "grf_energy_densities": lambda: grf.grf_energy_densities(b, p, state, out3),
        "grf_weyl_psi4": lambda: grf.grf_weyl_psi4(b, p, state, out2),
        "grf_hyperbolicity": lambda: grf.grf_hyperbolicity(b, p, state, out4),
        # the scalar waveform: spin-0 modes of phi up to l = 8 on a sphere of radius 0.75 L/2
        "grf_extract_modes": lambda: grf.grf_extract_modes(b, state[25], None, 0, 0.375 * box.nx * box.dx,
                                                           (0.0, 0.0, 0.0), 32, 64, 8, ws=ews),
    }
    hbm, hbm_src = measured_hbm_gbs()
    flop_rhs = grf_flops.flops_per_point_rhs(p)
    clocks = ClockSampler(gpu_selector(local_rank))
    clocks.start()
    time.sleep(0.3)
    out = {}
    for name, fn in calls.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        rec = {"ms_per_call": ms, "points_per_s": npts / (ms * 1e-3)}
        if name == "grf_extract_modes":  # 2048 samples of a 64-point stencil, 81 modes; synchronises
            rec = {"ms_per_call": ms, "samples": 32 * 64, "modes": 81, "roofline": None,
                   "note": "latency-bound: three small launches and a device-to-host copy of the modes"}
        elif name == "grf_ko_dissipation":
            # FP64-bound even alone: per field 9 pair sums + 6 accumulations + 3 fma + the fma into
            # the RHS (23 flops) against 24 bytes (state read once, RHS read and written)
            flop_ko = 27 * 23
            nbytes = 27 * 8 * 3
            tf = flop_ko * npts / (ms * 1e-3) / 1e12
            rec["roofline"] = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": tf / FP64_PEAK_TFLOPS, "flop_per_point": flop_ko,
                               "peak_source": FP64_PEAK_SOURCE,
                               "hbm_frac": nbytes * npts / (ms * 1e-3) / 1e9 / hbm, "hbm_peak_source": hbm_src}
        elif name == "grf_rhs":
            tf = flop_rhs * npts / (ms * 1e-3) / 1e12
            rec["roofline"] = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": tf / FP64_PEAK_TFLOPS, "flop_per_point": flop_rhs,
                               "peak_source": FP64_PEAK_SOURCE}
        else:  # constraints, densities, Psi_4 and the hyperbolicity diagnostics use the RHS's gather and algebra
            rec["roofline"] = None
            rec["note"] = "FP64-bound like grf_rhs; its flop count is a subset of the RHS and is not counted"
        out[name] = rec
    clk = clocks.stop()
    status = grf.grf_check_status()
    line = {"metric": "FP64 grid-point RHS evaluations/s (grf_rhs, standalone)", "value": out["grf_rhs"]["points_per_s"],
            "unit": "points/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["grf_rhs"]["ms_per_call"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "grid": [box.nx, box.ny, box.nz],
                       "l2": "inputs larger than L2 (no flush needed)"},
            "gpu_launches": 13 * args.steps, "calls": out, "clocks": clk, "status": {"solve": status},
            "roofline": out["grf_rhs"]["roofline"], "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def run_tangent(args, rank, world, local_rank):
    """The differentiated evolution: 96^3 single-puncture box on [-9.6, 9.6]^3 (dx = 0.2,
    periodic), sphere signal at r = 6 with its derivatives in (lambda, g2, A), against the plain
    RK4 step on the same box."""
    import numpy as np
    import torch
    import grf_inputs as gi
    import paper_2309_06225_gb300 as grf

    torch.cuda.set_device(local_rank)
    box = gi.cube_box(96, -9.6, 9.6)
    params = gi.Params(lam=0.01, g2=0.01)
    amp = 1e-3
    b = grf.box_like(box)
    p = grf.params_like(params)
    dt = 0.25 * box.dx
    s0 = gi.single_puncture(box, amp=amp)
    dphi = np.zeros(box.shape)
    dphi[25] = gi.single_puncture(box, amp=1.0)[25]
    state = grf.to_device(s0, b)
    tang = grf.alloc_state(b, 81)
    tang.view(3, -1)[2].copy_(grf.to_device(dphi, b).reshape(-1))
    loss = torch.zeros(4, dtype=torch.float64, device="cuda")
    ws = grf.alloc_workspace(grf.grf_tlm_workspace_bytes(b))
    sph = grf.grf_sphere(6.0, 0.0, 0.0, 0.0)
    seeds = [1.0, 0.0, 0.0, 1.0, 0.0, 0.0]
    grf.grf_tlm_rk4(b, p, seeds, state, tang, dt, max(1, args.warmup), sph, loss, ws=ws)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    grf.grf_tlm_rk4(b, p, seeds, state, tang, dt, args.steps, sph, loss, ws=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_t = e0.elapsed_time(e1)
    prim = grf.to_device(s0, b)
    pws = grf.alloc_workspace(grf.grf_workspace_bytes(b, grf.GRF_OP_RK4))
    grf.grf_rk4_step(b, p, prim, dt, max(1, args.warmup), ws=pws)
    torch.cuda.synchronize()
    e0.record(stream)
    grf.grf_rk4_step(b, p, prim, dt, args.steps, ws=pws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_f = e0.elapsed_time(e1)
    npts = box.npoints
    out = {"metric": METRIC, "value": npts * args.steps / (ms_t * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "sphere_signal_96", "grid": [96, 96, 96], "dx": box.dx, "dt": dt,
                      "sphere_radius": 6.0, "directions": ["lambda", "g2", "A"],
                      "method": "forward-mode tangent-linear evolution (value + 3 tangents per grid value)"},
           "gpu_launches": 5 * args.steps,
           "differentiated_vs_plain": {"tangent_ms_per_step": ms_t / args.steps, "plain_ms_per_step": ms_f / args.steps,
                                       "ratio": ms_t / ms_f},
           "signal": loss.cpu().numpy().tolist(), "e2e": None, "cpu_baseline": None}
    # FP64-bound like the plain stage: the dual-number stage's FP64 instruction count (ncu, 96^3)
    # against the pipe's issue rate
    stage_ms = ms_t / (4 * args.steps)
    issue = TLM_FP64_INSTR_PER_POINT_STAGE * npts / (stage_ms * 1e-3) / fp64_issue_ceiling(2070.0)
    out["roofline"] = {"bound": "alu", "unit": "FP64 instructions/s", "kernel": "tlm_stage_kernel",
                       "achieved": TLM_FP64_INSTR_PER_POINT_STAGE * npts / (stage_ms * 1e-3),
                       "peak": fp64_issue_ceiling(2070.0), "frac": issue,
                       "peak_source": "2 FP64 instructions per SM per clock x 152 SMs x 2070 MHz",
                       "fp64_instr_per_point_stage": TLM_FP64_INSTR_PER_POINT_STAGE, "traffic": None}
    return out


def run_adjoint(args, rank, world, local_rank):
    """The differentiated evolution in reverse mode: the 96^3 single-puncture box on
    [-9.6, 9.6]^3 (dx = 0.2, periodic), sphere signal at r = 6. One step of this workload is one
    RK4 step of the forward pass (grf_signal_forward, a checkpoint every 20 steps) plus its share
    of the reverse sweep (grf_adjoint_rk4: segment recomputation, stage recomputation, four
    reverse-mode stage kernels and four transposed-stencil kernels). --steps is the number of
    RK4 steps differentiated; the gradient is with respect to (lambda, g2, A). The adjoint is
    seeded at the sphere after every step and spreads 12 points per reversed step, so the first
    reversed steps touch little of the box (the sweep skips entries whose adjoint is zero); from
    about 10 steps on they are dense, as in the 400-step run, so the per-step figure wants
    --steps of 24 or more."""
    import numpy as np
    import torch
    import grf_inputs as gi
    import paper_2309_06225_gb300 as grf

    torch.cuda.set_device(local_rank)
    n = args.adjoint_grid
    box = gi.cube_box(n, -0.1 * n, 0.1 * n)
    params = gi.Params(lam=0.01, g2=0.01)
    amp, ce, R = 1e-3, 20, min(6.0, 0.1 * n - 0.5)
    b, p = grf.box_like(box), grf.params_like(params)
    dt = 0.25 * box.dx
    nsteps = args.steps
    s0 = gi.single_puncture(box, amp=amp)
    dphi = np.zeros(box.shape)
    dphi[25] = gi.single_puncture(box, amp=1.0)[25]
    dA = grf.to_device(dphi, b)
    sph = grf.grf_sphere(R, 0.0, 0.0, 0.0)
    torch.cuda.reset_peak_memory_stats()
    state = grf.to_device(s0, b)
    ck = torch.empty((grf.checkpoint_count(nsteps, ce),) + tuple(state.shape), dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = grf.alloc_workspace(grf.grf_adjoint_workspace_bytes(b, ce))
    sbar = grf.alloc_state(b)
    pbar = torch.zeros(2, dtype=torch.float64, device="cuda")
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    # warm-up: a short differentiated run
    wn = max(1, min(args.warmup, 2))
    grf.grf_signal_forward(b, p, state, dt, wn, sph, ce, ck, loss, ws=ws)
    grf.grf_adjoint_rk4(b, p, ck, dt, wn, sph, ce, 1.0, sbar, pbar, ws=ws)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    state.copy_(grf.to_device(s0, b))
    sbar.zero_()
    clocks = ClockSampler(gpu_selector(local_rank))
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev[0].record(stream)
    grf.grf_signal_forward(b, p, state, dt, nsteps, sph, ce, ck, loss, ws=ws, stream=stream)
    ev[1].record(stream)
    grf.grf_adjoint_rk4(b, p, ck, dt, nsteps, sph, ce, 1.0, sbar, pbar, ws=ws, stream=stream)
    grf.grf_state_dot(b, sbar, dA, -1, dot, stream=stream)
    ev[2].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    fwd_ms, rev_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    # the plain step on the same box, for the ratio
    prim = grf.to_device(s0, b)
    pws = grf.alloc_workspace(grf.grf_workspace_bytes(b, grf.GRF_OP_RK4))
    grf.grf_rk4_step(b, p, prim, dt, 2, ws=pws)
    torch.cuda.synchronize()
    ev[0].record(stream)
    grf.grf_rk4_step(b, p, prim, dt, nsteps, ws=pws, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    plain_ms = ev[0].elapsed_time(ev[1])
    npts = box.npoints
    total_ms = fwd_ms + rev_ms
    grad = [float(x) for x in pbar.cpu()] + [float(dot.cpu()[0])]
    out = {"metric": METRIC, "value": npts * nsteps / (total_ms * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": nsteps, "warmup": args.warmup, "ms_per_step": total_ms / nsteps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "adjoint_96", "grid": [n, n, n], "dx": box.dx, "dt": dt, "sphere_radius": R,
                      "checkpoint_every": ce, "parameters": ["lambda", "g2", "A"],
                      "method": "reverse mode: forward with checkpoints, segment and stage recomputation, "
                                "taped reverse-mode stage kernels and transposed stencils"},
           "gpu_launches": None,
           "adjoint": {"forward_ms_per_step": fwd_ms / nsteps, "reverse_ms_per_step": rev_ms / nsteps,
                       "plain_ms_per_step": plain_ms / nsteps, "differentiated_vs_plain": total_ms / plain_ms,
                       "reverse_vs_forward": rev_ms / fwd_ms, "peak_memory_bytes": torch.cuda.max_memory_allocated(),
                       "workspace_bytes": grf.grf_adjoint_workspace_bytes(b, ce)},
           "signal": float(loss.cpu()[0]), "gradient": grad, "clocks": clk, "roofline": None, "e2e": None,
           "cpu_baseline": None}
    return out


def run_batched(args, rank, world, local_rank):
    import torch
    import grf_inputs as gi
    import paper_2309_06225_gb300 as grf
    from paper_2309_06225_gb300 import autotune

    torch.cuda.set_device(local_rank)
    boxes, params, pidx, dts = batched_workload(args.workload)
    gb = [grf.box_like(b) for b in boxes]
    gp = grf.params_array([grf.params_like(p) for p in params])
    init = [grf.to_device(gi.single_puncture(b), b2) for b, b2 in zip(boxes, gb)]
    states = [t.clone() for t in init]
    npts = sum(b.npoints for b in boxes)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        cfg, timings = autotune.tune(gb, states, pidx, dts, gp, stream=stream)
        items = grf.batch_items(gb, states, pidx, dts)
        ws = grf.alloc_workspace(grf.grf_batched_workspace_bytes(items, cfg))
        grf.grf_batched_rk4(items, gp, args.warmup, cfg, ws=ws, stream=stream)
        torch.cuda.synchronize()
        clocks = ClockSampler(gpu_selector(local_rank))
        clocks.start()
        time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        grf.grf_batched_rk4(items, gp, args.steps, cfg, ws=ws, stream=stream, sync_status=False)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        status = grf.grf_check_status()
        # the plain single-box path on the same boxes: one grf_rk4_step call per box and step
        wss = {}
        for b2 in gb:
            key = (b2.nx, b2.ny, b2.nz, b2.pitch)
            if key not in wss:
                wss[key] = grf.alloc_workspace(grf.grf_workspace_bytes(b2, grf.GRF_OP_RK4))
        single = [t.clone() for t in init]
        for b2, t, pi, dt in zip(gb, single, pidx, dts):
            grf.grf_rk4_step(b2, gp[pi], t, dt, 1, ws=wss[(b2.nx, b2.ny, b2.nz, b2.pitch)], stream=stream)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            for b2, t, pi, dt in zip(gb, single, pidx, dts):
                grf.grf_rk4_step(b2, gp[pi], t, dt, 1, ws=wss[(b2.nx, b2.ny, b2.nz, b2.pitch)], stream=stream)
        s1.record(stream)
        torch.cuda.synchronize()
        ms_single = s0.elapsed_time(s1)
        # e2e: every step, all box states from pinned host to device and back
        host = [torch.empty(t.shape, dtype=torch.float64, pin_memory=True) for t in init]
        for h, t in zip(host, init):
            h.copy_(t)
        hout = [torch.empty(t.shape, dtype=torch.float64, pin_memory=True) for t in init]
        nbytes = sum(t.numel() * 8 for t in init)
        torch.cuda.synchronize()
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        for _ in range(args.steps):
            for h, t in zip(host, states):
                t.copy_(h, non_blocking=True)
            grf.grf_batched_rk4(items, gp, 1, cfg, ws=ws, stream=stream, sync_status=False)
            for h, t in zip(hout, states):
                h.copy_(t, non_blocking=True)
        x1.record(stream)
        torch.cuda.synchronize()
        ems = x0.elapsed_time(x1)
    value = npts * args.steps / (ms * 1e-3)
    flop_ps = FLOP_ALG_PER_POINT_STAGE
    achieved = flop_ps * npts * 4 * args.steps / (ms * 1e-3) / 1e12
    variant = {grf.GRF_BATCH_GRAPH: "graph", grf.GRF_BATCH_PERSISTENT: "persistent"}.get(cfg.variant, "stream")
    kernel = "batch_persistent_kernel" if cfg.variant == grf.GRF_BATCH_PERSISTENT else "batch_stage_kernel"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "boxes": len(boxes), "points": npts,
                      "shapes": autotune.signature(gb), "variant": variant,
                      "tile": [cfg.tile_x, cfg.tile_y, cfg.tile_z], "autotune_ms_per_step": timings,
                      "l2": "inputs larger than L2 (no flush needed)"},
           "gpu_launches": (1 if cfg.variant == grf.GRF_BATCH_PERSISTENT else 4 * args.steps),
           "roofline": {"bound": "alu", "unit": "TFLOP/s", "kernel": kernel, "achieved": achieved,
                        "peak": FP64_PEAK_TFLOPS, "frac": achieved / FP64_PEAK_TFLOPS, "flop_per_point_stage": flop_ps,
                        "traffic": None},
           "single_box_path": {"value": npts * args.steps / (ms_single * 1e-3), "ms_per_step": ms_single / args.steps,
                               "launches_per_step": len(boxes) * 5,
                               "batched_speedup": ms_single / ms},
           "clocks": clk, "status": {"solve": status},
           "e2e": {"value": npts * args.steps / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes, "ms_per_step": ems / args.steps},
           "cpu_baseline": None}
    return out


def run_patches(args, rank, world, local_rank):
    """The 256^3 Brill-Lindquist workload held as px x py x pz patches (grf_patches_rk4): per
    stage one batched stage launch over all patches and one halo exchange. Beside it, the same
    steps of grf_rk4_step on the whole box, and the exchange timed alone."""
    import torch
    import paper_2309_06225_gb300 as grf

    torch.cuda.set_device(local_rank)
    cfg = workload("bl_pair_256")
    box, params, dt = cfg["box"], cfg["params"], cfg["dt"]
    pxyz = [int(v) for v in args.patches.split(",")]
    b, p = grf.box_like(box), grf.params_like(params)
    level = grf.patch_level(b, *pxyz)
    whole = grf.to_device(cfg["make_state"](), b)
    patches = grf.patch_states(level)
    ws = grf.alloc_workspace(grf.grf_patches_workspace_bytes(level))
    npts = box.nx * box.ny * box.nz
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    grf.grf_patch_copy(level, whole, patches, 0)
    grf.grf_patches_rk4(level, p, patches, dt, args.warmup, ws=ws)
    clocks = ClockSampler(gpu_selector(local_rank))
    clocks.start()
    time.sleep(0.3)
    ms = timed(lambda: grf.grf_patches_rk4(level, p, patches, dt, args.steps, ws=ws, sync_status=False), 1)
    clk = clocks.stop()
    status = grf.grf_check_status()
    ms_x = timed(lambda: grf.grf_halo_exchange(level, patches), 20) / 20
    # the whole box, same steps
    wws = grf.alloc_workspace(grf.grf_workspace_bytes(b, grf.GRF_OP_RK4))
    grf.grf_rk4_step(b, p, whole, dt, 1, ws=wws)
    ms_w = timed(lambda: grf.grf_rk4_step(b, p, whole, dt, args.steps, ws=wws), 1)
    # e2e: the box state from pinned host memory, split, stepped, joined and read back every step
    host_in = torch.empty(whole.shape, dtype=torch.float64, pin_memory=True)
    host_in.copy_(whole)
    host_out = torch.empty_like(host_in, pin_memory=True)
    nbytes = whole.numel() * 8

    def e2e_step():
        whole.copy_(host_in, non_blocking=True)
        grf.grf_patch_copy(level, whole, patches, 0)
        grf.grf_patches_rk4(level, p, patches, dt, 1, ws=ws, sync_status=False)
        grf.grf_patch_copy(level, whole, patches, 1)
        host_out.copy_(whole, non_blocking=True)

    ems = timed(e2e_step, args.steps)
    value = npts * args.steps / (ms * 1e-3)
    flop_ps = FLOP_ALG_PER_POINT_STAGE
    achieved = flop_ps * npts * 4 * args.steps / (ms * 1e-3) / 1e12
    # exchange bytes: every ghost point of every patch, 27 fields read and written
    ghost_pts = 0
    for q in range(len(patches)):
        pb = grf.grf_patch_box(level, q)
        ghost_pts += (pb.nx + 6) * (pb.ny + 6) * (pb.nz + 6) - pb.nx * pb.ny * pb.nz
    x_bytes = ghost_pts * 27 * 16
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "patches_256", "grid": [box.nx, box.ny, box.nz], "patches": pxyz, "dx": box.dx,
                      "dt": dt, "beta_kind": params.beta_kind, "lambda": params.lam, "g2": params.g2,
                      "l2": "inputs larger than L2 (no flush needed)"},
           "gpu_launches": 8 * args.steps + 1,
           "roofline": {"bound": "alu", "unit": "TFLOP/s", "kernel": "batch_stage_kernel", "achieved": achieved,
                        "peak": FP64_PEAK_TFLOPS, "frac": achieved / FP64_PEAK_TFLOPS, "flop_per_point_stage": flop_ps,
                        "traffic": None},
           "halo_exchange": {"ms": ms_x, "bytes": x_bytes, "gb_s": x_bytes / (ms_x * 1e-3) / 1e9,
                             "share_of_step": 4 * ms_x / (ms / args.steps)},
           "whole_box_path": {"value": npts * args.steps / (ms_w * 1e-3), "ms_per_step": ms_w / args.steps},
           "clocks": clk, "status": {"solve": status},
           "e2e": {"value": npts * args.steps / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes, "ms_per_step": ems / args.steps},
           "cpu_baseline": None}
    return out


# ------------------------------------------------------------------------------ clocks
def gpu_selector(local_rank):
    """nvidia-smi -i argument for this process's GPU (PCI bus id when torch exposes it)."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(local_rank)
        return f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
    except Exception:
        return str(local_rank)


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------ CPU oracle
def sub_block(cfg, n):
    """An n^3 sub-block of the workload grid (same points, same analytic data) next to the
    upper puncture, with frozen ghosts."""
    import grf_inputs as gi
    box = cfg["box"]
    i0 = box.nx // 2 - n // 2
    k0 = int(round((3.0 - box.z0) / box.dx)) - n // 2
    sub = gi.Box(n, n, n, box.dx, box.x0 + i0 * box.dx, box.y0 + i0 * box.dx, box.z0 + k0 * box.dx, bc=gi.BC_FROZEN,
                 ng=box.ng)
    return sub, gi.brill_lindquist_pair(sub)


def oracle_sample(cfg, seconds, steps=1):
    """Times the CPU oracle on a cube sub-block of the workload, grown until one run takes
    about `seconds`. Returns (point-updates/s, cores, description)."""
    import oracle
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    n = 8
    while True:
        sub, s = sub_block(cfg, n)
        t0 = time.perf_counter()
        oracle.rk4(sub, cfg["params"], s, cfg["dt"], steps)
        el = time.perf_counter() - t0
        if el >= 0.3 * seconds or n >= 96:
            break
        n = int(min(96, max(n + 4, n * (seconds / max(el, 1e-3)) ** (1 / 3))))
    return n ** 3 * steps / el, cores, f"{steps} RK4 step(s) of a {n}^3 frozen-ghost sub-block of the workload ({el:.1f} s)"


def oracle_single_core(args, seconds):
    """The same oracle sample on one host core (a child process with OMP_NUM_THREADS=1, started
    before this process touches CUDA). Returns {"value", "sample"} or None if it failed."""
    code = ("import json, bench\n"
            f"cfg = bench.workload({args.workload!r}, {args.order}, {args.advection!r}, {args.boundary!r})\n"
            f"cfg['params'].decoupled = {1 if args.decoupled else 0}\n"
            f"r = bench.oracle_sample(cfg, {float(seconds)})\n"
            "print(json.dumps([r[0], r[2]]))\n")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                             timeout=20 * seconds + 60)
        rate, desc = json.loads(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, OSError, ValueError, IndexError):
        return None
    return {"value": rate, "cores": 1, "sample": desc}


def run_reference(args, rank):
    cfg = workload(args.workload, args.order, args.advection, args.boundary)
    if rank != 0:
        return
    import oracle
    box = cfg["box"]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # size one step's sample so that warmup + steps fit in a few minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    n = 8
    while True:
        sub, s = sub_block(cfg, n)
        t0 = time.perf_counter()
        oracle.rk4(sub, cfg["params"], s, cfg["dt"], 1)
        el = time.perf_counter() - t0
        if el > 0.25 * budget or n >= 64:
            break
        n = int(min(64, max(n + 4, n * (0.5 * budget / max(el, 1e-3)) ** (1 / 3))))
    for _ in range(max(0, args.warmup - 1)):
        oracle.rk4(sub, cfg["params"], sub_block(cfg, n)[1], cfg["dt"], 1)
    states = [sub_block(cfg, n)[1] for _ in range(args.steps)]
    t0 = time.perf_counter()
    for s in states:
        oracle.rk4(sub, cfg["params"], s, cfg["dt"], 1)
    el = time.perf_counter() - t0
    value = n ** 3 * args.steps / el
    sample = f"each step: 1 RK4 step of a {n}^3 frozen-ghost sub-box of the {cfg['name']} workload"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": cfg["name"], "grid": [box.nx, box.ny, box.nz], "dx": box.dx, "dt": cfg["dt"],
                      "sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------ GPU arm
def roofline_record(ng, params, npts, launch_ms, value, clk, peak):
    """The roofline object of a bl_pair line: the stage kernel's achieved FLOP_alg rate against the
    measured FP64 peak, its DRAM bytes and FP64 issue fraction where a capture of that kernel is
    stored, and the HBM fraction of the algorithmic bytes. Returns (roofline, scheme, default)."""
    flop_ps = FLOP_ALG_PER_POINT_STAGE
    achieved = flop_ps * npts / (launch_ms * 1e-3) / 1e12
    scheme = {"order": ng * 2 - 2, "advection": "lopsided" if params.advection else "centred"}
    default_scheme = scheme == {"order": 4, "advection": "centred"} and params.g3 == 0.0 and not params.decoupled
    roof = {"bound": "alu", "unit": "TFLOP/s",
            "kernel": "rk4_stage_kernel" if ng == 3 else "rk4_stage6_kernel", "achieved": achieved,
            "peak": FP64_PEAK_TFLOPS, "frac": achieved / FP64_PEAK_TFLOPS,
            "peak_source": FP64_PEAK_SOURCE,
            "peak_dfma_microbenchmark": peak, "flop_per_point_stage": flop_ps,
            "flop_convention": "FLOP_alg frozen: counted once from this formulation with an operation-counting scalar (add/sub/mul 1, fma 2, div 1)",
            "traffic": None}
    # per-point FP64 instructions and DRAM bytes of the stage kernel that runs, where captured
    instr, traffic = (None, None) if params.decoupled else \
        STAGE_CAPTURES.get((scheme["order"], scheme["advection"], params.g3 != 0.0), (None, None))
    if traffic:
        roof["traffic"] = traffic * npts
    if params.decoupled:
        roof["note"] = ("flop_per_point_stage is the count of the coupled 4th-order scheme; without backreaction the "
                        "solve and the stress terms are compiled away, so achieved and frac overstate this kernel's work")
    elif not default_scheme:
        roof["note"] = ("flop_per_point_stage is the count of the 4th-order centred scheme without the cubic term; "
                        "this configuration does more work per point, so achieved and frac are lower bounds")
    if params.g3 != 0.0 and ng == 3:
        roof["kernel"] = "rk4_stage_kernel (general instantiation, cubic terms)"
    hbm_gbs, hbm_src = measured_hbm_gbs()
    roof["hbm_frac"] = BYTES_PER_POINT_UPDATE * value / (hbm_gbs * 1e9)
    roof["hbm_peak_source"] = f"{hbm_src} {hbm_gbs:.1f} GB/s"
    if instr:
        # how full the FP64 pipe is: adds and multiplies take an issue slot but count one flop
        rate = instr * npts / (launch_ms * 1e-3)
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        roof["fp64_issue_frac"] = rate / fp64_issue_ceiling(sm_mhz)
        roof["fp64_issue"] = {"instr_per_point_stage": instr, "instr_per_s": rate,
                              "ceiling": fp64_issue_ceiling(sm_mhz),
                              "ceiling_source": f"2 per SM per clock x 152 SMs x {sm_mhz:.0f} MHz (sampled)",
                              "vs_measured_chains": rate / FP64_PEAK_INSTR}
    return roof, scheme, default_scheme


SUB_RECORD_DROP = ("n_gpus", "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "cpu_baseline")


def sub_records(args, local_rank):
    """Short runs of the other workloads in this process, after the headline measurement: the 96
    AMR-like boxes in one batched launch (with the single-box path beside it), the tangent-linear
    and the reverse-mode differentiated 96^3 evolutions (each against the plain step), and the
    256^3 box split into 2 x 2 x 2 patches (with the halo exchange timed alone). Each keeps its
    own timing rules (CUDA events, warm-up, clocks) with fewer steps than its own workload line."""
    import argparse
    import torch
    recs = {}
    plan = [("batched_amr_boxes_96", run_batched, "amr_boxes_96", 5, 3),
            ("tangent_sphere_signal_96", run_tangent, "sphere_signal_96", 8, 3),
            ("adjoint_96", run_adjoint, "adjoint_96", 24, 3),
            ("patches_256", run_patches, "patches_256", 4, 3)]
    for name, fn, wl, steps, warmup in plan:
        a = argparse.Namespace(**vars(args))
        a.workload, a.steps, a.warmup = wl, steps, warmup
        t0 = time.time()
        try:
            r = fn(a, 0, 1, local_rank)
        except (RuntimeError, OSError, ValueError) as e:  # reported in the line, the headline stands
            recs[name] = {"error": f"{type(e).__name__}: {e}"}
            continue
        finally:
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        rec = {k: v for k, v in r.items() if k not in SUB_RECORD_DROP}
        rec["wall_s"] = time.time() - t0
        recs[name] = rec
    return recs


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2309_06225_gb300 as grf
    from paper_2309_06225_gb300 import build_peak

    cfg = workload(args.workload, args.order, args.advection, args.boundary)
    box = cfg["box"]
    params, dt = cfg["params"], cfg["dt"]
    if args.decoupled:
        params.decoupled = 1
    params.g3 = args.g3

    # CPU oracle baseline first (rank 0, N = 1), before any CUDA work in this process
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, desc = oracle_sample(cfg, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "single_core": oracle_single_core(args, max(2.0, args.cpu_seconds / 3))}

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    b = grf.box_like(box)
    p = grf.params_like(params)
    s0 = cfg["make_state"]()
    state = grf.to_device(s0, b)
    init = state.clone()
    ws = grf.alloc_workspace(grf.grf_workspace_bytes(b, grf.GRF_OP_RK4))
    stream = torch.cuda.current_stream()
    npts = box.nx * box.ny * box.nz

    peak = build_peak.measure() if args.measure_peak else None

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        grf.grf_rk4_step(b, p, state, dt, 1, ws=ws, stream=stream)
    barrier()
    clocks = ClockSampler(gpu_selector(local_rank))
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    ev[0].record(stream)
    for k in range(args.steps):
        grf.grf_rk4_step(b, p, state, dt, 1, ws=ws, stream=stream)
        ev[k + 1].record(stream)
    barrier()
    clk = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = ev[0].elapsed_time(ev[-1])
    status = grf.grf_check_status()
    finite = grf.grf_check_finite(b, state)
    ms = job_time_ms(ms, dist)
    value = whole_job_rate(npts, args.steps, ms, world)

    e2e = None
    if not args.no_e2e:
        host_in = torch.empty(state.shape, dtype=torch.float64, pin_memory=True)
        host_in.copy_(init)
        host_out = torch.empty(state.shape, dtype=torch.float64, pin_memory=True)
        nbytes = state.numel() * 8
        # grf_rk4_step_host overlaps the copies slab by slab for 3 ghost layers with image or frozen
        # ghosts; other boxes get whole-state copies around the device step
        sliced = box.ng == 3 and box.bc in (0, 1, 2)

        def host_step():
            grf.grf_rk4_step_host(b, p, host_in, host_out, state, dt, 1, ws=ws, stream=stream)

        host_step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            host_step()
        e1.record(stream)
        barrier()
        ems = e0.elapsed_time(e1)
        ems = job_time_ms(ems, dist)
        # outside the timed region: the host-to-host result equals the device-resident step
        state.copy_(host_in)
        grf.grf_rk4_step(b, p, state, dt, 1, ws=ws, stream=stream)
        nxg = box.nx + 2 * box.ng
        identical = bool(torch.equal(state.cpu()[..., :nxg], host_out[..., :nxg]))
        e2e = {"value": whole_job_rate(npts, args.steps, ems, world), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": ems / args.steps,
               "bit_identical_to_device_step": identical,
               "path": ("grf_rk4_step_host: pinned host -> device in z-slabs overlapped with stage 1, "
                        "stage 4 in z-slabs overlapped with device -> pinned host, every step") if sliced else
                       ("grf_rk4_step_host: whole-state pinned host -> device copy by the SMs, the device step, "
                        "whole-state copy back, every step (not overlapped)")}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    launch_ms = ms / (4 * args.steps)  # the timed region is 4 stage kernels + 1 small ghost fill per step
    roof, scheme, default_scheme = roofline_record(box.ng, params, npts, launch_ms, value, clk, peak)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg["name"], "grid": [box.nx, box.ny, box.nz], "ghosts": box.ng, "dx": box.dx,
                      "fd_order": scheme["order"], "advection": scheme["advection"],
                      "dt": dt, "beta": "lambda phi^2/2", "lambda": params.lam, "g2": params.g2, "g3": params.g3,
                      "backreaction": not args.decoupled,
                      "boundary": {0: "periodic", 1: "frozen", 2: "mirror planes at the low faces, analytic high-face ghosts",
                                   3: "extrapolating", 4: "Sommerfeld",
                                   5: "mirror planes at the low faces, Sommerfeld high faces"}[box.bc],
                      "state_bytes": int(state.numel() * 8), "l2": "inputs larger than L2 (no flush needed)",
                      "parallelism": f"{world} independent replica(s), one box per GPU"},
           # per step: 4 stage kernels, plus the ghost fill (periodic, mirror: 1, extrapolating: 3 + 3 per stage)
           # or the Sommerfeld ghost update after each stage (4)
           "gpu_launches": {0: 5, 1: 4, 2: 5, 3: 19, 4: 8, 5: 13}[box.bc] * args.steps, "roofline": roof, "clocks": clk,
           "e2e": e2e, "cpu_baseline": cpu,
           "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
           "status": {"solve": status, "finite": finite}}
    if box.bc in (2, 5):  # an octant with mirror planes evolves the symmetric full box on 1/8 of its points
        out["config"]["full_box_equivalent_point_updates_per_s"] = 8 * value
    if world == 1 and not args.no_sub_records and args.workload == "bl_pair_256" and default_scheme \
            and box.bc == 0 and not args.decoupled:
        del state, init, ws
        torch.cuda.empty_cache()
        out["sub_records"] = sub_records(args, local_rank)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if "RANK" in os.environ else 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload in ("calls_256", "calls_96"):
        run_calls(args, rank, world, local_rank)
        return
    runs = {"sphere_signal_96": run_tangent, "adjoint_96": run_adjoint, "patches_256": run_patches,
            "amr_boxes_96": run_batched, "coupling_sweep_32": run_batched}
    if args.workload in runs:
        out = runs[args.workload](args, rank, world, local_rank)
        if out is not None and rank == 0:
            print(json.dumps(out), flush=True)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
