"""Autotuner for the batched RK4 launch (grf_batched_rk4).

For a batch signature (the multiset of box shapes and boundary types, together with the
kernel variants the boxes' parameters select: coupling kind, backreaction and advection
stencil), each candidate configuration (launch variant x tile shape) is timed on scratch
copies of the states with CUDA events: one untimed step, then the median of REPEATS timed
steps. The fastest is returned and cached in a JSON file keyed by the signature and the GPU
name. The states passed in are not modified.
"""
from __future__ import annotations

import json
import os
import statistics

from . import (GRF_BATCH_GRAPH, GRF_BATCH_PERSISTENT, alloc_workspace, batch_config, batch_items,
               grf_batched_rk4, grf_batched_workspace_bytes)

CANDIDATES = [
    (GRF_BATCH_GRAPH, (32, 4, 1)),
    (GRF_BATCH_GRAPH, (64, 2, 1)),
    (GRF_BATCH_GRAPH, (32, 2, 2)),
    (GRF_BATCH_GRAPH, (16, 8, 1)),
    (GRF_BATCH_GRAPH, (16, 4, 2)),
    (GRF_BATCH_PERSISTENT, (32, 4, 1)),
    (GRF_BATCH_PERSISTENT, (64, 2, 1)),
]
REPEATS = 3


def default_cache_path():
    return os.environ.get("GRF_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "grf_batch_autotune.json"))


def signature(boxes, params=None, params_index=None):
    """Multiset of (shape, boundary, kernel variant) over the boxes. The kernel variant is the
    coupling kind, the backreaction switch and the advection stencil of the box's parameters
    (they select different stage instantiations with different costs)."""
    def variant(i):
        if params is None or params_index is None:
            return ""
        p = params[params_index[i]]
        return f"/b{int(p.beta_kind)}d{int(p.decoupled)}a{int(p.advection)}"
    shapes = sorted((b.nx, b.ny, b.nz, b.bc, variant(i)) for i, b in enumerate(boxes))
    counts = {}
    for s in shapes:
        counts[s] = counts.get(s, 0) + 1
    return ";".join(f"{k[0]}x{k[1]}x{k[2]}/{k[3]}{k[4]}:{v}" for k, v in sorted(counts.items()))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(boxes, states, params_index, dts, params, cache_path=None, use_cache=True, stream=None, verbose=False):
    """Returns (grf_batch_config, timings) for this batch: the fastest candidate, from the
    cache when the signature was tuned before on this GPU."""
    import torch
    path = cache_path or default_cache_path()
    key = f"{torch.cuda.get_device_name()}|{signature(boxes, params, params_index)}"
    cache = _load(path) if use_cache else {}
    if key in cache:
        c = cache[key]
        return batch_config(c["variant"], tuple(c["tile"])), c.get("timings", {})
    scratch = [s.clone() for s in states]
    stream = stream or torch.cuda.Stream()
    timings = {}
    best = None
    with torch.cuda.stream(stream):
        for variant, tile in CANDIDATES:
            cfg = batch_config(variant, tile)
            items = batch_items(boxes, scratch, params_index, dts)
            ws = alloc_workspace(grf_batched_workspace_bytes(items, cfg))
            grf_batched_rk4(items, params, 1, cfg, ws=ws, stream=stream)
            times = []
            for _ in range(REPEATS):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                grf_batched_rk4(items, params, 1, cfg, ws=ws, stream=stream, sync_status=False)
                e1.record(stream)
                stream.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            name = f"{'graph' if variant == GRF_BATCH_GRAPH else 'persistent'}:{tile[0]}x{tile[1]}x{tile[2]}"
            timings[name] = ms
            if verbose:
                print(f"autotune {name}: {ms:.3f} ms/step", flush=True)
            if best is None or ms < best[0]:
                best = (ms, variant, tile)
            del ws
    del scratch
    cache[key] = {"variant": best[1], "tile": list(best[2]), "timings": timings}
    if use_cache:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return batch_config(best[1], best[2]), timings
