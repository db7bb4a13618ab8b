"""Shared helpers of the GPU-vs-oracle parity tests."""
import numpy as np

import grf_inputs as gi


def field_errors(gpu, cpu, box, floor=1e-12):
    """err_f = max|gpu_f - cpu_f| / max(max|cpu_f|, floor) over interior points, per field."""
    g = box.interior(gpu)
    c = box.interior(cpu)
    nf = c.shape[0]
    out = np.zeros(nf)
    for f in range(nf):
        den = max(np.max(np.abs(c[f])), floor)
        out[f] = np.max(np.abs(g[f] - c[f])) / den
    return out


def describe(errs, names=gi.FIELD_NAMES):
    worst = np.argsort(errs)[::-1][:5]
    return ", ".join(f"{names[i] if i < len(names) else i}={errs[i]:.2e}" for i in worst)
