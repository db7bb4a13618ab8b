"""Shared helpers of the GPU-vs-oracle parity tests."""
import numpy as np

import grf_inputs as gi


def field_errors(gpu, cpu, box, floor=1e-12, state=None, sigma=0.0):
    """err_f = max|gpu_f - cpu_f| / max(max|cpu_f|, floor_f) over interior points, per field.

    For right-hand sides, pass the input `state` and the KO strength: the floor then also
    includes 1e-4 * sigma/dx * max|u_f|. The KO sum of 19 values weighted by up to 20 has a
    rounding error of ~1e-15 sigma/dx max|u|, which a field whose RHS is only the (tiny,
    cancelling) dissipation term would otherwise divide by its own small value."""
    g = box.interior(gpu)
    c = box.interior(cpu)
    nf = c.shape[0]
    out = np.zeros(nf)
    for f in range(nf):
        fl = floor
        if state is not None:
            fl = max(fl, 1e-4 * sigma / box.dx * np.max(np.abs(state[f])))
        den = max(np.max(np.abs(c[f])), fl)
        out[f] = np.max(np.abs(g[f] - c[f])) / den
    return out


def describe(errs, names=gi.FIELD_NAMES):
    worst = np.argsort(errs)[::-1][:5]
    return ", ".join(f"{names[i] if i < len(names) else i}={errs[i]:.2e}" for i in worst)
