"""A box whose state holds more than 2^31 doubles (512 x 512 x 320 interior points, 2.37e9 values,
19 GB per state): one RK4 step in the production launch, with sampled points recomputed by the
oracle on frozen-ghost sub-boxes. Offsets past 2^31 elements (the last fields, the high-k planes)
are exercised by the ghost fill, the gather, the stage update and the stores. The state is
generated on the device from smooth analytic profiles, so host memory stays small."""
import math

import numpy as np
import pytest

import grf_inputs as gi

pytestmark = pytest.mark.gpu

N = (512, 512, 320)
DX = 0.1


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


def fill_smooth_state(torch, t, box, ng):
    """Every field a constant plus a product of sinusoids of its own wave numbers and phases (the
    metric near flat, the lapse near one, the rest small), evaluated on the ghosted grid. The wave
    numbers are whole multiples of 2 pi / L per axis, so the data are smooth across the periodic
    seam too."""
    nzg, nyg, pitch = t.shape[1], t.shape[2], t.shape[3]
    dev = t.device
    x = box.x0 + (torch.arange(pitch, dtype=torch.float64, device=dev) - ng) * box.dx
    y = box.y0 + (torch.arange(nyg, dtype=torch.float64, device=dev) - ng) * box.dx
    z = box.z0 + (torch.arange(nzg, dtype=torch.float64, device=dev) - ng) * box.dx
    rng = np.random.default_rng(17)
    base = np.zeros(27)
    base[0] = 1.0                     # chi
    base[[1, 4, 6]] = 1.0             # h_ii
    base[18] = 1.0                    # lapse
    amp = np.full(27, 0.02)
    amp[[0, 18]] = 0.05
    lx, ly, lz = (n * box.dx for n in (box.nx, box.ny, box.nz))
    for f in range(27):
        kx, ky, kz = (2.0 * math.pi * rng.integers(1, 6) / ln for ln in (lx, ly, lz))
        px, py, pz = rng.uniform(0.0, 2.0 * math.pi, 3)
        sx = torch.sin(kx * x + px)
        sy = torch.cos(ky * y + py)
        sz = torch.sin(kz * z + pz)
        t[f] = base[f] + amp[f] * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def test_box_beyond_2_31_elements(g, orc):
    import torch
    box = gi.Box(*N, DX, -0.5 * N[0] * DX, -0.5 * N[1] * DX, -0.5 * N[2] * DX)
    b = g.box_like(box)
    shape = g.state_shape(b)
    assert shape[0] * shape[1] * shape[2] * shape[3] > 2 ** 31
    params = gi.Params(lam=0.2, g2=0.1, beta_kind=gi.BETA_LINEAR)
    dt = 0.25 * DX
    t = g.alloc_state(b)
    fill_smooth_state(torch, t, box, box.ng)
    g.grf_fill_ghosts(b, t)
    # samples: the corners of the interior (highest offsets at the last k plane) and a few inside
    nx, ny, nz = N
    samples = [(nx - 1, ny - 1, nz - 1), (0, 0, 0), (nx - 1, 0, nz - 1), (0, ny - 1, nz - 2), (257, 130, 301),
               (11, 400, 160)]
    R = 9
    subs = []
    for (i, j, k) in samples:
        idx = [torch.tensor((np.arange(2 * R + 7) + c - R - 3) % n + 3, device="cuda") for c, n in ((k, nz), (j, ny), (i, nx))]
        blk = t.index_select(1, idx[0]).index_select(2, idx[1]).index_select(3, idx[2])
        subs.append(blk.cpu().numpy())
    scale0 = np.array([float(torch.amax(torch.abs(t[f, 3:3 + nz, 3:3 + ny, 3:3 + nx]))) for f in range(27)])
    g.grf_rk4_step(b, g.params_like(params), t, dt, 1)
    assert g.grf_check_status() == 0
    gots = [t[:, k + 3, j + 3, i + 3].cpu().numpy() for (i, j, k) in samples]
    del t
    torch.cuda.empty_cache()
    sub = gi.Box(2 * R + 1, 2 * R + 1, 2 * R + 1, DX, 0.0, 0.0, 0.0, bc=gi.BC_FROZEN)
    refs, noise = [], []
    for s0 in subs:
        ss = s0.copy()  # the oracle steps its argument in place; s0 stays the initial state
        orc.rk4(sub, params, ss, dt, 1)
        ref = ss[:, R + 3, R + 3, R + 3]
        spread = np.zeros(27)
        for seed in (1, 2):
            sp = s0 * (1.0 + 2.0 ** -52 * np.random.default_rng(seed).standard_normal(s0.shape))
            orc.rk4(sub, params, sp, dt, 1)
            spread = np.maximum(spread, np.abs(sp[:, R + 3, R + 3, R + 3] - ref))
        refs.append(ref)
        noise.append(spread)
    scale = np.maximum(np.maximum(scale0, np.max(np.abs(refs), axis=0)), 1e-12)
    for n, (i, j, k) in enumerate(samples):
        # the noise floor is rounding (~1e-15 absolute here), far below what a stale state would give
        assert np.max(noise[n] / scale) < 1e-11
        err = np.abs(gots[n] - refs[n]) / np.maximum(1e-11 * scale, 64.0 * noise[n])
        assert np.max(err) < 1.0, (i, j, k, int(np.argmax(err)), float(np.max(err)))
