"""Waveform extraction on spheres ("Diagnostics": tensor and scalar waveforms) on the GPU against
the oracle: modes of spin weight 0 and -2 to 1e-12 of the largest mode, and exactly the solid
harmonics' modes."""
import math

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


def field_on_device(g, b, f):
    """A single ghosted field (numpy, shape of one field of the box) on the device, padded rows."""
    import torch
    t = torch.zeros(g.state_shape(b, 1), dtype=torch.float64, device="cuda")
    t[..., :f.shape[-1]].copy_(torch.from_numpy(np.ascontiguousarray(f)))
    return t[0]


@pytest.mark.parametrize("ng", [3, 4])
def test_scalar_waveform_modes_parity(g, orc, ng):
    """phi of a generic state on a sphere off the box centre: spin-0 modes up to l = 8."""
    box = gi.Box(30, 28, 26, 0.2, -2.9, -2.7, -2.5, bc=gi.BC_PERIODIC, ng=ng)
    s = gi.random_perturbed_state(box, 71, base=gi.single_puncture(box, amp=0.05), eps=3e-2)
    orc.fill_ghosts(box, s)
    b = g.box_like(box)
    c, R = (0.1, -0.15, 0.05), 1.9
    ref = orc.extract_modes(box, s[25], None, 0, R, c, 12, 24, 8)
    got = g.grf_extract_modes(b, field_on_device(g, b, s[25]), None, 0, R, c, 12, 24, 8)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_spin_minus_two_modes_parity(g, orc):
    """A complex field (two fields of the state as real and imaginary parts), spin -2, l <= 6."""
    box = gi.Box(26, 26, 26, 0.2, -2.5, -2.5, -2.5, bc=gi.BC_PERIODIC)
    s = gi.random_perturbed_state(box, 73, eps=3e-2)
    orc.fill_ghosts(box, s)
    b = g.box_like(box)
    c, R = (0.0, 0.0, 0.0), 2.0
    ref = orc.extract_modes(box, s[8], s[9], -2, R, c, 16, 32, 6)
    got = g.grf_extract_modes(b, field_on_device(g, b, s[8]), field_on_device(g, b, s[9]), -2, R, c, 16, 32, 6)
    assert np.all(got[:4] == 0)  # l < 2 has no spin -2 modes
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("lm", [(1, 1), (2, -2), (3, 1)])
def test_solid_harmonic_modes_are_exact(g, lm):
    """r^l Y_lm (l <= 3) is reproduced by the cubic interpolation and the quadrature: a_lm = R^l."""
    sph = pytest.importorskip("scipy.special")
    l, m = lm
    box = gi.Box(20, 18, 19, 0.2, -1.9, -1.7, -1.8, bc=gi.BC_FROZEN)
    X, Y, Z = box.coords()
    c = (0.13, -0.07, 0.21)
    dx, dy, dz = X - c[0], Y - c[1], Z - c[2]
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    th = np.arccos(np.clip(dz / np.where(r > 0, r, 1), -1, 1))
    f = r ** l * sph.sph_harm_y(l, m, th, np.arctan2(dy, dx))
    b = g.box_like(box)
    got = g.grf_extract_modes(b, field_on_device(g, b, f.real), field_on_device(g, b, f.imag), 0, 1.1, c, 8, 16, 4)
    ref = np.zeros(25, complex)
    ref[l * l + l + m] = 1.1 ** l
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_extraction_rejects_spheres_leaving_the_box(g):
    import torch
    box = gi.Box(16, 16, 16, 0.2, -1.5, -1.5, -1.5, bc=gi.BC_FROZEN)
    b = g.box_like(box)
    f = torch.zeros(g.state_shape(b, 1), dtype=torch.float64, device="cuda")[0]
    g.grf_extract_modes(b, f, None, 0, 1.4, (0.0, 0.0, 0.0), 4, 8, 2)  # fits (stencils reach the ghosts)
    with pytest.raises(g.GrfError) as e:
        g.grf_extract_modes(b, f, None, 0, 1.7, (0.0, 0.0, 0.0), 4, 8, 2)
    assert e.value.code == g.GRF_EINVAL


@pytest.mark.parametrize("ng", [3, 4])
def test_weyl_psi4_parity(g, orc, ng):
    """Psi_4 on a generic state (couplings on) against the oracle's full-Weyl contraction, to
    1e-11 of its maximum; then the tensor waveform: the spin -2 modes of the GPU's Psi_4 against
    the oracle's modes of its own Psi_4."""
    import torch
    box = gi.Box(22, 20, 18, 0.25, -2.6, -2.4, -2.1, bc=gi.BC_PERIODIC, ng=ng)
    params = gi.Params(lam=0.3, g2=0.2, beta_kind=1)
    s = gi.random_perturbed_state(box, 79, base=gi.single_puncture(box, amp=0.05), eps=3e-2)
    orc.enforce(box, params, s)
    orc.fill_ghosts(box, s)
    ref = orc.psi4(box, params, s)
    b = g.box_like(box)
    t = g.to_device(s, b)
    out = g.alloc_state(b, 2)
    g.grf_weyl_psi4(b, g.params_like(params), t, out)
    assert g.grf_check_status() == 0
    got = g.to_host(out, b)
    psi = box.interior(got[0]) + 1j * box.interior(got[1])
    assert np.max(np.abs(ref)) > 1e-4
    assert np.max(np.abs(psi - ref)) <= 1e-11 * np.max(np.abs(ref))
    # modes: the oracle extracts from its Psi_4 placed in a ghosted field (ghosts from the GPU's
    # fill, which the sphere's stencils do not reach)
    full = np.zeros((2,) + box.shape[1:])
    full[0], full[1] = got[0], got[1]
    gg = box.ng
    full[0][gg:-gg, gg:-gg, gg:-gg] = ref.real
    full[1][gg:-gg, gg:-gg, gg:-gg] = ref.imag
    c, R = (0.1, 0.05, -0.1), 1.6
    mref = orc.extract_modes(box, full[0], full[1], -2, R, c, 12, 24, 6)
    mgot = g.grf_extract_modes(b, out[0], out[1], -2, R, c, 12, 24, 6)
    assert np.max(np.abs(mgot - mref)) <= 1e-10 * np.max(np.abs(mref))
    torch.cuda.synchronize()
