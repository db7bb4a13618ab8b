"""Host-side checks of the C-ABI library (no GPU needed): it builds for sm_103a, loads, and
exports every entry point declared in include/grf.h; argument validation that needs no
device memory rejects bad boxes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def grf():
    from paper_2309_06225_gb300 import build
    build.build()
    import paper_2309_06225_gb300 as g
    try:
        g.lib()
    except OSError as e:  # libcudart missing on a machine without the toolkit
        pytest.skip(f"cannot load libgrf.so here: {e}")
    return g


def declared_functions():
    src = open(os.path.join(ROOT, "include", "grf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("grf_rhs", "grf_rk4_step", "grf_constraints", "grf_ko_dissipation"):
        assert n in names


def test_library_exports_every_declared_symbol(grf):
    L = grf.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_peak_library_exports_its_declared_symbol():
    """include/grf_peak.h (the FP64 microbenchmark of the roofline denominator) and libgrf_peak.so."""
    from paper_2309_06225_gb300 import build_peak
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "grf_peak.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(grf_[a-z0-9_]+)\s*\(", src)))
    assert names == ["grf_peak_fp64"]
    try:
        L = C.CDLL(build_peak.build())
    except OSError as e:  # libcudart missing on a machine without the toolkit
        pytest.skip(f"cannot load libgrf_peak.so here: {e}")
    for name in names:
        assert hasattr(L, name), name


def test_workspace_and_validation_without_gpu(grf):
    b = grf.make_box(32, 32, 32, 0.25)
    nbytes = grf.grf_workspace_bytes(b, grf.GRF_OP_RK4)
    assert nbytes == 3 * 8 * 27 * 38 * 38 * b.pitch
    bad = grf.make_box(32, 32, 32, 0.25)
    bad.ng = 2
    assert grf.grf_workspace_bytes(bad, grf.GRF_OP_RK4) == 0
    bad = grf.make_box(32, 32, 32, 0.25, pitch=30)
    assert grf.grf_workspace_bytes(bad, grf.GRF_OP_RK4) == 0
    L = grf.lib()
    p = grf.grf_params()
    # invalid boxes / null pointers are rejected before any CUDA call
    assert L.grf_rhs(C.byref(bad), C.byref(p), None, None, None, 0, None) == grf.GRF_EINVAL
    assert L.grf_rk4_step(C.byref(b), C.byref(p), None, 0.1, 1, None, 0, None) == grf.GRF_EINVAL
    good_state = C.c_void_p(0x1000)
    assert L.grf_rk4_step(C.byref(b), C.byref(p), good_state, 0.1, 1, None, 0, None) == grf.GRF_EWORKSPACE
    assert "workspace" in grf.grf_error_string(grf.GRF_EWORKSPACE)


def test_host_step_validation_without_gpu(grf):
    b = grf.make_box(16, 16, 16, 0.25)
    p = grf.grf_params()
    L = grf.lib()
    fake = C.c_void_p(0x1000)
    assert L.grf_rk4_step_host(C.byref(b), C.byref(p), None, fake, fake, 0.1, 1, fake, 1 << 30, None) == grf.GRF_EINVAL
    assert L.grf_rk4_step_host(C.byref(b), C.byref(p), fake, fake, fake, 0.1, -1, fake, 1 << 30, None) == grf.GRF_EINVAL
    assert L.grf_rk4_step_host(C.byref(b), C.byref(p), fake, fake, fake, 0.1, 1, None, 0, None) == grf.GRF_EWORKSPACE


def test_scheme_validation_without_gpu(grf):
    """4-ghost boxes (6th-order scheme) are sized with their ghosts; lopsided advection is rejected
    by the tangent call and any advection value other than 0 or 1 everywhere, all before a CUDA
    call."""
    b6 = grf.make_box(20, 18, 16, 0.25, ng=4)
    assert b6.pitch >= 28 and b6.pitch % 4 == 0
    assert grf.grf_workspace_bytes(b6, grf.GRF_OP_RK4) == 3 * 8 * 27 * 24 * 26 * b6.pitch
    small = grf.make_box(3, 8, 8, 0.25, ng=4)  # periodic 6th-order boxes need >= 4 points per axis
    assert grf.grf_workspace_bytes(small, grf.GRF_OP_RK4) == 0
    L = grf.lib()
    fake = C.c_void_p(0x1000)
    p = grf.grf_params()
    assert L.grf_rk4_step_host(C.byref(b6), C.byref(p), None, fake, fake, 0.1, 1, fake, 1 << 40, None) == grf.GRF_EINVAL
    b3 = grf.make_box(16, 16, 16, 0.25)
    p.advection = 2
    assert L.grf_rhs(C.byref(b3), C.byref(p), fake, fake, None, 0, None) == grf.GRF_EINVAL
    item = grf.grf_batch_item(b3, fake, 0, 0.1)
    cfg = grf.grf_batch_config(grf.GRF_BATCH_STREAM, 32, 4, 1, 0, 0)
    assert L.grf_batched_rk4(C.byref(item), 1, C.byref(p), 1, 1, C.byref(cfg), fake, 1 << 40, None, None) == grf.GRF_EINVAL
    p.advection = 1
    sphere = grf.grf_sphere()
    sphere.radius = 1.0
    dpar = (C.c_double * 6)()
    loss = (C.c_double * 4)()
    assert L.grf_tlm_rk4(C.byref(b3), C.byref(p), dpar, fake, fake, 0.1, 1, C.byref(sphere), loss, fake, 1 << 40,
                         None) == grf.GRF_EINVAL


def test_outer_boundaries_validation_without_gpu(grf):
    """Extrapolating and Sommerfeld boxes need n >= ng."""
    L = grf.lib()
    fake = C.c_void_p(0x1000)
    p = grf.grf_params()
    for bc in (grf.GRF_BC_EXTRAPOLATE, grf.GRF_BC_SOMMERFELD):
        b = grf.make_box(8, 8, 8, 0.25, bc=bc)
        assert grf.grf_workspace_bytes(b, grf.GRF_OP_RK4) > 0
        assert L.grf_rk4_step_host(C.byref(b), C.byref(p), fake, fake, None, 0.1, 1, fake, 1 << 40, None) == grf.GRF_EINVAL
        assert grf.grf_workspace_bytes(grf.make_box(2, 8, 8, 0.25, bc=bc), grf.GRF_OP_RK4) == 0
    assert grf.grf_workspace_bytes(grf.make_box(8, 8, 8, 0.25, bc=6), grf.GRF_OP_RK4) == 0


def test_extraction_validation_without_gpu(grf):
    """Argument ranges of grf_extract_modes are checked before any CUDA call."""
    L = grf.lib()
    b = grf.make_box(16, 16, 16, 0.2, -1.5, -1.5, -1.5, bc=grf.GRF_BC_FROZEN)
    fake = C.c_void_p(0x1000)
    host = (C.c_double * 400)()
    assert grf.grf_extract_workspace_bytes(8, 4) > 0
    assert grf.grf_extract_workspace_bytes(8, 13) == 0 and grf.grf_extract_workspace_bytes(0, 4) == 0
    for spin, R, nth, nph, lmax in ((1, 1.0, 8, 16, 4), (0, 1.0, 8, 4096, 4), (0, 1.0, 8, 16, 13), (0, -1.0, 8, 16, 4),
                                    (0, 1.7, 8, 16, 4), (-2, 1.0, 600, 16, 4)):
        sph = grf.grf_sphere(R, 0.0, 0.0, 0.0)
        assert L.grf_extract_modes(C.byref(b), fake, None, spin, C.byref(sph), nth, nph, lmax, host, fake, 1 << 30,
                                   None) == grf.GRF_EINVAL
    sph = grf.grf_sphere(1.0, 0.0, 0.0, 0.0)
    assert L.grf_extract_modes(C.byref(b), fake, None, 0, C.byref(sph), 8, 16, 4, host, fake, 8, None) == grf.GRF_EWORKSPACE


def test_mirror_sommerfeld_validation_without_gpu(grf):
    L = grf.lib()
    fake = C.c_void_p(0x1000)
    p = grf.grf_params()
    b = grf.make_box(8, 8, 8, 0.25, bc=grf.GRF_BC_REFLECT_LOW_SOMMERFELD)
    assert grf.grf_workspace_bytes(b, grf.GRF_OP_RK4) > 0
    assert L.grf_rk4_step_host(C.byref(b), C.byref(p), fake, None, fake, 0.1, 1, fake, 1 << 40, None) == grf.GRF_EINVAL
    assert grf.grf_workspace_bytes(grf.make_box(2, 8, 8, 0.25, bc=grf.GRF_BC_REFLECT_LOW_SOMMERFELD),
                                   grf.GRF_OP_RK4) == 0


def test_adjoint_validation_without_gpu(grf):
    """The reverse sweep accepts 3-ghost periodic / frozen boxes with centred advection; other
    boxes have no workspace size and every bad argument is rejected before any CUDA call."""
    b = grf.make_box(16, 16, 16, 0.5)
    assert grf.grf_adjoint_workspace_bytes(b, 20) > 0
    assert grf.grf_adjoint_workspace_bytes(b, 0) == 0
    assert grf.grf_adjoint_workspace_bytes(grf.make_box(16, 16, 16, 0.5, ng=4), 20) == 0
    assert grf.grf_adjoint_workspace_bytes(grf.make_box(16, 16, 16, 0.5, bc=grf.GRF_BC_SOMMERFELD), 20) == 0
    import grf_inputs as gi
    L = grf.lib()
    sph = grf.grf_sphere(2.0, 0.0, 0.0, 0.0)
    lop = grf.params_like(gi.Params(advection=1))
    ok = grf.params_like(gi.Params())
    fake = C.c_void_p(256)  # never dereferenced: validation fails first
    assert L.grf_adjoint_rk4(C.byref(b), C.byref(lop), fake, 0.1, 4, C.byref(sph), 2, 1.0, fake, fake, fake,
                             1 << 40, None) == grf.GRF_EINVAL
    assert L.grf_adjoint_rk4(C.byref(b), C.byref(ok), fake, 0.1, 4, C.byref(sph), 0, 1.0, fake, fake, fake,
                             1 << 40, None) == grf.GRF_EINVAL
    bad = grf.grf_sphere(-1.0, 0.0, 0.0, 0.0)
    assert L.grf_signal_forward(C.byref(b), C.byref(ok), fake, 0.1, 4, C.byref(bad), 2, fake, fake, fake, 1 << 40,
                                None) == grf.GRF_EINVAL
    assert L.grf_adjoint_rk4(C.byref(b), C.byref(ok), fake, 0.1, 4, C.byref(sph), 2, 1.0, fake, fake, None, 0,
                             None) == grf.GRF_EWORKSPACE


def test_empty_and_degenerate_calls_without_gpu(grf):
    """Empty boxes and negative step counts are rejected, and zero steps is a successful no-op, all
    before any CUDA call (so these run without a GPU). A 1 x 1 x 1 frozen box is a valid box."""
    L = grf.lib()
    p = grf.grf_params()
    fake_state = C.c_void_p(0x1000)
    fake_ws = C.c_void_p(0x10000)  # 256-byte aligned, never touched
    for n in ((0, 8, 8), (8, 0, 8), (8, 8, 0)):
        b = grf.make_box(*n, 0.25)
        assert grf.grf_workspace_bytes(b, grf.GRF_OP_RK4) == 0
        assert L.grf_rk4_step(C.byref(b), C.byref(p), fake_state, 0.1, 1, fake_ws, 1 << 40, None) == grf.GRF_EINVAL
        assert L.grf_rhs(C.byref(b), C.byref(p), fake_state, fake_state, None, 0, None) == grf.GRF_EINVAL
    b = grf.make_box(8, 8, 8, 0.25)
    nbytes = grf.grf_workspace_bytes(b, grf.GRF_OP_RK4)
    assert L.grf_rk4_step(C.byref(b), C.byref(p), fake_state, 0.1, -1, fake_ws, nbytes, None) == grf.GRF_EINVAL
    assert L.grf_rk4_step(C.byref(b), C.byref(p), fake_state, 0.1, 0, fake_ws, nbytes, None) == grf.GRF_OK
    one = grf.make_box(1, 1, 1, 0.25, bc=grf.GRF_BC_FROZEN)
    assert grf.grf_workspace_bytes(one, grf.GRF_OP_RK4) > 0
    assert L.grf_rk4_step(C.byref(one), C.byref(p), fake_state, 0.1, 0, fake_ws, 1 << 40, None) == grf.GRF_OK
    # a periodic box needs at least the ghost width of points per axis
    two = grf.make_box(2, 8, 8, 0.25)
    assert grf.grf_workspace_bytes(two, grf.GRF_OP_RK4) == 0


def test_hyperbolicity_output_shape_is_checked_without_gpu(grf):
    """grf_hyperbolicity writes 4 fields: an output tensor of another shape is refused before
    anything reaches the library."""
    import torch
    b = grf.make_box(8, 8, 8, 0.25)
    state = torch.zeros(grf.state_shape(b), dtype=torch.float64)
    with pytest.raises(ValueError):
        grf.grf_hyperbolicity(b, grf.grf_params(), state, torch.zeros(grf.state_shape(b, 3), dtype=torch.float64))
