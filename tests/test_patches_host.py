"""Host-side checks of the split-box calls (no GPU needed): the patch geometry tiles the box,
and every argument error is rejected before any CUDA call."""
import ctypes as C

import pytest


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


@pytest.mark.parametrize("n,p", [((37, 20, 11), (3, 2, 1)), ((32, 32, 32), (2, 2, 2)), ((5, 3, 16), (5, 3, 16)),
                                 ((64, 7, 9), (16, 1, 4))])
def test_patches_tile_the_box(grf, n, p):
    """Patch (a, b, c) covers [floor(a n / p), floor((a + 1) n / p)) per axis: consecutive, disjoint,
    covering; origin shifted by the offset; frozen ghosts; 32-byte rows."""
    box = grf.make_box(*n, 0.2, -1.0, 0.5, 2.0)
    L = grf.patch_level(box, *p)
    for c in range(p[2]):
        for b in range(p[1]):
            for a in range(p[0]):
                q = a + p[0] * (b + p[1] * c)
                pb = grf.grf_patch_box(L, q)
                lo = [(a * n[0]) // p[0], (b * n[1]) // p[1], (c * n[2]) // p[2]]
                hi = [((a + 1) * n[0]) // p[0], ((b + 1) * n[1]) // p[1], ((c + 1) * n[2]) // p[2]]
                assert (pb.nx, pb.ny, pb.nz) == tuple(h - l for h, l in zip(hi, lo))
                assert min(pb.nx, pb.ny, pb.nz) >= 1
                assert (pb.x0, pb.y0, pb.z0) == (-1.0 + lo[0] * 0.2, 0.5 + lo[1] * 0.2, 2.0 + lo[2] * 0.2)
                assert pb.ng == 3 and pb.dx == 0.2 and pb.bc == grf.GRF_BC_FROZEN
                assert pb.pitch == grf.pitch_for(pb.nx) and pb.pitch % 4 == 0
    # the x-extents of one row of patches add up to the box
    assert sum(grf.grf_patch_box(L, a).nx for a in range(p[0])) == n[0]


def test_patch_level_validation(grf):
    box = grf.make_box(16, 16, 16, 0.25)
    lib = grf.lib()
    out = grf.grf_box()
    bad = [grf.patch_level(box, 0, 1, 1), grf.patch_level(box, 17, 1, 1), grf.patch_level(box, 1, 1, 17),
           grf.patch_level(grf.make_box(4, 16, 16, 0.25), 5, 1, 1),                 # more patches than points
           grf.patch_level(grf.make_box(16, 16, 16, 0.25, bc=grf.GRF_BC_REFLECT_LOW), 2, 2, 2),
           grf.patch_level(grf.make_box(16, 16, 16, 0.25, bc=grf.GRF_BC_SOMMERFELD), 2, 2, 2),
           grf.patch_level(grf.make_box(16, 16, 16, 0.25, ng=4), 2, 2, 2),
           grf.patch_level(grf.make_box(2, 16, 16, 0.25), 1, 1, 1),                 # periodic box below 3 points
           grf.patch_level(grf.make_box(16, 16, 16, 0.0), 2, 2, 2)]
    big = grf.patch_level(grf.make_box(64, 64, 64, 0.25), 16, 16, 2)              # 512 patches
    for L in bad + [big]:
        assert lib.grf_patch_box(C.byref(L), 0, C.byref(out)) == grf.GRF_EINVAL
        assert lib.grf_patches_workspace_bytes(C.byref(L)) == 0
        ptrs = (C.c_void_p * 512)(*([256] * 512))
        assert lib.grf_halo_exchange(C.byref(L), ptrs, None) == grf.GRF_EINVAL
        assert lib.grf_patches_constraints_workspace_bytes(C.byref(L)) == 0
    # a frozen box may be thinner than the ghost layers; a periodic one may not
    thin = grf.patch_level(grf.make_box(2, 16, 1, 0.25, bc=grf.GRF_BC_FROZEN), 2, 4, 1)
    assert lib.grf_patch_box(C.byref(thin), 7, C.byref(out)) == grf.GRF_OK and (out.nx, out.ny, out.nz) == (1, 4, 1)
    assert lib.grf_patches_workspace_bytes(C.byref(thin)) > 0
    ok = grf.patch_level(box, 2, 2, 2)
    assert lib.grf_patch_box(C.byref(ok), 8, C.byref(out)) == grf.GRF_EINVAL       # index out of range
    assert lib.grf_patch_box(C.byref(ok), -1, C.byref(out)) == grf.GRF_EINVAL
    assert lib.grf_patch_box(C.byref(ok), 0, None) == grf.GRF_EINVAL
    ptrs = (C.c_void_p * 8)(*([256] * 8))
    ptrs_null = (C.c_void_p * 8)(*([256] * 7 + [None]))
    assert lib.grf_halo_exchange(C.byref(ok), ptrs_null, None) == grf.GRF_EINVAL
    assert lib.grf_halo_exchange(C.byref(ok), None, None) == grf.GRF_EINVAL
    assert lib.grf_patch_copy(C.byref(ok), C.c_void_p(256), ptrs, 2, None) == grf.GRF_EINVAL
    assert lib.grf_patch_copy(C.byref(ok), None, ptrs, 0, None) == grf.GRF_EINVAL
    p = grf.grf_params()
    assert lib.grf_patches_constraints(C.byref(ok), C.byref(p), ptrs, ptrs_null, None, None, 0, None) == grf.GRF_EINVAL
    assert lib.grf_patches_constraints(C.byref(ok), None, ptrs, ptrs, None, None, 0, None) == grf.GRF_EINVAL
    # the largest patch's constraint scratch
    assert lib.grf_patches_constraints_workspace_bytes(C.byref(ok)) == \
        grf.grf_workspace_bytes(grf.grf_patch_box(ok, 0), grf.GRF_OP_CONSTRAINTS)


def test_patches_rk4_rejects_before_any_cuda_call(grf):
    box = grf.make_box(16, 16, 16, 0.25)
    L = grf.patch_level(box, 2, 2, 2)
    lib = grf.lib()
    p = grf.grf_params()
    p.kappa1, p.kappa3, p.shift_F, p.eta, p.sigma_ko = 0.1, 1.0, 0.75, 1.0, 0.3
    nbytes = lib.grf_patches_workspace_bytes(C.byref(L))
    # three state-sized buffers per patch (8^3 interiors, 14^3 ghosted, pitch 16) plus descriptors
    assert nbytes > 8 * 3 * 27 * 14 * 14 * 16 * 8
    ptrs = (C.c_void_p * 8)(*([256] * 8))
    none = C.cast(None, grf.grf_halo_fn)
    call = lambda params, nsteps, ws, nb: lib.grf_patches_rk4(C.byref(L), params, ptrs, 0.05, nsteps, none, None,
                                                              ws, nb, None, None)
    assert call(C.byref(p), 0, C.c_void_p(256), nbytes) == grf.GRF_OK          # nothing to do
    assert call(C.byref(p), -1, C.c_void_p(256), nbytes) == grf.GRF_EINVAL
    assert call(None, 1, C.c_void_p(256), nbytes) == grf.GRF_EINVAL
    q = grf.grf_params.from_buffer_copy(p)
    q.beta_kind = 7
    assert call(C.byref(q), 1, C.c_void_p(256), nbytes) == grf.GRF_EINVAL
    q = grf.grf_params.from_buffer_copy(p)
    q.a0 = -1.0
    assert call(C.byref(q), 1, C.c_void_p(256), nbytes) == grf.GRF_EINVAL
    assert call(C.byref(p), 1, None, nbytes) == grf.GRF_EWORKSPACE
    assert call(C.byref(p), 1, C.c_void_p(256), nbytes - 1) == grf.GRF_EWORKSPACE
    assert call(C.byref(p), 1, C.c_void_p(264), nbytes) == grf.GRF_EWORKSPACE  # not 256-byte aligned
