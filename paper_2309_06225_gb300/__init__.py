"""Python binding of libgrf.so, the GB300 C-ABI library for the modified-CCZ4 + 4dST
evolution (GRFolres, arXiv:2309.06225).

Argument marshalling only: every computation runs in the library's CUDA kernels. PyTorch
provides device memory and streams. There is no CPU fallback: if libgrf.so is missing or
cannot be loaded, importing a function raises.

State tensors are float64 CUDA tensors of shape (27, nz+6, ny+6, pitch) (field-major,
ghosted, x fastest, rows padded to `pitch` doubles); see include/grf.h for the layout and
the meaning of every argument.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrf.so")

GRF_OK, GRF_EINVAL, GRF_EWORKSPACE, GRF_ECUDA, GRF_ENONFINITE, GRF_ESINGULAR, GRF_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
GRF_ETOOLARGE = -7
GRF_NOALLOC_SCRATCH_BYTES = 48 * 1024 * 1024
GRF_BC_PERIODIC, GRF_BC_FROZEN, GRF_BC_REFLECT_LOW, GRF_BC_EXTRAPOLATE, GRF_BC_SOMMERFELD = 0, 1, 2, 3, 4
GRF_BC_REFLECT_LOW_SOMMERFELD = 5
GRF_BETA_LINEAR, GRF_BETA_QUADRATIC = 0, 1
GRF_OP_RHS, GRF_OP_RK4, GRF_OP_CONSTRAINTS = 0, 1, 2
NFIELDS, NG = 27, 3


class grf_box(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("ng", C.c_int), ("dx", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double), ("bc", C.c_int),
                ("pitch", C.c_longlong)]


class grf_params(C.Structure):
    _fields_ = [("kappa1", C.c_double), ("kappa2", C.c_double), ("kappa3", C.c_double),
                ("shift_F", C.c_double), ("eta", C.c_double), ("a0", C.c_double), ("b0", C.c_double),
                ("lambda_", C.c_double), ("g2", C.c_double), ("sigma_ko", C.c_double),
                ("min_chi", C.c_double), ("min_lapse", C.c_double),
                ("beta_kind", C.c_int), ("enforce_algebraic", C.c_int), ("decoupled", C.c_int),
                ("advection", C.c_int), ("beta_kappa", C.c_double), ("g3", C.c_double)]


GRF_BATCH_GRAPH, GRF_BATCH_PERSISTENT, GRF_BATCH_STREAM = 1, 2, 3


class grf_batch_item(C.Structure):
    _fields_ = [("box", grf_box), ("state", C.c_void_p), ("params_index", C.c_int), ("dt", C.c_double)]


class grf_batch_config(C.Structure):
    _fields_ = [("variant", C.c_int), ("tile_x", C.c_int), ("tile_y", C.c_int), ("tile_z", C.c_int),
                ("blocks_per_sm", C.c_int), ("barrier_timeout_cycles", C.c_longlong)]


class grf_sphere(C.Structure):
    _fields_ = [("radius", C.c_double), ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double)]


GRF_MAX_PATCHES_PER_AXIS, GRF_MAX_PATCHES = 16, 256


class grf_patch_level(C.Structure):
    _fields_ = [("box", grf_box), ("px", C.c_int), ("py", C.c_int), ("pz", C.c_int)]


class grf_halo_block(C.Structure):
    _fields_ = [("dst", C.c_int), ("src", C.c_int), ("dst_i", C.c_int), ("dst_j", C.c_int), ("dst_k", C.c_int),
                ("src_i", C.c_int), ("src_j", C.c_int), ("src_k", C.c_int), ("ni", C.c_int), ("nj", C.c_int),
                ("nk", C.c_int)]


# int (*)(void* ctx, const grf_patch_level*, double* const* patches, grf_stream_t)
grf_halo_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(grf_patch_level), C.POINTER(C.c_void_p), C.c_void_p)


class GrfError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = f"{what}: {lib().grf_error_string(code).decode()} (code {code})"
        if code == GRF_ECUDA:
            msg += f": {lib().grf_last_cuda_error().decode()}"
        super().__init__(msg)


_lib = None
_VP = C.c_void_p


def lib():
    """Loads libgrf.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libgrf.so not built ({LIB_PATH}); run paper_2309_06225_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        B, P = C.POINTER(grf_box), C.POINTER(grf_params)
        L.grf_rhs.argtypes = [B, P, _VP, _VP, _VP, C.c_size_t, _VP]
        L.grf_rk4_step.argtypes = [B, P, _VP, C.c_double, C.c_int, _VP, C.c_size_t, _VP]
        L.grf_rk4_step_host.argtypes = [B, P, _VP, _VP, _VP, C.c_double, C.c_int, _VP, C.c_size_t, _VP]
        L.grf_constraints.argtypes = [B, P, _VP, _VP, C.POINTER(C.c_double), _VP, C.c_size_t, _VP]
        L.grf_energy_densities.argtypes = [B, P, _VP, _VP, _VP]
        L.grf_ko_dissipation.argtypes = [B, C.c_double, _VP, _VP, _VP]
        L.grf_fill_ghosts.argtypes = [B, _VP, _VP]
        L.grf_workspace_bytes.argtypes = [B, C.c_int]
        L.grf_workspace_bytes.restype = C.c_size_t
        L.grf_check_status.argtypes = [_VP]
        L.grf_check_finite.argtypes = [B, _VP, _VP, C.c_size_t, _VP]
        BI, BC = C.POINTER(grf_batch_item), C.POINTER(grf_batch_config)
        L.grf_batched_workspace_bytes.argtypes = [BI, C.c_int, BC]
        L.grf_batched_workspace_bytes.restype = C.c_size_t
        L.grf_batched_rk4.argtypes = [BI, C.c_int, P, C.c_int, C.c_int, BC, _VP, C.c_size_t, C.POINTER(C.c_int), _VP]
        L.grf_batched_rk4.restype = C.c_int
        L.grf_tlm_workspace_bytes.argtypes = [B]
        L.grf_tlm_workspace_bytes.restype = C.c_size_t
        L.grf_weyl_psi4.argtypes = [B, P, _VP, _VP, _VP]
        L.grf_hyperbolicity.argtypes = [B, P, _VP, _VP, _VP]
        L.grf_hyperbolicity.restype = C.c_int
        L.grf_extract_workspace_bytes.argtypes = [C.c_int, C.c_int]
        L.grf_extract_workspace_bytes.restype = C.c_size_t
        L.grf_extract_modes.argtypes = [B, _VP, _VP, C.c_int, C.POINTER(grf_sphere), C.c_int, C.c_int, C.c_int,
                                        C.POINTER(C.c_double), _VP, C.c_size_t, _VP]
        L.grf_tlm_rk4.argtypes = [B, P, C.POINTER(C.c_double), _VP, _VP, C.c_double, C.c_int, C.POINTER(grf_sphere),
                                  _VP, _VP, C.c_size_t, _VP]
        L.grf_tlm_rk4.restype = C.c_int
        L.grf_adjoint_workspace_bytes.argtypes = [B, C.c_int]
        L.grf_adjoint_workspace_bytes.restype = C.c_size_t
        L.grf_signal_forward.argtypes = [B, P, _VP, C.c_double, C.c_int, C.POINTER(grf_sphere), C.c_int, _VP, _VP,
                                         _VP, C.c_size_t, _VP]
        L.grf_signal_forward.restype = C.c_int
        L.grf_adjoint_rk4.argtypes = [B, P, _VP, C.c_double, C.c_int, C.POINTER(grf_sphere), C.c_int, C.c_double, _VP,
                                      _VP, _VP, C.c_size_t, _VP]
        L.grf_adjoint_rk4.restype = C.c_int
        L.grf_state_dot.argtypes = [B, _VP, _VP, C.c_int, _VP, _VP, C.c_size_t, _VP]
        L.grf_state_dot.restype = C.c_int
        L.grf_rk4_step_noalloc.argtypes = [B, P, _VP, C.c_double, C.c_int, _VP]
        L.grf_rk4_step_noalloc.restype = C.c_int
        PL, PP = C.POINTER(grf_patch_level), C.POINTER(C.c_void_p)
        L.grf_patch_box.argtypes = [PL, C.c_int, B]
        L.grf_patch_copy.argtypes = [PL, _VP, PP, C.c_int, _VP]
        L.grf_halo_exchange.argtypes = [PL, PP, _VP]
        L.grf_halo_plan.argtypes = [PL, C.POINTER(grf_halo_block), C.c_int]
        L.grf_halo_plan.restype = C.c_int
        L.grf_patches_workspace_bytes.argtypes = [PL]
        L.grf_patches_workspace_bytes.restype = C.c_size_t
        L.grf_patches_rk4.argtypes = [PL, P, PP, C.c_double, C.c_int, grf_halo_fn, _VP, _VP, C.c_size_t,
                                      C.POINTER(C.c_int), _VP]
        L.grf_patches_constraints_workspace_bytes.argtypes = [PL]
        L.grf_patches_constraints_workspace_bytes.restype = C.c_size_t
        L.grf_patches_constraints.argtypes = [PL, P, PP, PP, C.POINTER(C.c_double), _VP, C.c_size_t, _VP]
        for name in ("grf_patch_box", "grf_patch_copy", "grf_halo_exchange", "grf_patches_rk4",
                     "grf_patches_constraints"):
            getattr(L, name).restype = C.c_int
        L.grf_error_string.argtypes = [C.c_int]
        L.grf_error_string.restype = C.c_char_p
        L.grf_last_cuda_error.restype = C.c_char_p
        for name in ("grf_rhs", "grf_rk4_step", "grf_rk4_step_host", "grf_constraints", "grf_energy_densities",
                     "grf_extract_modes", "grf_weyl_psi4", "grf_ko_dissipation", "grf_fill_ghosts",
                     "grf_check_status", "grf_check_finite"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


# ------------------------------------------------------------------------------ marshalling
def pitch_for(nx, ng=NG):
    """Row pitch in doubles: nx + 2 ng rounded up to a multiple of 4 (32-byte rows)."""
    return ((nx + 2 * ng + 3) // 4) * 4


def make_box(nx, ny, nz, dx, x0=0.0, y0=0.0, z0=0.0, bc=GRF_BC_PERIODIC, pitch=None, ng=NG) -> grf_box:
    """ng = 3: 4th-order scheme, ng = 4: 6th-order scheme."""
    return grf_box(int(nx), int(ny), int(nz), int(ng), float(dx), float(x0), float(y0), float(z0), int(bc),
                   int(pitch if pitch is not None else pitch_for(nx, ng)))


def box_like(b, pitch=None) -> grf_box:
    """grf_box from any object with nx, ny, nz, dx, x0, y0, z0, bc (and optionally ng) attributes."""
    return make_box(b.nx, b.ny, b.nz, b.dx, b.x0, b.y0, b.z0, b.bc, pitch, int(getattr(b, "ng", NG)))


def params_like(p) -> grf_params:
    """grf_params from any object with the parameter attributes (lambda under `lam`)."""
    return grf_params(p.kappa1, p.kappa2, p.kappa3, p.shift_F, p.eta, p.a0, p.b0, p.lam, p.g2, p.sigma_ko,
                      p.min_chi, p.min_lapse, int(p.beta_kind), int(p.enforce_algebraic),
                      int(getattr(p, "decoupled", 0)), int(getattr(p, "advection", 0)),
                      float(getattr(p, "beta_kappa", 1.0)), float(getattr(p, "g3", 0.0)))


def state_shape(box: grf_box, nfields=NFIELDS):
    return (nfields, box.nz + 2 * box.ng, box.ny + 2 * box.ng, box.pitch)


def _torch():
    import torch
    return torch


def alloc_state(box: grf_box, nfields=NFIELDS, device="cuda"):
    torch = _torch()
    return torch.zeros(state_shape(box, nfields), dtype=torch.float64, device=device)


def to_device(state_np, box: grf_box, device="cuda", out=None):
    """Copies a (27, nz + 2 ng, ny + 2 ng, nx + 2 ng) numpy array into a padded device tensor."""
    torch = _torch()
    nxg = box.nx + 2 * box.ng
    if out is None:
        out = alloc_state(box, state_np.shape[0], device)
    out[..., :nxg].copy_(torch.from_numpy(np.ascontiguousarray(state_np)))
    return out


def to_host(t, box: grf_box):
    return t[..., :box.nx + 2 * box.ng].cpu().numpy()


def alloc_workspace(nbytes, device="cuda"):
    torch = _torch()
    ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


def _stream(stream):
    if stream is None:
        return _VP(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _VP(stream)
    return _VP(stream.cuda_stream)


def _dev(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous() and str(t.dtype) in ("torch.float64", "torch.uint8")
    return _VP(t.data_ptr())


def _host(t, n):
    """Address of a contiguous float64 host array of n elements (numpy array or CPU tensor)."""
    if isinstance(t, np.ndarray):
        assert t.dtype == np.float64 and t.flags.c_contiguous and t.size == n
        return _VP(t.ctypes.data)
    assert (not t.is_cuda) and t.is_contiguous() and t.dtype == _torch().float64 and t.numel() == n
    return _VP(t.data_ptr())


def _check(code, what):
    if code != GRF_OK:
        raise GrfError(code, what)
    return code


# ------------------------------------------------------------------------------ entry points
def grf_workspace_bytes(box: grf_box, op: int) -> int:
    return int(lib().grf_workspace_bytes(C.byref(box), int(op)))


def grf_fill_ghosts(box: grf_box, state, stream=None):
    return _check(lib().grf_fill_ghosts(C.byref(box), _dev(state), _stream(stream)), "grf_fill_ghosts")


def grf_rhs(box: grf_box, params: grf_params, state, rhs, ws=None, stream=None):
    nb = 0 if ws is None else ws.numel()
    return _check(lib().grf_rhs(C.byref(box), C.byref(params), _dev(state), _dev(rhs), _dev(ws), nb,
                                _stream(stream)), "grf_rhs")


def grf_rk4_step(box: grf_box, params: grf_params, state, dt, nsteps, ws=None, stream=None):
    if ws is None:
        ws = alloc_workspace(grf_workspace_bytes(box, GRF_OP_RK4), state.device)
    return _check(lib().grf_rk4_step(C.byref(box), C.byref(params), _dev(state), float(dt), int(nsteps), _dev(ws),
                                     ws.numel(), _stream(stream)), "grf_rk4_step")


def grf_rk4_step_host(box: grf_box, params: grf_params, host_in, host_out, state, dt, nsteps, ws=None, stream=None):
    """grf_rk4_step from a host array to a host array (layout state_shape(box)), the copies
    overlapped with the first and last RK stage; `state` is the device buffer the step runs in.
    host_in and host_out may be the same array; pinned CPU tensors let the copies overlap."""
    n = int(np.prod(state_shape(box)))
    if ws is None:
        ws = alloc_workspace(grf_workspace_bytes(box, GRF_OP_RK4), state.device)
    return _check(lib().grf_rk4_step_host(C.byref(box), C.byref(params), _host(host_in, n), _host(host_out, n),
                                          _dev(state), float(dt), int(nsteps), _dev(ws), ws.numel(),
                                          _stream(stream)), "grf_rk4_step_host")


def grf_constraints(box: grf_box, params: grf_params, state, out4, norms=True, ws=None, stream=None):
    """Returns the 8 norms {L2(H), max|H|, L2(M1), max|M1|, ...} when norms=True (synchronises)."""
    host = (C.c_double * 8)() if norms else None
    if norms and ws is None:
        ws = alloc_workspace(grf_workspace_bytes(box, GRF_OP_CONSTRAINTS), state.device)
    nb = 0 if ws is None else ws.numel()
    _check(lib().grf_constraints(C.byref(box), C.byref(params), _dev(state), _dev(out4), host, _dev(ws), nb,
                                 _stream(stream)), "grf_constraints")
    return np.array(list(host)) if norms else None


def grf_energy_densities(box: grf_box, params: grf_params, state, out3, stream=None):
    """8 pi rho of the X, g2 X^2 and Gauss-Bonnet terms into out3 (3 fields, state layout)."""
    return _check(lib().grf_energy_densities(C.byref(box), C.byref(params), _dev(state), _dev(out3),
                                             _stream(stream)), "grf_energy_densities")


def grf_hyperbolicity(box: grf_box, params: grf_params, state, out4, stream=None):
    """det M of the coupled system, det(g_eff)/det(g), -g_eff^nn and the system's smallest pivot
    ratio at the interior points (out4: device, 4 fields in the state's layout). See include/grf.h."""
    if hasattr(out4, "shape") and tuple(out4.shape) != state_shape(box, 4):
        raise ValueError(f"grf_hyperbolicity writes 4 fields: out4 must have shape {state_shape(box, 4)}")
    return _check(lib().grf_hyperbolicity(C.byref(box), C.byref(params), _dev(state), _dev(out4), _stream(stream)),
                  "grf_hyperbolicity")


def grf_weyl_psi4(box: grf_box, params: grf_params, state, out2, stream=None):
    """Psi_4 (re, im) at the interior points into out2 (2 fields, state layout)."""
    return _check(lib().grf_weyl_psi4(C.byref(box), C.byref(params), _dev(state), _dev(out2), _stream(stream)),
                  "grf_weyl_psi4")


def grf_extract_workspace_bytes(ntheta, lmax):
    return lib().grf_extract_workspace_bytes(int(ntheta), int(lmax))


def grf_extract_modes(box: grf_box, f_re, f_im, spin, radius, centre, ntheta, nphi, lmax, ws=None, stream=None):
    """Modes a_lm (complex numpy array indexed l^2 + l + m) of the single device field f_re
    (+ i f_im) on the sphere; synchronises."""
    n = 2 * (int(lmax) + 1) ** 2
    host = (C.c_double * n)()
    if ws is None:
        ws = alloc_workspace(lib().grf_extract_workspace_bytes(int(ntheta), int(lmax)), f_re.device)
    sph = grf_sphere(float(radius), *map(float, centre))
    _check(lib().grf_extract_modes(C.byref(box), _dev(f_re), _dev(f_im), int(spin), C.byref(sph), int(ntheta),
                                   int(nphi), int(lmax), host, _dev(ws), ws.numel(), _stream(stream)),
           "grf_extract_modes")
    a = np.array(list(host))
    return a[0::2] + 1j * a[1::2]


def grf_ko_dissipation(box: grf_box, sigma, state, rhs_accum, stream=None):
    return _check(lib().grf_ko_dissipation(C.byref(box), float(sigma), _dev(state), _dev(rhs_accum),
                                           _stream(stream)), "grf_ko_dissipation")


def grf_check_status(stream=None):
    return int(lib().grf_check_status(_stream(stream)))


def grf_check_finite(box: grf_box, state, ws=None, stream=None):
    if ws is None:
        ws = alloc_workspace(256, state.device)
    return int(lib().grf_check_finite(C.byref(box), _dev(state), _dev(ws), ws.numel(), _stream(stream)))


def grf_error_string(code: int) -> str:
    return lib().grf_error_string(int(code)).decode()


# ------------------------------------------------------------------------------ batched boxes
def batch_config(variant=GRF_BATCH_GRAPH, tile=(32, 4, 1), blocks_per_sm=0, barrier_timeout_cycles=0):
    return grf_batch_config(int(variant), int(tile[0]), int(tile[1]), int(tile[2]), int(blocks_per_sm),
                            int(barrier_timeout_cycles))


def batch_items(boxes, states, params_index, dts):
    """ctypes array of grf_batch_item from parallel lists (boxes: grf_box, states: device tensors)."""
    arr = (grf_batch_item * len(boxes))()
    for i, (b, t, pi, dt) in enumerate(zip(boxes, states, params_index, dts)):
        assert t.is_cuda and t.is_contiguous()
        arr[i] = grf_batch_item(b, C.c_void_p(t.data_ptr()), int(pi), float(dt))
    return arr


def params_array(params):
    arr = (grf_params * len(params))()
    for i, p in enumerate(params):
        arr[i] = p
    return arr


def grf_batched_workspace_bytes(items, cfg) -> int:
    return int(lib().grf_batched_workspace_bytes(items, len(items), C.byref(cfg)))


def grf_batched_rk4(items, params, nsteps, cfg, ws=None, stream=None, sync_status=True):
    """Advances every box of `items` (batch_items) by nsteps RK4 steps; params: grf_params array."""
    if ws is None:
        ws = alloc_workspace(grf_batched_workspace_bytes(items, cfg))
    st = C.c_int(0)
    code = lib().grf_batched_rk4(items, len(items), params, len(params), int(nsteps), C.byref(cfg), _dev(ws),
                                 ws.numel(), C.byref(st) if sync_status else None, _stream(stream))
    return _check(code, "grf_batched_rk4")


# ------------------------------------------------------------------------------ one box as patches
def patch_level(box: grf_box, px: int, py: int, pz: int) -> grf_patch_level:
    """A box (periodic or with frozen ghosts) split into px x py x pz patches."""
    return grf_patch_level(box, int(px), int(py), int(pz))


def grf_patch_box(level: grf_patch_level, index: int) -> grf_box:
    """The geometry (frozen-ghost layout) of patch `index` (a + px (b + py c))."""
    out = grf_box()
    _check(lib().grf_patch_box(C.byref(level), int(index), C.byref(out)), "grf_patch_box")
    return out


def patch_states(level: grf_patch_level, device="cuda"):
    """Zeroed patch states, one per patch, each in its grf_patch_box layout."""
    import torch
    n = level.px * level.py * level.pz
    return [torch.zeros(state_shape(grf_patch_box(level, q)), dtype=torch.float64, device=device) for q in range(n)]


def _ptr_array(tensors):
    arr = (C.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        assert t.is_cuda and t.is_contiguous()
        arr[i] = t.data_ptr()
    return arr


def grf_patch_copy(level: grf_patch_level, box_state, patches, direction: int, stream=None):
    """direction 0: every point of the patches, ghosts included, from the box; 1: the box's interior
    from the patches'."""
    return _check(lib().grf_patch_copy(C.byref(level), _dev(box_state), _ptr_array(patches), int(direction),
                                       _stream(stream)), "grf_patch_copy")


def grf_halo_exchange(level: grf_patch_level, patches, stream=None):
    """Every ghost point of every patch from the patch that owns it in the periodic box."""
    return _check(lib().grf_halo_exchange(C.byref(level), _ptr_array(patches), _stream(stream)),
                  "grf_halo_exchange")


def grf_halo_plan(level: grf_patch_level):
    """The level's halo exchange as a list of grf_halo_block (host data; see include/grf.h)."""
    n = lib().grf_halo_plan(C.byref(level), None, 0)
    if n < 0:
        raise GrfError(n, "grf_halo_plan")
    arr = (grf_halo_block * max(n, 1))()
    _check(0 if lib().grf_halo_plan(C.byref(level), arr, n) == n else GRF_EINVAL, "grf_halo_plan")
    return list(arr)[:n]


def grf_patches_workspace_bytes(level: grf_patch_level) -> int:
    return int(lib().grf_patches_workspace_bytes(C.byref(level)))


def grf_patches_rk4(level: grf_patch_level, params: grf_params, patches, dt, nsteps, exchange=None, ws=None,
                    stream=None, sync_status=True):
    """Advances the box held as `patches` by nsteps RK4 steps. exchange: None for the built-in halo
    exchange, or a Python callable (level_ptr, patch_ptr_array, stream) -> int with the grf_halo_fn
    contract (it may call the library, e.g. lib().grf_halo_exchange)."""
    if ws is None:
        ws = alloc_workspace(grf_patches_workspace_bytes(level))
    raised = []

    def call(ctx, lv, ptrs, st):
        # an exception cannot cross the C frames: it ends the step with GRF_EINVAL and is
        # raised again once the call has returned
        try:
            return int(exchange(lv, ptrs, st))
        except BaseException as e:  # noqa: BLE001
            raised.append(e)
            return GRF_EINVAL

    fn = C.cast(None, grf_halo_fn) if exchange is None else grf_halo_fn(call)
    status = C.c_int(0)
    code = lib().grf_patches_rk4(C.byref(level), C.byref(params), _ptr_array(patches), float(dt), int(nsteps), fn,
                                 None, _dev(ws), ws.numel(), C.byref(status) if sync_status else None,
                                 _stream(stream))
    if raised:
        raise raised[0]
    return _check(code, "grf_patches_rk4")


def grf_patches_constraints(level: grf_patch_level, params: grf_params, patches, out4, ws=None, stream=None):
    """H, M_i of every patch into out4 (one 4-field tensor per patch); returns the whole box's 8 norms
    (L2 and max of H, M1, M2, M3)."""
    if ws is None:
        ws = alloc_workspace(lib().grf_patches_constraints_workspace_bytes(C.byref(level)))
    norms = (C.c_double * 8)()
    _check(lib().grf_patches_constraints(C.byref(level), C.byref(params), _ptr_array(patches), _ptr_array(out4),
                                         norms, _dev(ws), ws.numel(), _stream(stream)), "grf_patches_constraints")
    return np.array(norms[:])


def grf_rk4_step_noalloc(box: grf_box, params: grf_params, state, dt, nsteps, stream=None):
    """grf_rk4_step without a workspace: for callers that cannot allocate device memory (the
    scratch is a fixed 48 MiB device array inside the library; boxes whose three stage states
    exceed it are rejected with GRF_ETOOLARGE). See include/grf.h."""
    return _check(lib().grf_rk4_step_noalloc(C.byref(box), C.byref(params), _dev(state), float(dt), int(nsteps),
                                             _stream(stream)), "grf_rk4_step_noalloc")


# ------------------------------------------------------------------------------ tangent-linear signal
def grf_tlm_workspace_bytes(box: grf_box) -> int:
    return int(lib().grf_tlm_workspace_bytes(C.byref(box)))


def grf_tlm_rk4(box: grf_box, params: grf_params, dparams, state, tangents, dt, nsteps, sphere: grf_sphere, loss,
                ws=None, stream=None):
    """Advances state and its 3 tangent states by nsteps RK4 steps and accumulates the sphere
    signal and its 3 directional derivatives into loss (device, 4 doubles). dparams: 6 floats
    {d lambda, d g2} per direction. See include/grf.h."""
    if ws is None:
        ws = alloc_workspace(grf_tlm_workspace_bytes(box))
    dp = (C.c_double * 6)(*[float(x) for x in dparams])
    return _check(lib().grf_tlm_rk4(C.byref(box), C.byref(params), dp, _dev(state), _dev(tangents), float(dt),
                                    int(nsteps), C.byref(sphere), _dev(loss), _dev(ws), ws.numel(), _stream(stream)),
                  "grf_tlm_rk4")


# ------------------------------------------------------------------------------ adjoint signal
def grf_adjoint_workspace_bytes(box: grf_box, checkpoint_every: int) -> int:
    return int(lib().grf_adjoint_workspace_bytes(C.byref(box), int(checkpoint_every)))


def checkpoint_count(nsteps: int, checkpoint_every: int) -> int:
    """States grf_signal_forward stores: one before steps 0, c, 2c, ... below nsteps."""
    return (int(nsteps) + int(checkpoint_every) - 1) // int(checkpoint_every)


def grf_signal_forward(box: grf_box, params: grf_params, state, dt, nsteps, sphere: grf_sphere, checkpoint_every,
                       checkpoints, loss, ws=None, stream=None):
    """Evolves state in place, stores checkpoints (device, checkpoint_count(...) states) and sets
    loss (device, 1 double) to the sphere signal. See include/grf.h."""
    if ws is None:
        ws = alloc_workspace(grf_adjoint_workspace_bytes(box, checkpoint_every))
    return _check(lib().grf_signal_forward(C.byref(box), C.byref(params), _dev(state), float(dt), int(nsteps),
                                           C.byref(sphere), int(checkpoint_every), _dev(checkpoints), _dev(loss),
                                           _dev(ws), ws.numel(), _stream(stream)), "grf_signal_forward")


def grf_adjoint_rk4(box: grf_box, params: grf_params, checkpoints, dt, nsteps, sphere: grf_sphere, checkpoint_every,
                    loss_bar, state_bar, param_bar, ws=None, stream=None):
    """Reverse sweep: state_bar (device state) in = cotangent of the final state, out = gradient
    with respect to the initial state; param_bar (device, 2 doubles) = d/d(lambda, g2). See
    include/grf.h."""
    if ws is None:
        ws = alloc_workspace(grf_adjoint_workspace_bytes(box, checkpoint_every))
    return _check(lib().grf_adjoint_rk4(C.byref(box), C.byref(params), _dev(checkpoints), float(dt), int(nsteps),
                                        C.byref(sphere), int(checkpoint_every), float(loss_bar), _dev(state_bar),
                                        _dev(param_bar), _dev(ws), ws.numel(), _stream(stream)), "grf_adjoint_rk4")


def grf_state_dot(box: grf_box, x, y, field, out, ws=None, stream=None):
    """out (device, 1 double) = interior sum of x * y over one field (or all, field = -1)."""
    if ws is None:
        ws = alloc_workspace(8 * 304, x.device)
    return _check(lib().grf_state_dot(C.byref(box), _dev(x), _dev(y), int(field), _dev(out), _dev(ws), ws.numel(),
                                      _stream(stream)), "grf_state_dot")
