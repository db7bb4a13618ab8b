"""Python binding of the CPU oracle (ctypes over oracle/liborc.so).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference arm. The product path (paper_2309_06225_gb300) never imports it.
All arrays are float64 numpy arrays in the ghosted field-major layout of grf_inputs.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build


class OrcParams(C.Structure):
    _fields_ = [("kappa1", C.c_double), ("kappa2", C.c_double), ("kappa3", C.c_double),
                ("shift_F", C.c_double), ("eta", C.c_double),
                ("a0", C.c_double), ("b0", C.c_double),
                ("lam", C.c_double), ("g2", C.c_double),
                ("sigma_ko", C.c_double), ("min_chi", C.c_double), ("min_lapse", C.c_double),
                ("beta_kind", C.c_int), ("enforce_algebraic", C.c_int), ("decoupled", C.c_int),
                ("advection", C.c_int), ("beta_kappa", C.c_double), ("g3", C.c_double)]


class OrcBox(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("ng", C.c_int),
                ("dx", C.c_double), ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("bc", C.c_int), ("pad_", C.c_int)]


_lib = None
_P = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_point_rhs.argtypes = [C.POINTER(OrcParams), _P, _P, _P, _P, _P]
        L.orc_point_rhs.restype = C.c_int
        L.orc_point_rhs_adv.argtypes = [C.POINTER(OrcParams), _P, _P, _P, _P, _P, _P]
        L.orc_point_rhs_adv.restype = C.c_int
        L.orc_adv_lopsided.argtypes = [C.POINTER(OrcBox), _P, _P]
        L.orc_point_constraints.argtypes = [C.POINTER(OrcParams), _P, _P, _P, _P]
        L.orc_phys_sources.argtypes = [C.POINTER(OrcParams), _P, _P, C.c_double, _P]
        L.orc_solve.argtypes = [C.c_int, _P, _P, _P]
        L.orc_solve.restype = C.c_int
        L.orc_fill_ghosts.argtypes = [C.POINTER(OrcBox), _P]
        L.orc_derivs.argtypes = [C.POINTER(OrcBox), _P, _P, _P]
        L.orc_rhs.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P, _P, C.c_int]
        L.orc_rhs.restype = C.c_int
        L.orc_ko.argtypes = [C.POINTER(OrcBox), C.c_double, _P, _P]
        L.orc_enforce.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P]
        L.orc_rk4.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P, C.c_double, C.c_int]
        L.orc_rk4.restype = C.c_int
        L.orc_constraints.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P, _P]
        L.orc_energy_densities.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P, _P]
        L.orc_point_energy.argtypes = [C.POINTER(OrcParams), _P, _P, _P, _P]
        L.orc_gauss_legendre.argtypes = [C.c_int, _P, _P]
        L.orc_sylm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _P, _P]
        L.orc_extract_modes.argtypes = [C.POINTER(OrcBox), _P, _P, C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_int, C.c_int, C.c_int, _P]
        L.orc_extract_modes.restype = C.c_int
        L.orc_interp.argtypes = [C.POINTER(OrcBox), _P, C.c_int, _P, _P]
        L.orc_point_psi4.argtypes = [C.POINTER(OrcParams), _P, _P, _P, _P, _P]
        L.orc_psi4.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P, _P]
        L.orc_phys_sources_psi4.argtypes = [C.POINTER(OrcParams), _P, _P, C.c_double, _P, _P]
        L.orc_point_hyperbolicity.argtypes = [C.POINTER(OrcParams), _P, _P, _P, _P]
        L.orc_point_system.argtypes = [C.POINTER(OrcParams), _P, _P, _P, _P]
        L.orc_hyperbolicity.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P, _P]
        L.orc_rk4_signal.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P, C.c_double, C.c_int, _P, _P]
        L.orc_rk4_signal.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P)


def params(p) -> OrcParams:
    """From a grf_inputs.Params (or anything with the same attributes)."""
    return OrcParams(p.kappa1, p.kappa2, p.kappa3, p.shift_F, p.eta, p.a0, p.b0, p.lam, p.g2,
                     p.sigma_ko, p.min_chi, p.min_lapse, int(p.beta_kind), int(p.enforce_algebraic),
                     int(getattr(p, "decoupled", 0)), int(getattr(p, "advection", 0)),
                     float(getattr(p, "beta_kappa", 1.0)), float(getattr(p, "g3", 0.0)))


def box(b) -> OrcBox:
    return OrcBox(b.nx, b.ny, b.nz, b.ng, b.dx, b.x0, b.y0, b.z0, int(b.bc), 0)


def set_threads(n):
    os.environ["OMP_NUM_THREADS"] = str(n)


def point_rhs(p, v, d1, d2):
    """Pointwise RHS (no dissipation). v[27], d1[27,3], d2[27,6] -> (rhs[27], diag[64], status)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    d1 = np.ascontiguousarray(d1, dtype=np.float64)
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    rhs = np.zeros(27)
    diag = np.zeros(64)
    st = lib().orc_point_rhs(C.byref(params(p)), _ptr(v), _ptr(d1), _ptr(d2), _ptr(rhs), _ptr(diag))
    return rhs, diag, st


def point_rhs_adv(p, v, d1, d2, adv):
    """As point_rhs with the 27 advection terms beta^k d_k u given."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    d1 = np.ascontiguousarray(d1, dtype=np.float64)
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    adv = np.ascontiguousarray(adv, dtype=np.float64)
    rhs = np.zeros(27)
    diag = np.zeros(64)
    st = lib().orc_point_rhs_adv(C.byref(params(p)), _ptr(v), _ptr(d1), _ptr(d2), _ptr(adv), _ptr(rhs), _ptr(diag))
    return rhs, diag, st


def adv_lopsided(b, s):
    """Lopsided advection terms beta^k d_k u of every field at the interior points: (27, nz, ny, nx)."""
    out = np.zeros((27, b.nz, b.ny, b.nx))
    lib().orc_adv_lopsided(C.byref(box(b)), _ptr(s), _ptr(out))
    return out


def point_constraints(p, v, d1, d2):
    v = np.ascontiguousarray(v, dtype=np.float64)
    d1 = np.ascontiguousarray(d1, dtype=np.float64)
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_point_constraints(C.byref(params(p)), _ptr(v), _ptr(d1), _ptr(d2), _ptr(out))
    return out


def phys_sources(p, phys, u6, w):
    phys = np.ascontiguousarray(phys, dtype=np.float64)
    assert phys.size == 120
    u6 = np.ascontiguousarray(u6, dtype=np.float64)
    out = np.zeros(19)
    lib().orc_phys_sources(C.byref(params(p)), _ptr(phys), _ptr(u6), float(w), _ptr(out))
    return out


def solve(M, r):
    M = np.ascontiguousarray(M, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = r.size
    x = np.zeros(n)
    st = lib().orc_solve(n, _ptr(M), _ptr(r), _ptr(x))
    return x, st


def fill_ghosts(b, s):
    lib().orc_fill_ghosts(C.byref(box(b)), _ptr(s))
    return s


def derivs(b, s):
    npt = b.npoints
    d1 = np.zeros((27, 3, b.nz, b.ny, b.nx))
    d2 = np.zeros((27, 6, b.nz, b.ny, b.nx))
    lib().orc_derivs(C.byref(box(b)), _ptr(s), _ptr(d1), _ptr(d2))
    return d1, d2


def rhs(b, p, s, with_ko=True):
    out = np.zeros_like(s)
    st = lib().orc_rhs(C.byref(box(b)), C.byref(params(p)), _ptr(s), _ptr(out), int(with_ko))
    if st != 0:
        raise RuntimeError(f"oracle rhs status {st}")
    return out


def ko(b, sigma, s, out=None):
    if out is None:
        out = np.zeros_like(s)
    lib().orc_ko(C.byref(box(b)), float(sigma), _ptr(s), _ptr(out))
    return out


def enforce(b, p, s):
    lib().orc_enforce(C.byref(box(b)), C.byref(params(p)), _ptr(s))
    return s


def rk4(b, p, s, dt, nsteps):
    """Advances s in place by nsteps RK4 steps."""
    st = lib().orc_rk4(C.byref(box(b)), C.byref(params(p)), _ptr(s), float(dt), int(nsteps))
    if st != 0:
        raise RuntimeError(f"oracle rk4 status {st}")
    return s


def constraints(b, p, s):
    out = np.zeros((4, b.nz, b.ny, b.nx))
    lib().orc_constraints(C.byref(box(b)), C.byref(params(p)), _ptr(s), _ptr(out))
    return out


def point_energy(p, v, d1, d2):
    """8 pi rho of the X, g2 X^2 and Gauss-Bonnet terms at one point (3 doubles)."""
    out = np.zeros(3)
    lib().orc_point_energy(C.byref(params(p)), _ptr(np.ascontiguousarray(v, dtype=np.float64)),
                           _ptr(np.ascontiguousarray(d1, dtype=np.float64)),
                           _ptr(np.ascontiguousarray(d2, dtype=np.float64)), _ptr(out))
    return out


def energy_densities(b, p, s):
    """8 pi rho of the three scalar terms at the interior points: array (3, nz, ny, nx)."""
    out = np.zeros((3, b.nz, b.ny, b.nx))
    lib().orc_energy_densities(C.byref(box(b)), C.byref(params(p)), _ptr(s), _ptr(out))
    return out


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def sylm(s, l, m, theta, phi):
    re, im = C.c_double(), C.c_double()
    lib().orc_sylm(s, l, m, float(theta), float(phi), C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def extract_modes(b, f_re, f_im, spin, radius, centre, ntheta, nphi, lmax):
    """Modes a_lm (complex array indexed l^2 + l + m) of the single ghosted field f_re (+ i f_im)
    on the sphere of the given radius and centre."""
    f_re = np.ascontiguousarray(f_re, dtype=np.float64)
    fi = None if f_im is None else np.ascontiguousarray(f_im, dtype=np.float64)
    out = np.zeros(2 * (lmax + 1) ** 2)
    st = lib().orc_extract_modes(C.byref(box(b)), _ptr(f_re), None if fi is None else _ptr(fi), int(spin),
                                 float(radius), *map(float, centre), int(ntheta), int(nphi), int(lmax), _ptr(out))
    if st != 0:
        raise ValueError("sphere stencil leaves the box")
    return out[0::2] + 1j * out[1::2]


def interp(b, f, xyz):
    """4-point Lagrange interpolant of the single ghosted field f at the points xyz (n, 3)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = np.zeros(xyz.shape[0])
    lib().orc_interp(C.byref(box(b)), _ptr(f), xyz.shape[0], _ptr(xyz), _ptr(out))
    return out


def point_psi4(p, v, d1, d2, xyz):
    """Psi_4 (complex) at one point with the triad about the origin at coordinates xyz."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    d1 = np.ascontiguousarray(d1, dtype=np.float64)
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = np.zeros(2)
    lib().orc_point_psi4(C.byref(params(p)), _ptr(v), _ptr(d1), _ptr(d2), _ptr(xyz), _ptr(out))
    return complex(out[0], out[1])


def psi4(b, p, s):
    """Psi_4 at the interior points: complex array (nz, ny, nx)."""
    out = np.zeros((2, b.nz, b.ny, b.nx))
    lib().orc_psi4(C.byref(box(b)), C.byref(params(p)), _ptr(s), _ptr(out))
    return out[0] + 1j * out[1]


def phys_psi4(p, phys, u6, w, xyz):
    phys = np.ascontiguousarray(phys, dtype=np.float64)
    u6 = np.ascontiguousarray(u6, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = np.zeros(21)
    lib().orc_phys_sources_psi4(C.byref(params(p)), _ptr(phys), _ptr(u6), float(w), _ptr(xyz), _ptr(out))
    return complex(out[19], out[20])


def point_hyperbolicity(p, v, d1, d2):
    """(det M of the coupled system, det(g_eff)/det(g), -g_eff^nn, smallest pivot ratio of M) at
    one point."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    d1 = np.ascontiguousarray(d1, dtype=np.float64)
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_point_hyperbolicity(C.byref(params(p)), _ptr(v), _ptr(d1), _ptr(d2), _ptr(out))
    return out


def point_system(p, v, d1, d2):
    """The coupled system's normalised 7 x 7 matrix at one point (rows 0..5: the d_t K_ij rows,
    row 6: the scalar equation over its d_t Pi coefficient)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    d1 = np.ascontiguousarray(d1, dtype=np.float64)
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    out = np.zeros(49)
    lib().orc_point_system(C.byref(params(p)), _ptr(v), _ptr(d1), _ptr(d2), _ptr(out))
    return out.reshape(7, 7)


def hyperbolicity(b, p, s):
    """The four hyperbolicity diagnostics at every interior point: [4, nz, ny, nx]."""
    out = np.zeros((4, b.nz, b.ny, b.nx))
    lib().orc_hyperbolicity(C.byref(box(b)), C.byref(params(p)), _ptr(np.ascontiguousarray(s)), _ptr(out))
    return out


_tlm = None


def tlm_lib():
    """The tangent-linear builds of the same core (dual numbers and complex step)."""
    global _tlm
    if _tlm is None:
        L = C.CDLL(_build.build_tlm())
        L.orc_tlm_rk4.argtypes = [C.POINTER(OrcBox), C.POINTER(OrcParams), _P, _P, _P, C.c_double, C.c_int, _P, _P,
                                  C.c_int, C.c_double]
        L.orc_tlm_rk4.restype = C.c_int
        _tlm = L
    return _tlm


def rk4_signal(b, p, s, dt, nsteps, sphere):
    """RK4 in place with the sphere-averaged scalar signal L = sum_n dt sum_q w_q phi(c + R xhat_q, t_n);
    sphere = (R, cx, cy, cz). Returns (status, L)."""
    sp = np.ascontiguousarray(sphere, dtype=np.float64)
    L = np.zeros(1)
    st = lib().orc_rk4_signal(C.byref(box(b)), C.byref(params(p)), _ptr(s), dt, nsteps, _ptr(sp), _ptr(L))
    return st, float(L[0])


def tlm_rk4(b, p, s, ds, dparams, dt, nsteps, sphere=None, mode="dual", h=1e-30):
    """Tangent-linear RK4: s (value) and ds (tangent) in place along (ds, dlambda, dg2) =
    (ds, dparams[0], dparams[1]). mode "dual" (dual numbers) or "cs" (complex step with step h).
    Returns (status, L, dL) (L, dL = None without a sphere)."""
    dp = np.ascontiguousarray(dparams, dtype=np.float64)
    L = np.zeros(2)
    sp = None if sphere is None else np.ascontiguousarray(sphere, dtype=np.float64)
    st = tlm_lib().orc_tlm_rk4(C.byref(box(b)), C.byref(params(p)), _ptr(dp), _ptr(s), _ptr(ds), dt, nsteps,
                               None if sp is None else _ptr(sp), _ptr(L), 0 if mode == "dual" else 1, h)
    return (st, None, None) if sp is None else (st, float(L[0]), float(L[1]))
