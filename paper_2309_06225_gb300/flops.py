"""FP64 operation counts of the kernels' formulation (host build of the kernel source).

The pointwise part (RHS + 7x7 solve) is counted by running the kernel's own source with an
operation-counting scalar (libgrf_flops.so). The stencil gather, KO dissipation and stage
update are fixed expressions in grf_kernels.cuh and are counted here from their code:
  fd1  (u-2 - u+2) + 8 (u+1 - u-1), * 1/(12dx)            : 2 add, 1 fma, 1 mul
  fd2  16 (u+1 + u-1) - (u+2 + u-2) - 30 u0, * 1/(12dx^2)  : 2 fma, 1 mul (the two pair sums
       are shared with the KO sum of the same field)
  d_x d_y, d_x d_z, d_y d_z: the first-derivative stencil applied to the rounded first
       derivatives of the four neighbours (neighbouring lanes of the warp for x, the block's
       shared rows for y)                                              : 2 add, 1 fma, 1 mul
  halos: 3 first derivatives per point for the warp's row ends (the y / z derivatives at the 4
       points past the ends of a 32-point row, 12 fields) and 12 per point for the block's 4 halo
       rows of z-derivatives                                          : 15 x (2 add, 1 fma, 1 mul)
  ko6  3 x (3 pair sums + 3 accumulations) - 3, 3 fma; + ko*value into the RHS: 15 add, 4 fma
  stage update (per field): 1-2 fma (+1 add on the last stage)
Counting convention: add/sub/mul = 1 flop, fma = 2, division = 1.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

N_D1_FIELDS, N_D2_FIELDS, NFIELDS = 24, 12, 27


def _lib():
    L = C.CDLL(_build.build_flops())
    P = C.POINTER(C.c_double)
    L.grf_count_point_ops.argtypes = [C.c_void_p, P, P, P, C.POINTER(C.c_longlong)]
    L.grf_host_point_rhs.argtypes = [C.c_void_p, P, P, P, P, P]
    L.grf_host_point_psi4.argtypes = [C.c_void_p, P, P, P, P, P]
    L.grf_host_point_hyp.argtypes = [C.c_void_p, P, P, P, P]
    return L


def point_ops(params, v=None, d1=None, d2=None):
    """Per-section operation counts [sections][add, mul, fma, div, cmp, waste] of one
    pointwise RHS evaluation (generic point data by default)."""
    rng = np.random.default_rng(0)
    v = rng.uniform(0.5, 1.0, 27) if v is None else np.ascontiguousarray(v, dtype=np.float64)
    d1 = rng.normal(size=72) * 0.1 if d1 is None else np.ascontiguousarray(d1, dtype=np.float64)
    d2 = rng.normal(size=72) * 0.1 if d2 is None else np.ascontiguousarray(d2, dtype=np.float64)
    out = np.zeros((24, 6), dtype=np.int64)
    P = C.POINTER(C.c_double)
    _lib().grf_count_point_ops(C.byref(params), v.ctypes.data_as(P), d1.ctypes.data_as(P), d2.ctypes.data_as(P),
                               out.ctypes.data_as(C.POINTER(C.c_longlong)))
    return out


def stencil_ops():
    """(add, mul, fma) of the gather + KO + stage update per point and stage (mean over stages)."""
    fd1 = np.array([2, 1, 1])      # add, mul, fma
    fd2 = np.array([0, 1, 2])
    mix = np.array([2, 1, 1])
    gather = N_D1_FIELDS * 3 * fd1 + N_D2_FIELDS * (3 * fd2 + 3 * mix) + 15 * fd1
    ko = NFIELDS * np.array([15, 0, 4])
    update = NFIELDS * np.array([0.25, 0, 1.75])   # stages: 1, 2, 2, 2 fma (+1 add on the last)
    return gather + ko + update


def flops_per_point_rhs(params):
    """Algorithmic FP64 flops per interior point of one RHS evaluation with dissipation
    (grf_rhs; the constraints kernel does the same work): the stage without its update."""
    ops = point_ops(params).sum(axis=0)
    add, mul, fma, div = ops[0], ops[1], ops[2], ops[3]
    s = stencil_ops() - NFIELDS * np.array([0.25, 0, 1.75])
    return float(add + mul + 2 * fma + div + s[0] + s[1] + 2 * s[2])


def flops_per_point_stage(params):
    """Algorithmic FP64 flops per interior point per RK4 stage kernel."""
    ops = point_ops(params).sum(axis=0)
    add, mul, fma, div = ops[0], ops[1], ops[2], ops[3]
    s = stencil_ops()
    return float(add + mul + 2 * fma + div + s[0] + s[1] + 2 * s[2])


def host_point_rhs(params, v, d1, d2):
    """The kernel's pointwise RHS evaluated on the host in FP64 (for CPU checks)."""
    P = C.POINTER(C.c_double)
    v = np.ascontiguousarray(v, dtype=np.float64)
    d1 = np.ascontiguousarray(d1, dtype=np.float64)
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    rhs = np.zeros(27)
    extra = np.zeros(4)
    st = _lib().grf_host_point_rhs(C.byref(params), v.ctypes.data_as(P), d1.ctypes.data_as(P), d2.ctypes.data_as(P),
                                   rhs.ctypes.data_as(P), extra.ctypes.data_as(P))
    return rhs, extra, st


def host_point_psi4(params, v, d1, d2, xyz):
    """The kernel's Psi_4 (Riemann blocks on the null tetrad) evaluated on the host in FP64."""
    P = C.POINTER(C.c_double)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (v, d1, d2, xyz)]
    out = np.zeros(2)
    st = _lib().grf_host_point_psi4(C.byref(params), *[a.ctypes.data_as(P) for a in arrs], out.ctypes.data_as(P))
    return complex(out[0], out[1]), st


def host_point_hyp(params, v, d1, d2):
    """The kernel's hyperbolicity diagnostics (det M, det g_eff / det g, -g_eff^nn, smallest pivot
    ratio) on the host."""
    P = C.POINTER(C.c_double)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (v, d1, d2)]
    out = np.zeros(4)
    st = _lib().grf_host_point_hyp(C.byref(params), *[a.ctypes.data_as(P) for a in arrs], out.ctypes.data_as(P))
    return out, st
