"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no arithmetic of the evolution method: it only builds initial states
(analytic puncture metrics and scalar profiles on a cell-centred grid), draws the seeded
random parameters of the workloads, and describes the box/parameter dictionaries that
both sides translate into their own structures.

State layout (the C-ABI layout, also used by the oracle): float64 array of shape
``(27, nz + 2*ng, ny + 2*ng, nx + 2*ng)``, field-major, x fastest. Grid point with
ghosted index (i, j, k) sits at ``x = x0 + (i - ng)*dx`` (likewise y, z), where x0 is the
coordinate of interior point 0. Field order (27 fields):

    0 chi | 1-6 h11 h12 h13 h22 h23 h33 | 7 K | 8-13 A11 A12 A13 A22 A23 A33 | 14 Theta |
    15-17 Gamma^1..3 | 18 lapse | 19-21 shift^1..3 | 22-24 B^1..3 | 25 phi | 26 Pi
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

NFIELDS = 27
NG = 3
FIELD_NAMES = ["chi", "h11", "h12", "h13", "h22", "h23", "h33", "K",
               "A11", "A12", "A13", "A22", "A23", "A33", "Theta",
               "Gamma1", "Gamma2", "Gamma3", "lapse", "shift1", "shift2", "shift3",
               "B1", "B2", "B3", "phi", "Pi"]
IDX = {n: i for i, n in enumerate(FIELD_NAMES)}

BC_PERIODIC = 0
BC_FROZEN = 1
BC_REFLECT_LOW = 2   # mirror planes half a cell below the first point of the three low faces
BC_EXTRAPOLATE = 3   # ghosts refilled by linear extrapolation from the interior, axis by axis
BC_SOMMERFELD = 4    # ghosts evolved by the radiative (Sommerfeld) condition
BC_REFLECT_LOW_SOMMERFELD = 5  # mirror planes at the low faces, Sommerfeld at the high faces
BETA_LINEAR = 0      # beta(phi) = lambda * phi
BETA_QUADRATIC = 1   # beta(phi) = lambda * phi^2 / 2
BETA_EXPONENTIAL = 2  # beta(phi) = lambda / (2 kappa) * (1 - exp(-kappa phi^2))


@dataclass
class Box:
    nx: int
    ny: int
    nz: int
    dx: float
    x0: float
    y0: float
    z0: float
    bc: int = BC_PERIODIC
    ng: int = NG

    @property
    def shape(self):
        return (NFIELDS, self.nz + 2 * self.ng, self.ny + 2 * self.ng, self.nx + 2 * self.ng)

    @property
    def npoints(self):
        return self.nx * self.ny * self.nz

    def coords(self):
        """Coordinate arrays (3D, ghosted) of every grid point."""
        g = self.ng
        x = self.x0 + (np.arange(self.nx + 2 * g) - g) * self.dx
        y = self.y0 + (np.arange(self.ny + 2 * g) - g) * self.dx
        z = self.z0 + (np.arange(self.nz + 2 * g) - g) * self.dx
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X, Y, Z

    def interior(self, a):
        g = self.ng
        return a[..., g:g + self.nz, g:g + self.ny, g:g + self.nx]


def cube_box(n, lo, hi, bc=BC_PERIODIC):
    """Cell-centred box of n^3 interior points covering [lo, hi]^3."""
    dx = (hi - lo) / n
    c = lo + 0.5 * dx
    return Box(n, n, n, dx, c, c, c, bc)


@dataclass
class Params:
    kappa1: float = 0.1
    kappa2: float = 0.0
    kappa3: float = 1.0
    shift_F: float = 0.75
    eta: float = 1.0
    a0: float = 0.2
    b0: float = 0.4
    beta_kind: int = BETA_LINEAR
    lam: float = 0.01
    g2: float = 0.01
    sigma_ko: float = 0.3
    min_chi: float = 1e-4
    min_lapse: float = 1e-4
    enforce_algebraic: int = 1
    decoupled: int = 0          # 1: 4dST without backreaction (metric evolves by vacuum CCZ4)
    advection: int = 0          # 0: centred advection derivatives, 1: lopsided (upwind-biased)
    beta_kappa: float = 1.0     # kappa of the exponential coupling (beta_kind = BETA_EXPONENTIAL)
    g3: float = 0.0             # cubic Horndeski coupling (the action's g3 X box(phi) term)

    def to_dict(self):
        return asdict(self)


# ---------------------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood 2014): the one documented generator for all seeded draws.
# ---------------------------------------------------------------------------------------
class SplitMix64:
    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def choice(self, seq):
        return seq[self.next_u64() % len(seq)]


# ---------------------------------------------------------------------------------------
# Initial data (analytic; evaluated on every grid point, ghosts included)
# ---------------------------------------------------------------------------------------
def _empty(box):
    return np.zeros(box.shape, dtype=np.float64)


def flat_state(box):
    """Minkowski slice, unit lapse, zero shift, zero scalar."""
    s = _empty(box)
    s[IDX["chi"]] = 1.0
    for n in ("h11", "h22", "h33"):
        s[IDX[n]] = 1.0
    s[IDX["lapse"]] = 1.0
    return s


def conformally_flat_puncture(box, psi, phi, Pi=None):
    """chi = psi^-4, h = delta, K = A = Theta = Gamma = 0, lapse = chi^(1/2), shift = B = 0."""
    s = flat_state(box)
    chi = psi ** -4
    s[IDX["chi"]] = chi
    s[IDX["lapse"]] = np.sqrt(chi)
    s[IDX["phi"]] = phi
    if Pi is not None:
        s[IDX["Pi"]] = Pi
    return s


def single_puncture(box, M=1.0, amp=1e-3, r0=2.0, width=1.0, centre=(0.0, 0.0, 0.0)):
    """Schwarzschild puncture in isotropic coordinates plus phi = amp*exp(-(r-r0)^2/width^2)."""
    X, Y, Z = box.coords()
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    psi = 1.0 + M / (2.0 * r)
    phi = amp * np.exp(-((r - r0) ** 2) / width ** 2)
    return conformally_flat_puncture(box, psi, phi)


def gaussian_bumps(seed, n_bumps, lo, hi):
    """Seeded parameters of a sum of Gaussians: centres (uniform in [lo,hi]^3),
    widths U[1,3], amplitudes 1e-2*U[-1,1]; drawn in that order."""
    rng = SplitMix64(seed)
    centres = [[rng.uniform(lo, hi) for _ in range(3)] for _ in range(n_bumps)]
    widths = [rng.uniform(1.0, 3.0) for _ in range(n_bumps)]
    amps = [1e-2 * rng.uniform(-1.0, 1.0) for _ in range(n_bumps)]
    return centres, widths, amps


def mirror_symmetric_state(box, M=1.0, amp=0.05, eps=1e-2):
    """Puncture at the origin with a scalar shell, plus small smooth fields with the parity of
    each component under x_d -> -x_d (so that the state is symmetric under all three
    reflections): K ~ exp(-r^2/8), A_ij ~ (x_i x_j - delta_ij r^2/3) exp(-r^2/8) (trace-free in
    the flat conformal metric), shift^i, B^i and Gamma^i ~ x^i exp(-r^2/8), Pi ~ exp(-r^2/8)."""
    s = single_puncture(box, M=M, amp=amp)
    X, Y, Z = box.coords()
    xs = (X, Y, Z)
    e = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 8.0)
    r2 = X ** 2 + Y ** 2 + Z ** 2
    s[IDX["K"]] = eps * e
    for n, (a, b) in zip(("A11", "A12", "A13", "A22", "A23", "A33"),
                         ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        s[IDX[n]] = 0.5 * eps * (xs[a] * xs[b] - (r2 / 3.0 if a == b else 0.0)) * e
    for d, c in enumerate("123"):
        s[IDX["shift" + c]] = eps * xs[d] * e
        s[IDX["B" + c]] = 0.5 * eps * xs[d] * e
        s[IDX["Gamma" + c]] = 0.3 * eps * xs[d] * e
    s[IDX["Pi"]] = 0.5 * eps * e
    return s


def brill_lindquist_pair(box, m1=0.5, m2=0.5, sep=6.0, seed=0, n_bumps=8, lo=-16.0, hi=16.0):
    """Brill-Lindquist pair on the z axis at +-sep/2 plus a seeded sum of Gaussians for phi."""
    X, Y, Z = box.coords()
    r1 = np.sqrt(X ** 2 + Y ** 2 + (Z - sep / 2) ** 2)
    r2 = np.sqrt(X ** 2 + Y ** 2 + (Z + sep / 2) ** 2)
    psi = 1.0 + m1 / (2 * r1) + m2 / (2 * r2)
    centres, widths, amps = gaussian_bumps(seed, n_bumps, lo, hi)
    phi = np.zeros_like(X)
    for c, w, a in zip(centres, widths, amps):
        phi += a * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / w ** 2)
    return conformally_flat_puncture(box, psi, phi)


def scalar_plane_wave(box, amp, kvec, t=0.0):
    """Flat space with phi = amp*sin(k.x - |k| t), Pi = d_t phi = -amp |k| cos(k.x - |k| t)."""
    s = flat_state(box)
    X, Y, Z = box.coords()
    kn = math.sqrt(sum(k * k for k in kvec))
    ph = kvec[0] * X + kvec[1] * Y + kvec[2] * Z - kn * t
    s[IDX["phi"]] = amp * np.sin(ph)
    s[IDX["Pi"]] = -amp * kn * np.cos(ph)
    return s


def random_perturbed_state(box, seed, base=None, eps=1e-2):
    """A smooth, generic state: base (flat by default) plus seeded low-mode sinusoids in every
    field, so that every term of the equations is exercised (used by parity tests)."""
    s = flat_state(box) if base is None else base.copy()
    rng = SplitMix64(seed)
    X, Y, Z = box.coords()
    L = (box.nx * box.dx, box.ny * box.dx, box.nz * box.dx)
    for f in range(NFIELDS):
        for _ in range(2):
            kx = 2 * math.pi * rng.choice([1, 2]) / L[0]
            ky = 2 * math.pi * rng.choice([1, 2]) / L[1]
            kz = 2 * math.pi * rng.choice([1, 2]) / L[2]
            ph = rng.uniform(0, 2 * math.pi)
            a = eps * rng.uniform(-1, 1)
            s[f] += a * np.sin(kx * X + ph) * np.cos(ky * Y - ph) * np.sin(kz * Z + 0.5 * ph)
    return s


# ---------------------------------------------------------------------------------------
# Workload descriptions
# ---------------------------------------------------------------------------------------
def config_single_puncture_32():
    """32^3 interior on [-4,4]^3 (dx = 0.25), periodic, single puncture M=1 at the origin
    (cell-centred grid: the puncture sits half a cell from the nearest points on every
    axis), phi = 1e-3 exp(-(r-2)^2), beta = lambda*phi, lambda = g2 = 0.01, 10 steps."""
    box = cube_box(32, -4.0, 4.0)
    params = Params(beta_kind=BETA_LINEAR, lam=0.01, g2=0.01)
    return dict(name="single_puncture_32", box=box, params=params, dt=0.25 * box.dx, nsteps=10,
                make_state=lambda b=box: single_puncture(b))


def config_bl_pair_256(n=256):
    """256^3 interior on [-16,16]^3 (dx = 0.125), periodic, Brill-Lindquist pair m=0.5 each at
    z = +-3, phi = seeded sum of 8 Gaussians, beta = lambda*phi^2/2, lambda = 0.05, g2 = 0.01,
    100 steps at dt = 0.25*dx."""
    box = cube_box(n, -16.0, 16.0)
    params = Params(beta_kind=BETA_QUADRATIC, lam=0.05, g2=0.01)
    return dict(name=f"bl_pair_{n}", box=box, params=params, dt=0.25 * box.dx, nsteps=100,
                make_state=lambda b=box: brill_lindquist_pair(b))


def brill_lindquist_pair_symmetric(box, m1=0.5, m2=0.5, sep=6.0, amp=1e-2, r0=4.0, width=2.0):
    """The Brill-Lindquist pair on the z axis at +-sep/2 with equal masses, which is symmetric under
    the x, y and z reflections, plus a spherical scalar shell phi = amp exp(-(r - r0)^2 / width^2)
    that shares the symmetry."""
    X, Y, Z = box.coords()
    r1 = np.sqrt(X ** 2 + Y ** 2 + (Z - sep / 2) ** 2)
    r2 = np.sqrt(X ** 2 + Y ** 2 + (Z + sep / 2) ** 2)
    psi = 1.0 + m1 / (2 * r1) + m2 / (2 * r2)
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    return conformally_flat_puncture(box, psi, amp * np.exp(-((r - r0) ** 2) / width ** 2))


def config_bl_pair_octant(n=128):
    """The positive octant [0, 16]^3 of the 256^3 Brill-Lindquist domain (dx = 0.125), n^3 interior
    points, with mirror planes at the three low faces and the analytic data in the high-face
    ghosts; the scalar is the symmetric shell of brill_lindquist_pair_symmetric. It evolves the
    symmetric full-box problem on 1/8 of its points."""
    dx = 16.0 / n
    box = Box(n, n, n, dx, 0.5 * dx, 0.5 * dx, 0.5 * dx, bc=BC_REFLECT_LOW)
    params = Params(beta_kind=BETA_QUADRATIC, lam=0.05, g2=0.01)
    return dict(name=f"bl_pair_octant_{n}", box=box, params=params, dt=0.25 * dx, nsteps=100,
                make_state=lambda b=box: brill_lindquist_pair_symmetric(b))


def coupling_sweep(n_instances=32, seed=0):
    """Seeded couplings of the 32-instance sweep: lambda ~ U[0,0.1], g2 ~ U[0,0.05]."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n_instances):
        lam = rng.uniform(0.0, 0.1)
        g2 = rng.uniform(0.0, 0.05)
        out.append((lam, g2))
    return out


def amr_like_boxes(n_boxes=96, seed=0, edges=(16, 24, 32, 48, 64), levels=5, centre_range=4.0):
    """Seeded set of uneven AMR-like boxes: edge n drawn from `edges`, a cube or a 2:1 slab
    (n, n, n/2) with the short axis drawn, refinement level l in 0..levels-1 (dx = 2^-l), centre
    uniform in [-centre_range, centre_range]^3. Lower corners sit on multiples of dx, points at
    (k + 1/2) dx, ghosts frozen (filled from the analytic data). Draw order per box: edge,
    shape, short axis, level, centre (x, y, z)."""
    rng = SplitMix64(seed)
    boxes = []
    for _ in range(n_boxes):
        n = rng.choice(list(edges))
        slab = rng.next_u64() % 2 == 1
        axis = rng.next_u64() % 3
        level = rng.next_u64() % levels
        c = [rng.uniform(-centre_range, centre_range) for _ in range(3)]
        dims = [n, n, n]
        if slab:
            dims[axis] = n // 2
        dx = 2.0 ** (-level)
        x0 = [math.floor((c[a] - 0.5 * dims[a] * dx) / dx) * dx + 0.5 * dx for a in range(3)]
        boxes.append(Box(dims[0], dims[1], dims[2], dx, x0[0], x0[1], x0[2], bc=BC_FROZEN))
    return boxes


def coupling_sweep_boxes(n_instances=32, n=64, lo=-8.0, hi=8.0, seed=0):
    """n_instances periodic n^3 boxes on [lo, hi]^3 with the single-puncture data and seeded
    couplings (lambda ~ U[0, 0.1], g2 ~ U[0, 0.05]). Returns (boxes, params list)."""
    boxes = [cube_box(n, lo, hi) for _ in range(n_instances)]
    params = [Params(beta_kind=BETA_LINEAR, lam=lam, g2=g2) for lam, g2 in coupling_sweep(n_instances, seed)]
    return boxes, params
