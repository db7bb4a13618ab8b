// Outer boundaries ("Boundary Conditions": extrapolating and Sommerfeld/radiative).
//
// Extrapolating boxes refill every ghost by linear extrapolation along one axis,
//   u(last + m) = u(last) + m (u(last) - u(last - 1)),  m = 1 .. ng,
// axis by axis (x-ghosts on rows of interior y and z, then y-ghosts on rows of any x and interior
// z, then z-ghosts on rows of any x and y), so edges and corners extrapolate values already set.
// The roundings are pinned (no fused multiply-add), which makes the fill bit-exact against a plain
// evaluation of the formula.
//
// Sommerfeld boxes evolve every ghost point (behind mirror planes at the low faces: every ghost
// beyond a high face with no coordinate below the box; the rest are mirror images) with
//   d_t u = - (u - u_inf) / r - (x^i / r) d_i u,   r = |x| (the radiation centre is the origin),
// u_inf the flat values (chi = h_11 = h_22 = h_33 = lapse = 1, the rest 0), wave speed 1. Along an
// axis on which the point lies beyond the interior, d_i is the 2nd-order one-sided difference
// pointing into the box; along the others the centred 2nd-order difference. At r = 0 the right
// side is 0. The condition holds on outer faces (x^i / r pointing out of the box), where the
// one-sided differences are upwind.
#include "grf_kernels.cuh"
#include "grf_launch.h"
#include "grf_shell.cuh"

namespace grf {

// One thread per (line, field): the ghosts at both ends of a line along axis `ax`.
__global__ void extrapolate_fill_kernel(Geom g, double* __restrict__ s, int ax) {
    const int c1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int c2 = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z;
    const int n[3] = {g.nx, g.ny, g.nz};
    const int N[3] = {g.NX, g.NY, g.NZ};
    const int ng = g.ng;
    // transverse axes (a1, a2): full range where an earlier axis has filled them, else interior
    const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
    const int lo1 = a1 < ax ? 0 : ng, n1 = a1 < ax ? N[a1] : n[a1];
    const int lo2 = a2 < ax ? 0 : ng, n2 = a2 < ax ? N[a2] : n[a2];
    if (c1 >= n1 || c2 >= n2) return;
    int ijk[3];
    ijk[a1] = lo1 + c1;
    ijk[a2] = lo2 + c2;
    ijk[ax] = 0;
    const long long st[3] = {1, g.pitch, g.plane};
    double* u = s + (long long)f * g.fstride + gidx(g, ijk[0], ijk[1], ijk[2]);
    const long long sa = st[ax];
    const int lo = ng, hi = ng + n[ax] - 1;
    const double ah = u[hi * sa], bh = u[(hi - 1) * sa];
    const double al = u[lo * sa], bl = u[(lo + 1) * sa];
    const double dh = __dsub_rn(ah, bh), dl = __dsub_rn(al, bl);
    for (int m = 1; m <= ng; ++m) {
        u[(hi + m) * sa] = __dadd_rn(ah, __dmul_rn((double)m, dh));
        u[(lo - m) * sa] = __dadd_rn(al, __dmul_rn((double)m, dl));
    }
}

__device__ __forceinline__ double u_inf(int f) {
    return (f == F_CHI || f == F_H + 0 || f == F_H + 3 || f == F_H + 5 || f == F_LAPSE) ? 1.0 : 0.0;
}

// Geometry of a ghost point for the radiative condition: its coordinates times 1/r, 1/r, and
// per axis whether the point lies beyond the low (-1) or high (+1) face, or inside (0).
struct SommerfeldPoint {
    double xr[3];  // x^i / r
    double ir;     // 1 / r (0 at r = 0: the right side is then 0)
    int side[3];
};

__device__ __forceinline__ SommerfeldPoint sommerfeld_geometry(const Geom& g, int i, int j, int k, double x0, double y0,
                                                               double z0) {
    SommerfeldPoint q;
    const int idx[3] = {i, j, k};
    const int n[3] = {g.nx, g.ny, g.nz};
    const double x[3] = {x0 + (i - g.ng) * g.dx, y0 + (j - g.ng) * g.dx, z0 + (k - g.ng) * g.dx};
    const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    q.ir = r == 0.0 ? 0.0 : 1.0 / r;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        q.xr[d] = x[d] * q.ir;
        q.side[d] = idx[d] >= g.ng + n[d] ? 1 : (idx[d] < g.ng ? -1 : 0);
    }
    return q;
}

// Radiative right-hand side of field f at offset p of u:
//   -(u - u_inf) / r - sum_d (x^d / r) d_d u
__device__ __forceinline__ double sommerfeld_rhs(const Geom& g, const SommerfeldPoint& q, const double* __restrict__ u,
                                                 long long p, int f) {
    const long long st[3] = {1, g.pitch, g.plane};
    const double u0 = u[p];
    const double i2dx = 1.0 / (2.0 * g.dx);
    double adv = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double du;
        if (q.side[d] > 0) du = (3.0 * u0 - 4.0 * u[p - st[d]] + u[p - 2 * st[d]]) * i2dx;
        else if (q.side[d] < 0) du = (-3.0 * u0 + 4.0 * u[p + st[d]] - u[p + 2 * st[d]]) * i2dx;
        else du = (u[p + st[d]] - u[p - st[d]]) * i2dx;
        adv = fma(q.xr[d], du, adv);
    }
    return -fma(u0 - u_inf(f), q.ir, adv);
}

// The evolved ghost points of a Sommerfeld box (the shell from L: 0 for every ghost, ng behind
// mirror planes), one thread per point (all 27 fields). STAGE < 0: the right-hand side is written
// to `out`; STAGE 0..3: the RK4 stage update of a (as the interior stage kernels, without
// dissipation or enforcement).
template <int STAGE>
__global__ void __launch_bounds__(256) sommerfeld_kernel(Geom g, StageArgs a, double* __restrict__ out, double x0,
                                                         double y0, double z0, int L) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= shell_count(g, L)) return;
    int i, j, k;
    shell_point(g, L, t, i, j, k);
    const SommerfeldPoint q = sommerfeld_geometry(g, i, j, k, x0, y0, z0);
    const long long p = gidx(g, i, j, k);
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        const long long fo = (long long)f * g.fstride;
        const double* src = a.src + fo;
        const double kf = sommerfeld_rhs(g, q, src, p, f);
        if (STAGE < 0) {
            out[fo + p] = kf;
            continue;
        }
        const double unf = (STAGE == 0) ? src[p] : a.un[fo + p];
        a.dst[fo + p] = rk4_value<STAGE < 0 ? 0 : STAGE>(a, fo + p, kf, unf);
    }
}

void launch_extrapolate(const Geom& g, double* s, cudaStream_t st) {
    const dim3 blk(32, 8, 1);
    for (int ax = 0; ax < 3; ++ax) {
        const int n1 = ax == 0 ? g.ny : g.NX;                   // a1 = y (ax 0) or x
        const int n2 = ax == 0 ? g.nz : (ax == 1 ? g.nz : g.NY);  // a2 = z (ax 0, 1) or y
        const dim3 grd((n1 + 31) / 32, (n2 + 7) / 8, NFIELDS);
        extrapolate_fill_kernel<<<grd, blk, 0, st>>>(g, s, ax);
    }
}

void launch_sommerfeld(int stage, const Geom& g, const StageArgs& a, double* out, double x0, double y0, double z0,
                       cudaStream_t st) {
    const int L = g.reflect ? g.ng : 0;  // behind mirror planes only the high-face shell is evolved
    const dim3 blk(256, 1, 1), grd((unsigned)((shell_count(g, L) + 255) / 256), 1, 1);
    switch (stage) {
        case -1: sommerfeld_kernel<-1><<<grd, blk, 0, st>>>(g, a, out, x0, y0, z0, L); break;
        case 0: sommerfeld_kernel<0><<<grd, blk, 0, st>>>(g, a, out, x0, y0, z0, L); break;
        case 1: sommerfeld_kernel<1><<<grd, blk, 0, st>>>(g, a, out, x0, y0, z0, L); break;
        case 2: sommerfeld_kernel<2><<<grd, blk, 0, st>>>(g, a, out, x0, y0, z0, L); break;
        default: sommerfeld_kernel<3><<<grd, blk, 0, st>>>(g, a, out, x0, y0, z0, L); break;
    }
}

}  // namespace grf
