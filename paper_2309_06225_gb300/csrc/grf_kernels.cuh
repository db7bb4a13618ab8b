// Grid kernels of the GB300 path: stencil gather, fused RK4 stage, RHS, KO dissipation,
// periodic ghost fill, constraints and their norms.
#pragma once

#include <cuda_runtime.h>

#include "grf_point.cuh"

// Loads of stencil sources. By default the read-only, non-coherent path (__ldg): every kernel
// that reads a state through these helpers leaves it unwritten for the rest of its launch. A
// kernel that reads, in one launch, buffers that other blocks wrote earlier in the same launch
// (the persistent batched kernel, across its grid barriers) defines GRF_COHERENT_LOADS before
// including this header: the loads then go through L2 only (__ldcg), which is coherent.
#ifdef GRF_COHERENT_LOADS
#define GRF_LDG(p) __ldcg(p)
#else
#define GRF_LDG(p) __ldg(p)
#endif

namespace grf {

struct Geom {
    int nx, ny, nz;          // interior points
    int NX, NY, NZ;          // ghosted extents (n + 2 ng)
    long long pitch;         // doubles per x row
    long long plane;         // pitch * NY
    long long fstride;       // plane * NZ
    double dx;
    int periodic;            // ghosts are periodic images (written by the owner of each value)
    int reflect;             // the three low faces are mirror planes (images written by the owner)
    int ng;                  // ghost layers: 3 (4th-order scheme) or 4 (6th-order scheme)
};

constexpr int NG = 3;        // ghost layers of the 4th-order kernels (those of this header)

__device__ __forceinline__ long long gidx(const Geom& g, int i, int j, int k) {  // ghosted indices
    return (long long)k * g.plane + (long long)j * g.pitch + i;
}

// Centred 4th-order first and second derivatives at ghosted offset p.
// first: (u_-2 - 8 u_-1 + 8 u_+1 - u_+2)/(12 dx) ; second: (-u_-2 + 16 u_-1 - 30 u_0 + 16 u_+1 - u_+2)/(12 dx^2)
// Mixed derivatives (tensor product of the first-derivative weights) are formed below as the
// first-derivative stencil applied to rounded first derivatives.
__device__ __forceinline__ double fd1(const double* __restrict__ u, long long p, long long s, double i12) {
    return ((GRF_LDG(u + p - 2 * s) - GRF_LDG(u + p + 2 * s)) + 8.0 * (GRF_LDG(u + p + s) - GRF_LDG(u + p - s))) * i12;
}
__device__ __forceinline__ double fd2(const double* __restrict__ u, long long p, long long s, double u0, double i12s) {
    return (16.0 * (GRF_LDG(u + p + s) + GRF_LDG(u + p - s)) - (GRF_LDG(u + p + 2 * s) + GRF_LDG(u + p - 2 * s)) - 30.0 * u0) * i12s;
}

__device__ __forceinline__ bool has_d2(int f) {
    return f == F_CHI || (f >= F_H && f < F_H + 6) || f == F_LAPSE || (f >= F_SHIFT && f < F_SHIFT + 3) || f == F_PHI;
}

// Field index of d2 slot b (inverse of d2slot).
__host__ __device__ constexpr int d2field(int b) { return b < 7 ? b : (b == 7 ? F_LAPSE : (b < 11 ? b + 11 : F_PHI)); }

// Mixed derivatives d_x d_t u (t = y or z) are the x-stencil applied to the scaled first
// t-derivatives at x-2, x-1, x+1, x+2:  ((D(x-2) - D(x+2)) + 8 (D(x+1) - D(x-1))) / (12 dx),
// D = fd1 along t. Where a warp is one x-row of 32 consecutive points, the four D values come
// from the neighbouring lanes by shuffles (the lanes computed them as their own first
// derivatives), and the 4 points beyond the row ends from a halo computed once per warp.
// Elsewhere each thread evaluates the four D itself. Both give bit-identical results.
struct WarpRow {
    int lane;      // lane = x offset in the row
    int selA, selB;  // halo slot for the x-2 / x+2 (A) and x-1 / x+1 (B) neighbours of end lanes
    double hv[3];  // this lane's share of the halo: 12 d2 slots x {y, z} x 4 points, 3 per lane
};

// Halo of the warp's row: the first t-derivatives (t = y, z) of the 12 fields with second
// derivatives at x0-2, x0-1, x0+32, x0+33 (clamped to the last ghost column; values beyond
// nx+1 are never used by an interior point). Value (b, t, q) lives in lane 8 (b % 4) + 4 t + q,
// register b / 4. Every lane of the warp must call this.
__device__ __forceinline__ void warp_row_halo(const Geom& g, const double* __restrict__ s, int x0, int j, int k,
                                              int lane, WarpRow& wr) {
    const double i12 = 1.0 / (12.0 * g.dx);
    const int q = lane & 3, t = (lane >> 2) & 1, bq = lane >> 3;
    const int hx = min(q < 2 ? x0 - 2 + q : x0 + 30 + q, g.nx + 2);
    const long long ph = gidx(g, hx + NG, j + NG, k + NG);
    const long long sd = t ? g.plane : g.pitch;
#pragma unroll
    for (int r = 0; r < 3; ++r) wr.hv[r] = fd1(s + (long long)d2field(4 * r + bq) * g.fstride, ph, sd, i12);
    wr.lane = lane;
    wr.selA = lane == 0 ? 0 : (lane == 1 ? 1 : (lane == 30 ? 2 : 3));
    wr.selB = lane == 0 ? 1 : 2;
}

// d_x d_t u for d2 slot b from this lane's own D = fd1_t(u) and the neighbours' (warp path).
__device__ __forceinline__ double mixed_x_warp(const WarpRow& wr, int b, int t, double own, double i12) {
    const unsigned full = 0xffffffffu;
    const int base = 8 * (b & 3) + 4 * t;
    const double hA = __shfl_sync(full, wr.hv[b >> 2], base + wr.selA);
    const double hB = __shfl_sync(full, wr.hv[b >> 2], base + wr.selB);
    const double vm2 = __shfl_up_sync(full, own, 2), vm1 = __shfl_up_sync(full, own, 1);
    const double vp1 = __shfl_down_sync(full, own, 1), vp2 = __shfl_down_sync(full, own, 2);
    const double m2 = wr.lane < 2 ? hA : vm2;
    const double m1 = wr.lane < 1 ? hB : vm1;
    const double p1 = wr.lane > 30 ? hB : vp1;
    const double p2 = wr.lane > 29 ? hA : vp2;
    return __dmul_rn((m2 - p2) + 8.0 * (p1 - m1), i12);
}

// d_s d_t u with the four t-derivatives at the s-neighbours evaluated here (s = x or y). The
// scalings are explicitly rounded (__dmul_rn, never fused into a neighbouring add), so the sums
// are those of the shuffle and shared-memory paths, whose neighbour values arrive rounded.
__device__ __forceinline__ double fd1_rounded(const double* __restrict__ u, long long p, long long s, double i12) {
    return __dmul_rn((GRF_LDG(u + p - 2 * s) - GRF_LDG(u + p + 2 * s)) + 8.0 * (GRF_LDG(u + p + s) - GRF_LDG(u + p - s)), i12);
}
__device__ __forceinline__ double mixed_local(const double* __restrict__ u, long long p, long long so, long long t,
                                              double i12) {
    const double m2 = fd1_rounded(u, p - 2 * so, t, i12), m1 = fd1_rounded(u, p - so, t, i12);
    const double p1 = fd1_rounded(u, p + so, t, i12), p2 = fd1_rounded(u, p + 2 * so, t, i12);
    return __dmul_rn((m2 - p2) + 8.0 * (p1 - m1), i12);
}

// d_y d_z in blocks of 32 x 4 threads (every warp one x-row, the 4 warps consecutive y-rows):
// the rounded first z-derivatives of the 12 fields with second derivatives on rows y0-2 .. y0+5
// (row index y - y0 + 2) are shared through shared memory; each warp adds one halo row.
struct YzRows {
    double dz[12][8][32];
};

// Every thread of the block calls this, then __syncthreads(). x, y0 + wy: the thread's point
// (clamped to the last ghost column / row: values there are only read by points outside the
// interior); k: an interior plane.
__device__ __forceinline__ void yz_rows_fill(const Geom& g, const double* __restrict__ s, int x, int y0, int wy,
                                             int k, int lane, YzRows& sh) {
    const double i12 = 1.0 / (12.0 * g.dx);
    const int xc = min(x, g.nx + 2);
    const int yo = min(y0 + wy, g.ny + 2);
    const int yh = min(wy < 2 ? y0 - 2 + wy : y0 + 2 + wy, g.ny + 2);  // rows y0-2, y0-1, y0+4, y0+5
    const int rh = wy < 2 ? wy : wy + 4;
    const long long po = gidx(g, xc + NG, yo + NG, k + NG), ph = gidx(g, xc + NG, yh + NG, k + NG);
#pragma unroll
    for (int b = 0; b < 12; ++b) {
        const double* u = s + (long long)d2field(b) * g.fstride;
        sh.dz[b][wy + 2][lane] = fd1_rounded(u, po, g.plane, i12);
        sh.dz[b][rh][lane] = fd1_rounded(u, ph, g.plane, i12);
    }
}

// Values, first derivatives and second derivatives of all fields at ghosted offset p, and each
// field's Kreiss-Oliger sum (as ko6 below, same order of additions), the pair sums at distances
// 1 and 2 shared with the second derivatives.
//   wr != nullptr: the warp is one x-row; d_x d_y and d_x d_z come from the neighbouring lanes
//                  (every lane of the warp must call this).
//   sh != nullptr: d_y d_z (and the first z-derivatives of the 12 fields with second
//                  derivatives) come from the block's shared rows; wy = the thread's row.
// Every combination gives the same bits.
//   LOP = 1: also the lopsided advection terms adv[f] = sum_d beta^d D_d u_f, D_d the 4th-order
//            stencil on offsets -1..3 biased towards the side beta^d points to (mirrored for
//            beta^d < 0): beta^d D_d u = |beta^d| (-3 b1 - 10 u0 + 18 a1 - 6 a2 + a3) / (12 dx),
//            a_n = u at n points towards that side, b1 = u one point away from it. The points
//            are those the centred and Kreiss-Oliger stencils load anyway.
template <int LOP = 0>
__device__ __forceinline__ void gather(const Geom& g, const double* __restrict__ s, long long p, PointIn& in,
                                       double kos[NFIELDS], const WarpRow* wr, const YzRows* sh, int wy,
                                       double* adv = nullptr) {
    const double i12 = 1.0 / (12.0 * g.dx), i12s = 1.0 / (12.0 * g.dx * g.dx);
    const long long st[3] = {1, g.pitch, g.plane};
    const int lane = threadIdx.x & 31;
    double bet[3] = {0.0, 0.0, 0.0};
    if (LOP) {
#pragma unroll
        for (int d = 0; d < 3; ++d) bet[d] = GRF_LDG(s + (F_SHIFT + d) * g.fstride + p);
    }
#pragma unroll
    for (int f = 0; f < NFIELDS; ++f) {
        const double* u = s + f * g.fstride;
        const double u0 = GRF_LDG(u + p);
        in.v[f] = u0;
        double p1[3], p2[3], d1[3], p3[3], av = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double m1 = GRF_LDG(u + p - st[d]), q1 = GRF_LDG(u + p + st[d]);
            const double m2 = GRF_LDG(u + p - 2 * st[d]), q2 = GRF_LDG(u + p + 2 * st[d]);
            if (LOP) {
                const double m3 = GRF_LDG(u + p - 3 * st[d]), q3 = GRF_LDG(u + p + 3 * st[d]);
                p3[d] = m3 + q3;
                const bool fw = bet[d] >= 0.0;
                const double a1 = fw ? q1 : m1, a2 = fw ? q2 : m2, a3 = fw ? q3 : m3, b1 = fw ? m1 : q1;
                const double x = fma(18.0, a1, fma(-6.0, a2, a3)) - fma(3.0, b1, 10.0 * u0);
                av = fma(fabs(bet[d]), x * i12, av);
            }
            if (d == 2 && has_d2(f)) {  // rounded: shared with the neighbours' d_y d_z
                d1[d] = sh ? sh->dz[d2slot(f)][wy + 2][lane] : __dmul_rn((m2 - q2) + 8.0 * (q1 - m1), i12);
            } else {
                d1[d] = ((m2 - q2) + 8.0 * (q1 - m1)) * i12;
            }
            if (!(f >= F_B && f < F_B + 3)) in.d1[d1slot(f)][d] = d1[d];
            p1[d] = q1 + m1;
            p2[d] = q2 + m2;
        }
        if (has_d2(f)) {
            const int b = d2slot(f);
            in.d2[b][0] = (16.0 * p1[0] - p2[0] - 30.0 * u0) * i12s;
            in.d2[b][1] = wr ? mixed_x_warp(*wr, b, 0, d1[1], i12) : mixed_local(u, p, st[0], st[1], i12);
            in.d2[b][2] = wr ? mixed_x_warp(*wr, b, 1, d1[2], i12) : mixed_local(u, p, st[0], st[2], i12);
            in.d2[b][3] = (16.0 * p1[1] - p2[1] - 30.0 * u0) * i12s;
            if (sh) {
                const double(*r)[32] = sh->dz[b];
                in.d2[b][4] = __dmul_rn((r[wy][lane] - r[wy + 4][lane]) + 8.0 * (r[wy + 3][lane] - r[wy + 1][lane]), i12);
            } else {
                in.d2[b][4] = mixed_local(u, p, st[1], st[2], i12);
            }
            in.d2[b][5] = (16.0 * p1[2] - p2[2] - 30.0 * u0) * i12s;
        }
        if (LOP) adv[f] = av;
        const double t3 = LOP ? (p3[0] + p3[1]) + p3[2]
                              : ((GRF_LDG(u + p - 3 * st[0]) + GRF_LDG(u + p + 3 * st[0])) +
                                 (GRF_LDG(u + p - 3 * st[1]) + GRF_LDG(u + p + 3 * st[1]))) +
                                    (GRF_LDG(u + p - 3 * st[2]) + GRF_LDG(u + p + 3 * st[2]));
        const double t2 = (p2[0] + p2[1]) + p2[2];
        const double t1 = (p1[0] + p1[1]) + p1[2];
        kos[f] = t3 - 6.0 * t2 + 15.0 * t1 - 60.0 * u0;
    }
}

// sum_d (u_-3 - 6 u_-2 + 15 u_-1 - 20 u_0 + 15 u_+1 - 6 u_+2 + u_+3), pair sums added x, y, z
__device__ __forceinline__ double ko6(const double* __restrict__ u, long long p, long long sy, long long sz) {
    const long long st[3] = {1, sy, sz};
    double t[4];
#pragma unroll
    for (int r = 1; r <= 3; ++r)
        t[r] = ((GRF_LDG(u + p - r * st[0]) + GRF_LDG(u + p + r * st[0])) + (GRF_LDG(u + p - r * st[1]) + GRF_LDG(u + p + r * st[1]))) +
               (GRF_LDG(u + p - r * st[2]) + GRF_LDG(u + p + r * st[2]));
    return t[3] - 6.0 * t[2] + 15.0 * t[1] - 60.0 * GRF_LDG(u + p);
}

__device__ __forceinline__ bool interior_thread(const Geom& g, int& i, int& j, int& k) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y * blockDim.y + threadIdx.y;
    k = blockIdx.z * blockDim.z + threadIdx.z;
    return i < g.nx && j < g.ny && k < g.nz;
}

// Parity of field f under the reflections x_d -> -x_d of the axes in `mask` (bit d): -1 when
// the component has an odd number of indices along the reflected axes (the d-components of
// Gamma-hat, shift and B; h_ab and A_ab with exactly one index reflected), +1 otherwise.
__host__ __device__ __forceinline__ double mirror_sign(int f, int mask) {
    int odd = 0;
    if (f >= F_GAM && f < F_GAM + 3) odd = (mask >> (f - F_GAM)) & 1;
    else if (f >= F_SHIFT && f < F_SHIFT + 3) odd = (mask >> (f - F_SHIFT)) & 1;
    else if (f >= F_B && f < F_B + 3) odd = (mask >> (f - F_B)) & 1;
    else if ((f >= F_H && f < F_H + 6) || (f >= F_A && f < F_A + 6)) {
        const int m = (f < F_A) ? f - F_H : f - F_A;  // sym index of (a, b), a <= b
        const int a = m < 3 ? 0 : (m < 5 ? 1 : 2);
        const int b = m < 3 ? m : (m < 5 ? m - 2 : 2);
        odd = ((mask >> a) & 1) ^ ((mask >> b) & 1);
    }
    return odd ? -1.0 : 1.0;
}

// Writes value x of field f for interior point (i,j,k) and to every ghost location that is an
// image of it: periodic images, or for mirror boxes its reflections in the low faces (the
// mirror plane lies half a cell below the first point; ghost NG-1-i mirrors interior i), with
// the component's parity.
template <int NGT = NG>
__device__ __forceinline__ void store_with_images(const Geom& g, double* __restrict__ dst, int f, int i, int j, int k,
                                                  double x) {
    constexpr int NG = NGT;
    double* d = dst + f * g.fstride;
    if (!g.periodic) {
        d[gidx(g, i + NG, j + NG, k + NG)] = x;
        if (g.reflect) {
            const int near = (i < NG ? 1 : 0) | (j < NG ? 2 : 0) | (k < NG ? 4 : 0);
            for (int m = 1; m < 8; ++m) {
                if (m & ~near) continue;
                d[gidx(g, (m & 1) ? NG - 1 - i : i + NG, (m & 2) ? NG - 1 - j : j + NG, (m & 4) ? NG - 1 - k : k + NG)] =
                    mirror_sign(f, m) * x;
            }
        }
        return;
    }
    int xi[3], yi[3], zi[3];
    int nxi = 0, nyi = 0, nzi = 0;
    xi[nxi++] = i + NG;
    if (i < NG) xi[nxi++] = i + NG + g.nx;
    if (i >= g.nx - NG) xi[nxi++] = i + NG - g.nx;
    yi[nyi++] = j + NG;
    if (j < NG) yi[nyi++] = j + NG + g.ny;
    if (j >= g.ny - NG) yi[nyi++] = j + NG - g.ny;
    zi[nzi++] = k + NG;
    if (k < NG) zi[nzi++] = k + NG + g.nz;
    if (k >= g.nz - NG) zi[nzi++] = k + NG - g.nz;
    for (int c = 0; c < nzi; ++c)
        for (int b = 0; b < nyi; ++b)
            for (int a = 0; a < nxi; ++a) d[gidx(g, xi[a], yi[b], zi[c])] = x;
}

// Trace-free A_ij with respect to h_ij, and the chi / lapse floors, on one point's values.
__device__ __forceinline__ void enforce_point(double u[NFIELDS], double min_chi, double min_lapse) {
    double hh[6], hi[6], id;
#pragma unroll
    for (int m = 0; m < 6; ++m) hh[m] = u[F_H + m];
    sym3_inv(hh, hi, id);
    const double tr = hi[0] * u[F_A] + hi[3] * u[F_A + 3] + hi[5] * u[F_A + 5]
                      + 2.0 * (hi[1] * u[F_A + 1] + hi[2] * u[F_A + 2] + hi[4] * u[F_A + 4]);
#pragma unroll
    for (int m = 0; m < 6; ++m) u[F_A + m] -= hh[m] * tr * (1.0 / 3.0);
    u[F_CHI] = fmax(u[F_CHI], min_chi);
    u[F_LAPSE] = fmax(u[F_LAPSE], min_lapse);
}

struct StageArgs {
    const double* src;   // state whose RHS is evaluated (ghosts valid)
    const double* un;    // u_n (pointwise)
    double* acc;         // k1 + 2 k2 + 2 k3 accumulator (pointwise)
    double* dst;         // state written by this stage
    double dt;
    double ko;           // sigma / (64 dx)
    double min_chi, min_lapse;
    int enforce;
    int* status;
    int k0;              // first interior z-plane of the launch (grid.z covers planes k0, k0+1, ...)
    int fold;            // x-points per warp row: 32, or 16 / 8 / 4 for rk4_stage_fold_kernel
};

// Lopsided advection: the ADV terms of point_rhs come from in.adv (filled by the gather).
constexpr int kLopsided = 1;

// RK4 stage arithmetic for one value at offset q (u_1 = u_n + dt/2 k_1, u_2 = u_n + dt/2 k_2,
// u_3 = u_n + dt k_3, u_{n+1} = u_n + dt/6 (k_1 + 2 k_2 + 2 k_3 + k_4)): kf the stage's right-hand
// side, unf = u_n; the accumulator a.acc[q] is read (STAGE > 0) and written (STAGE < 3). Returns
// the stage's output value.
template <int STAGE>
__device__ __forceinline__ double rk4_value(const StageArgs& a, long long q, double kf, double unf) {
    double accf;
    if (STAGE == 0) accf = kf;
    else if (STAGE == 3) accf = a.acc[q] + kf;
    else accf = a.acc[q] + 2.0 * kf;
    if (STAGE < 3) a.acc[q] = accf;
    const double cs = (STAGE == 0 || STAGE == 1) ? 0.5 * a.dt : (STAGE == 2 ? a.dt : a.dt * (1.0 / 6.0));
    return (STAGE == 3) ? fma(cs, accf, unf) : fma(cs, kf, unf);
}

// How a stage's gather takes its mixed derivatives (all modes give the same bits).
enum GatherMode {
    GATHER_LOCAL = 0,  // per thread
    GATHER_WARP = 1,   // warps are x-rows: d_x d_y, d_x d_z by shuffles
    GATHER_BLOCK = 2,  // blocks of 32 x 4 (x-rows stacked in y): also d_y d_z through shared memory
};

// One RK4 stage at one point, fused: gather -> pointwise RHS -> + KO -> stage update ->
// enforcement -> store (with periodic images). STAGE 0..3. In the warp and block modes the
// threads past the interior (i >= nx, and j >= ny in block mode) take part in the gather, at the
// last ghost column / row at most, and then write nothing. sh: the block's rows (block mode,
// already filled and synchronised).
template <int STAGE, int DEC = -1, int LOP = 0, int COUP = 1>
__device__ __forceinline__ void stage_point(const Geom& g, const Coeffs& c, const StageArgs& a, int i, int j, int k,
                                            int mode, const YzRows* sh) {
    const bool live = i < g.nx && j < g.ny;
    const int ic = min(i, g.nx + 2), jc = min(j, g.ny + 2);
    const long long p = gidx(g, ic + NG, jc + NG, k + NG);
    PointIn in;
    double kos[NFIELDS];
    double adv[LOP ? NFIELDS : 1];
    if (mode != GATHER_LOCAL) {
        WarpRow wr;
        const int lane = threadIdx.x & 31;
        warp_row_halo(g, a.src, i - lane, jc, k, lane, wr);
        gather<LOP>(g, a.src, p, in, kos, &wr, mode == GATHER_BLOCK ? sh : nullptr, threadIdx.y, adv);
    } else {
        gather<LOP>(g, a.src, p, in, kos, nullptr, nullptr, 0, adv);
    }
    if (!live) return;
    double r[NFIELDS];
    bool ok = true;
    point_rhs<double, double, DEC, LOP, COUP>(c, in, r, nullptr, ok, adv);
    if (!ok) atomicOr(a.status, 1);
    double out[NFIELDS];
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        const double kf = r[f] + a.ko * kos[f];
        const double unf = (STAGE == 0) ? in.v[f] : a.un[f * g.fstride + p];
        out[f] = rk4_value<STAGE>(a, f * g.fstride + p, kf, unf);
    }
    if (a.enforce) enforce_point(out, a.min_chi, a.min_lapse);
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) store_with_images(g, a.dst, f, i, j, k, out[f]);
}

// Launched with blocks of (32, 4, 1) threads (block gather mode). Planes k0, k0+1, ...
// 3 resident blocks of 128 threads per SM (168 registers a thread): the extra warps hide more
// FP64 dependency latency than the added spills cost (measured 2% faster than 2 blocks).
// DEC: 0 full theory, 1 without backreaction (a separate instantiation each, so the full
// theory's kernel carries no test of the mode), -1 the mode read from c. LOP: lopsided advection.
// COUP = 0: the linear and quadratic couplings only.
template <int STAGE, int DEC = 0, int LOP = 0, int COUP = 1>
__global__ void __launch_bounds__(128, 3) rk4_stage_kernel(Geom g, Coeffs c, StageArgs a) {
    __shared__ YzRows sh;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int k = blockIdx.z + a.k0;
    if (k >= g.nz) return;  // whole block
    yz_rows_fill(g, a.src, i, blockIdx.y * 4, threadIdx.y, k, threadIdx.x, sh);
    __syncthreads();
    stage_point<STAGE, DEC, LOP, COUP>(g, c, a, i, j, k, GATHER_BLOCK, &sh);
}

// Folded variant for boxes whose x-extent is not a multiple of 32, chosen by the host when it
// fills more lanes: blocks of (32, 4, 1), each warp covering 32 / w rows of w = a.fold x-points,
// with the per-thread gather. It gives the same bits as rk4_stage_kernel.
template <int STAGE, int DEC>
__global__ void __launch_bounds__(128, 3) rk4_stage_fold_kernel(Geom g, Coeffs c, StageArgs a) {
    const int w = a.fold, per = 32 / a.fold;
    const int i = blockIdx.x * w + (int)threadIdx.x % w;
    const int j = blockIdx.y * (4 * per) + (int)threadIdx.y * per + (int)threadIdx.x / w;
    const int k = blockIdx.z + a.k0;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    stage_point<STAGE, DEC>(g, c, a, i, j, k, GATHER_LOCAL, nullptr);
}

}  // namespace grf
