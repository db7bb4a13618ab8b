// 6th-order scheme ("Accuracy": 4th- and 6th-order finite differences) on boxes with 4 ghost
// layers: centred 6th-order first, second and mixed differences, Kreiss-Oliger dissipation with
// the 8th difference, and the 6th-order lopsided advection stencil (offsets -2..4 towards the
// side the shift points to). Each thread gathers its own point (no shuffles or shared rows).
#pragma once

#include "grf_kernels.cuh"

namespace grf {

constexpr int NG6 = 4;  // ghost layers of the 6th-order scheme

// 6th-order centred first difference times 60 dx at offset p along stride t:
//   (u_3 - u_-3) - 9 (u_2 - u_-2) + 45 (u_1 - u_-1)
__device__ __forceinline__ double fd1_6(const double* __restrict__ u, long long p, long long t) {
    return fma(45.0, __ldg(u + p + t) - __ldg(u + p - t),
               fma(-9.0, __ldg(u + p + 2 * t) - __ldg(u + p - 2 * t), __ldg(u + p + 3 * t) - __ldg(u + p - 3 * t)));
}

// Values, first and second derivatives, lopsided advection terms adv[f] (LOP = 1) and the 8th
// differences sum_d Delta^8_d u of all fields at ghosted offset p.
//   first:  ((u_3 - u_-3) - 9 (u_2 - u_-2) + 45 (u_1 - u_-1)) / (60 dx)
//   second: (2 (u_3 + u_-3) - 27 (u_2 + u_-2) + 270 (u_1 + u_-1) - 490 u_0) / (180 dx^2)
//   mixed:  the first-difference stencil along s applied to first differences along t
//   KO:     (u_4 + u_-4) - 8 (u_3 + u_-3) + 28 (u_2 + u_-2) - 56 (u_1 + u_-1) + 70 u_0 per axis
//   lopsided, beta^d >= 0 (mirrored for beta^d < 0; a_n = u at n points towards the side beta^d
//   points to, b_n = u at n points away from it):
//           beta^d D_d u = |beta^d| (2 b_2 - 24 b_1 - 35 u_0 + 80 a_1 - 30 a_2 + 8 a_3 - a_4) / (60 dx)
template <int LOP>
__device__ __forceinline__ void gather6(const Geom& g, const double* __restrict__ s, long long p, PointIn& in,
                                        double kos[NFIELDS], double* adv) {
    const double i60 = 1.0 / (60.0 * g.dx), i180s = 1.0 / (180.0 * g.dx * g.dx);
    const long long st[3] = {1, g.pitch, g.plane};
    double bet[3] = {0.0, 0.0, 0.0};
    if (LOP) {
#pragma unroll
        for (int d = 0; d < 3; ++d) bet[d] = __ldg(s + (F_SHIFT + d) * g.fstride + p);
    }
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        const double* u = s + f * g.fstride;
        const double u0 = __ldg(u + p);
        in.v[f] = u0;
        double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // pair sums at distance 1..4 over the three axes
        double pr[3][5];
        double av = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double m[5], q[5];
#pragma unroll
            for (int r = 1; r <= 4; ++r) {
                m[r] = __ldg(u + p - r * st[d]);
                q[r] = __ldg(u + p + r * st[d]);
                pr[d][r] = m[r] + q[r];
            }
            const double d1 = fma(45.0, q[1] - m[1], fma(-9.0, q[2] - m[2], q[3] - m[3])) * i60;
            if (!(f >= F_B && f < F_B + 3)) in.d1[d1slot(f)][d] = d1;
            if (LOP) {
                const bool fw = bet[d] >= 0.0;
                const double a1 = fw ? q[1] : m[1], a2 = fw ? q[2] : m[2], a3 = fw ? q[3] : m[3], a4 = fw ? q[4] : m[4];
                const double b1 = fw ? m[1] : q[1], b2 = fw ? m[2] : q[2];
                const double x = fma(80.0, a1, fma(-30.0, a2, fma(8.0, a3, -a4))) + fma(2.0, b2, fma(-24.0, b1, -35.0 * u0));
                av = fma(fabs(bet[d]), x * i60, av);
            }
        }
        if (LOP) adv[f] = av;
        if (has_d2(f)) {
            const int b = d2slot(f);
#pragma unroll
            for (int d = 0; d < 3; ++d)
                in.d2[b][d == 0 ? 0 : (d == 1 ? 3 : 5)] =
                    fma(270.0, pr[d][1], fma(-27.0, pr[d][2], fma(2.0, pr[d][3], -490.0 * u0))) * i180s;
            const int pairs[3][3] = {{0, 1, 1}, {0, 2, 2}, {1, 2, 4}};  // (s, t, slot)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long so = st[pairs[c][0]], to = st[pairs[c][1]];
                const double dp1 = fd1_6(u, p + so, to) * i60, dm1 = fd1_6(u, p - so, to) * i60;
                const double dp2 = fd1_6(u, p + 2 * so, to) * i60, dm2 = fd1_6(u, p - 2 * so, to) * i60;
                const double dp3 = fd1_6(u, p + 3 * so, to) * i60, dm3 = fd1_6(u, p - 3 * so, to) * i60;
                in.d2[b][pairs[c][2]] = fma(45.0, dp1 - dm1, fma(-9.0, dp2 - dm2, dp3 - dm3)) * i60;
            }
        }
#pragma unroll
        for (int r = 1; r <= 4; ++r) t[r] = (pr[0][r] + pr[1][r]) + pr[2][r];
        kos[f] = fma(-56.0, t[1], fma(28.0, t[2], fma(-8.0, t[3], t[4]))) + 210.0 * u0;
    }
}

// ---- block gather of the 6th-order scheme: blocks of 32 x 4 threads, each warp one x-row of
// 32 consecutive points, the 4 warps consecutive y-rows. A mixed derivative d_s d_t u is the
// 6th-order s-stencil applied to the first t-derivatives D_t u at s-offsets +-1..3; along x those
// are the neighbouring lanes' own first derivatives (shuffles), plus a halo of 3 points beyond each
// end of the row; d_y d_z takes the first z-derivatives of the rows y0-3 .. y0+6 from shared
// memory. Threads past the interior take part at the last ghost column / row needed by interior
// points (x, y <= n + 2), so every load stays inside the ghosted box.

// Halo of a warp's row: D_t (t = y, z) of the 12 fields with second derivatives at x0-3 .. x0-1
// and x0+32 .. x0+34 (q = 0 .. 5). Combination c = 2 b + t (0 .. 23) lives in register c / 5 at
// lanes 6 (c % 5) + q, so the register is the same for every lane of a shuffle.
struct WarpRow6 {
    int lane;
    double hv[5];
};

__device__ __forceinline__ double fd1_6r(const double* __restrict__ u, long long p, long long t, double i60) {
    return __dmul_rn(fd1_6(u, p, t), i60);
}

__device__ __forceinline__ void warp_row_halo6(const Geom& g, const double* __restrict__ s, int x0, int j, int k, int lane,
                                               WarpRow6& wr) {
    const double i60 = 1.0 / (60.0 * g.dx);
    wr.lane = lane;
    const int q = lane % 6, cl = lane / 6;  // lanes 30, 31 hold nothing
    const int hx = min(q < 3 ? x0 - 3 + q : x0 + 29 + q, g.nx + 2);
    const long long ph = gidx(g, hx + NG6, j + NG6, k + NG6);
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int c = 5 * r + cl;
        double v = 0.0;
        if (lane < 30 && c < 24) {
            const int b = c >> 1, t = c & 1;
            v = fd1_6r(s + (long long)d2field(b) * g.fstride, ph, t ? g.plane : g.pitch, i60);
        }
        wr.hv[r] = v;
    }
}

// d_x d_t u of d2 slot b from this lane's own D = D_t u and its neighbours'.
__device__ __forceinline__ double mixed_x_warp6(const WarpRow6& wr, int b, int t, double own, double i60) {
    const unsigned full = 0xffffffffu;
    const int c = 2 * b + t, r = c / 5, base = 6 * (c % 5);
    const int L = wr.lane;
    double m[4], pl[4];
    const double dn1 = __shfl_up_sync(full, own, 1), dn2 = __shfl_up_sync(full, own, 2), dn3 = __shfl_up_sync(full, own, 3);
    const double up1 = __shfl_down_sync(full, own, 1), up2 = __shfl_down_sync(full, own, 2), up3 = __shfl_down_sync(full, own, 3);
#pragma unroll
    for (int o = 1; o <= 3; ++o) {
        // a lane needs the halo on at most one side for offset o: below x0 (q = L - o + 3) or
        // beyond x0 + 31 (q = L + o - 29)
        const int qh = (L - o < 0) ? L - o + 3 : (L + o > 31 ? L + o - 29 : 0);
        const double h = __shfl_sync(full, wr.hv[r], base + qh);
        const double nm = o == 1 ? dn1 : (o == 2 ? dn2 : dn3);
        const double np = o == 1 ? up1 : (o == 2 ? up2 : up3);
        m[o] = (L - o < 0) ? h : nm;
        pl[o] = (L + o > 31) ? h : np;
    }
    return __dmul_rn(fma(45.0, pl[1] - m[1], fma(-9.0, pl[2] - m[2], pl[3] - m[3])), i60);
}

struct YzRows6 {
    double dz[12][10][32];  // rounded first z-derivatives on rows y0-3 .. y0+6 (row index y - y0 + 3)
};

// Every thread of the block calls this, then __syncthreads(). Warp wy fills its own row (y0+wy)
// and, for wy < 3, the halo rows y0-3+wy and y0+4+wy.
__device__ __forceinline__ void yz_rows_fill6(const Geom& g, const double* __restrict__ s, int x, int y0, int wy, int k,
                                              int lane, YzRows6& sh) {
    const double i60 = 1.0 / (60.0 * g.dx);
    const int xc = min(x, g.nx + 2);
    const int rows[3] = {wy + 3, wy, wy + 7};
    const int nr = wy < 3 ? 3 : 1;
    for (int q = 0; q < nr; ++q) {
        const int ry = min(y0 - 3 + rows[q], g.ny + 2);
        const long long po = gidx(g, xc + NG6, ry + NG6, k + NG6);
#pragma unroll
        for (int b = 0; b < 12; ++b) sh.dz[b][rows[q]][lane] = fd1_6r(s + (long long)d2field(b) * g.fstride, po, g.plane, i60);
    }
}

// gather6 in block mode (all 128 threads of the block take part): as gather6, the x-mixed and
// d_y d_z derivatives from the neighbours, the first z-derivatives of the 12 fields with second
// derivatives from the shared rows.
template <int LOP>
__device__ __forceinline__ void gather6_block(const Geom& g, const double* __restrict__ s, long long p, PointIn& in,
                                              double kos[NFIELDS], double* adv, const WarpRow6& wr, const YzRows6& sh,
                                              int wy) {
    const double i60 = 1.0 / (60.0 * g.dx), i180s = 1.0 / (180.0 * g.dx * g.dx);
    const long long st[3] = {1, g.pitch, g.plane};
    const int lane = threadIdx.x & 31;
    double bet[3] = {0.0, 0.0, 0.0};
    if (LOP) {
#pragma unroll
        for (int d = 0; d < 3; ++d) bet[d] = __ldg(s + (F_SHIFT + d) * g.fstride + p);
    }
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        const double* u = s + f * g.fstride;
        const double u0 = __ldg(u + p);
        in.v[f] = u0;
        double pr[3][5], d1[3];
        double av = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double m[5], q[5];
#pragma unroll
            for (int r = 1; r <= 4; ++r) {
                m[r] = __ldg(u + p - r * st[d]);
                q[r] = __ldg(u + p + r * st[d]);
                pr[d][r] = m[r] + q[r];
            }
            const double x = fma(45.0, q[1] - m[1], fma(-9.0, q[2] - m[2], q[3] - m[3]));
            if (d == 1 && has_d2(f)) d1[d] = __dmul_rn(x, i60);      // shared with the neighbours' d_x d_y
            else if (d == 2 && has_d2(f)) d1[d] = sh.dz[d2slot(f)][wy + 3][lane];
            else d1[d] = x * i60;
            if (!(f >= F_B && f < F_B + 3)) in.d1[d1slot(f)][d] = d1[d];
            if (LOP) {
                const bool fw = bet[d] >= 0.0;
                const double a1 = fw ? q[1] : m[1], a2 = fw ? q[2] : m[2], a3 = fw ? q[3] : m[3], a4 = fw ? q[4] : m[4];
                const double b1 = fw ? m[1] : q[1], b2 = fw ? m[2] : q[2];
                const double y = fma(80.0, a1, fma(-30.0, a2, fma(8.0, a3, -a4))) + fma(2.0, b2, fma(-24.0, b1, -35.0 * u0));
                av = fma(fabs(bet[d]), y * i60, av);
            }
        }
        if (LOP) adv[f] = av;
        if (has_d2(f)) {
            const int b = d2slot(f);
#pragma unroll
            for (int d = 0; d < 3; ++d)
                in.d2[b][d == 0 ? 0 : (d == 1 ? 3 : 5)] =
                    fma(270.0, pr[d][1], fma(-27.0, pr[d][2], fma(2.0, pr[d][3], -490.0 * u0))) * i180s;
            in.d2[b][1] = mixed_x_warp6(wr, b, 0, d1[1], i60);
            in.d2[b][2] = mixed_x_warp6(wr, b, 1, d1[2], i60);
            const double(*rz)[32] = sh.dz[b];
            const int c = wy + 3;
            in.d2[b][4] = __dmul_rn(fma(45.0, rz[c + 1][lane] - rz[c - 1][lane],
                                        fma(-9.0, rz[c + 2][lane] - rz[c - 2][lane], rz[c + 3][lane] - rz[c - 3][lane])),
                                    i60);
        }
        double t[5];
#pragma unroll
        for (int r = 1; r <= 4; ++r) t[r] = (pr[0][r] + pr[1][r]) + pr[2][r];
        kos[f] = fma(-56.0, t[1], fma(28.0, t[2], fma(-8.0, t[3], t[4]))) + 210.0 * u0;
    }
}

// One RK4 stage at one point of a 6th-order box, as stage_point (a.ko = -sigma/(256 dx)).
template <int STAGE, int LOP>
__device__ __forceinline__ void stage_point6(const Geom& g, const Coeffs& c, const StageArgs& a, int i, int j, int k,
                                             const YzRows6& sh) {
    const int lane = threadIdx.x & 31;
    const int ic = min(i, g.nx + 2), jc = min(j, g.ny + 2);
    const long long p = gidx(g, ic + NG6, jc + NG6, k + NG6);
    PointIn in;
    double kos[NFIELDS], adv[LOP ? NFIELDS : 1];
    WarpRow6 wr;
    warp_row_halo6(g, a.src, i - lane, jc, k, lane, wr);
    gather6_block<LOP>(g, a.src, p, in, kos, adv, wr, sh, threadIdx.y);
    if (i >= g.nx || j >= g.ny) return;
    double r[NFIELDS];
    bool ok = true;
    point_rhs<double, double, -1, LOP>(c, in, r, nullptr, ok, adv);
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
    for (int f = 0; f < NFIELDS; ++f) store_with_images<NG6>(g, a.dst, f, i, j, k, out[f]);
}

// Blocks of (32, 4, 1) threads (block gather); planes k0, k0+1, ... The decoupled mode is read
// from c at run time.
template <int STAGE, int LOP>
__global__ void __launch_bounds__(128, 3) rk4_stage6_kernel(Geom g, Coeffs c, StageArgs a) {
    __shared__ YzRows6 sh;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int k = blockIdx.z + a.k0;
    if (k >= g.nz) return;  // whole block
    yz_rows_fill6(g, a.src, i, blockIdx.y * 4, threadIdx.y, k, threadIdx.x, sh);
    __syncthreads();
    stage_point6<STAGE, LOP>(g, c, a, i, j, k, sh);
}

// sum_d Delta^8_d u at ghosted offset p (pair sums added x, y, z)
__device__ __forceinline__ double ko8(const double* __restrict__ u, long long p, long long sy, long long sz) {
    const long long st[3] = {1, sy, sz};
    double t[5];
#pragma unroll
    for (int r = 1; r <= 4; ++r)
        t[r] = ((__ldg(u + p - r * st[0]) + __ldg(u + p + r * st[0])) + (__ldg(u + p - r * st[1]) + __ldg(u + p + r * st[1]))) +
               (__ldg(u + p - r * st[2]) + __ldg(u + p + r * st[2]));
    return fma(-56.0, t[1], fma(28.0, t[2], fma(-8.0, t[3], t[4]))) + 210.0 * __ldg(u + p);
}

}  // namespace grf
