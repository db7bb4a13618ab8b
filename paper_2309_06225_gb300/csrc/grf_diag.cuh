// Constraint and energy-density kernel of both schemes (included by grf_rhs.cu and grf_rhs6.cu).
#pragma once

#include "grf_kernels6.cuh"

namespace grf {

// Constraints H, M_i at interior points (state layout, 4 fields) and per-block partial norms:
// part[block][8] = {sum H^2, max|H|, sum M1^2, max|M1|, ...}
// out4 (H, M_i; with the per-block norm partials in `part`) and dens (the energy densities of the
// three scalar terms) are each written when non-null.
// ORD = 4: block gather mode (as rhs_kernel); ORD = 6: the 6th-order per-thread gather.
// psi4 (2 fields, re and im) receives the Weyl scalar with the triad about the origin; o = the
// coordinates of interior point (0, 0, 0); hyp (4 fields) the hyperbolicity diagnostics of the
// coupled system (PointExtraT::hyp). PSI4 = 1 compiles those outputs in (they need the assembled
// or solved coupled system); with PSI4 = 0 the compiler drops the coupled solve, which H, M_i and
// the densities do not use.
template <int ORD, int PSI4>
__global__ void __launch_bounds__(128) constraints_kernel(Geom g, Coeffs c, const double* __restrict__ s,
                                                          double* __restrict__ out4, double* __restrict__ part,
                                                          double* __restrict__ dens, double* __restrict__ psi4,
                                                          double3 o, double* __restrict__ hyp) {
    // blocks of (32, 4, 1); every thread stays to the reduction
    __shared__ double red[8][128];
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int k = blockIdx.z;
    const bool live = i < g.nx && j < g.ny;
    long long p;
    PointIn in;
    double kos[NFIELDS];
    if constexpr (ORD == 4) {
        __shared__ YzRows sh;
        yz_rows_fill(g, s, i, blockIdx.y * 4, threadIdx.y, k, lane, sh);
        __syncthreads();
        const int jc = min(j, g.ny + 2);
        p = gidx(g, min(i, g.nx + 2) + NG, jc + NG, k + NG);
        WarpRow wr;
        warp_row_halo(g, s, i - lane, jc, k, lane, wr);
        gather(g, s, p, in, kos, &wr, &sh, threadIdx.y);
    } else {
        p = gidx(g, min(i, g.nx - 1) + NG6, min(j, g.ny - 1) + NG6, k + NG6);
        if (live) gather6<0>(g, s, p, in, kos, nullptr);
    }
    double vals[4] = {0.0, 0.0, 0.0, 0.0};
    if (live) {
        double r[NFIELDS];
        PointExtra ex;
        if (PSI4 && psi4) {
            ex.want_psi4 = 1;
            ex.xyz[0] = o.x + i * g.dx;
            ex.xyz[1] = o.y + j * g.dx;
            ex.xyz[2] = o.z + k * g.dx;
        }
        if (PSI4 && hyp) ex.want_hyp = 1;
        bool ok = true;
        point_rhs<double>(c, in, r, &ex, ok);
        vals[0] = ex.ham;
        vals[1] = ex.mom[0];
        vals[2] = ex.mom[1];
        vals[3] = ex.mom[2];
        if (out4)
            for (int m = 0; m < 4; ++m) out4[m * g.fstride + p] = vals[m];
        if (dens)
            for (int m = 0; m < 3; ++m) dens[m * g.fstride + p] = ex.rho8[m];
        if (PSI4 && psi4) {
            psi4[p] = ex.psi4[0];
            psi4[g.fstride + p] = ex.psi4[1];
        }
        if (PSI4 && hyp)
            for (int m = 0; m < 4; ++m) hyp[m * g.fstride + p] = ex.hyp[m];
    }
    const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    for (int m = 0; m < 4; ++m) {
        red[2 * m][t] = vals[m] * vals[m];
        red[2 * m + 1][t] = fabs(vals[m]);
    }
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (t < w)
            for (int m = 0; m < 4; ++m) {
                red[2 * m][t] += red[2 * m][t + w];
                red[2 * m + 1][t] = fmax(red[2 * m + 1][t], red[2 * m + 1][t + w]);
            }
        __syncthreads();
    }
    if (t == 0 && part) {
        const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        for (int m = 0; m < 8; ++m) part[b * 8 + m] = red[m][0];
    }
}

}  // namespace grf
