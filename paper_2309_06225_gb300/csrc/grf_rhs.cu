// Single-state RHS and constraint kernels.
#include "grf_kernels.cuh"
#include "grf_launch.h"

namespace grf {

// Launched with blocks of (32, 4, 1) threads (block gather mode, see stage_point).
__global__ void __launch_bounds__(128) rhs_kernel(Geom g, Coeffs c, const double* __restrict__ s, double* __restrict__ rhs,
                                                  double ko, int* status) {
    __shared__ YzRows sh;
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int k = blockIdx.z;
    yz_rows_fill(g, s, i, blockIdx.y * 4, threadIdx.y, k, lane, sh);
    __syncthreads();
    const int jc = min(j, g.ny + 2);
    const long long p = gidx(g, min(i, g.nx + 2) + NG, jc + NG, k + NG);
    PointIn in;
    double kos[NFIELDS];
    WarpRow wr;
    warp_row_halo(g, s, i - lane, jc, k, lane, wr);
    gather(g, s, p, in, kos, &wr, &sh, threadIdx.y);
    if (i >= g.nx || j >= g.ny) return;
    double r[NFIELDS];
    bool ok = true;
    point_rhs<double>(c, in, r, nullptr, ok);
    if (!ok) atomicOr(status, 1);
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) rhs[f * g.fstride + p] = r[f] + ko * kos[f];
}

// Constraints H, M_i at interior points (state layout, 4 fields) and per-block partial norms:
// part[block][8] = {sum H^2, max|H|, sum M1^2, max|M1|, ...}
// out4 (H, M_i; with the per-block norm partials in `part`) and dens (the energy densities of the
// three scalar terms) are each written when non-null.
__global__ void __launch_bounds__(128) constraints_kernel(Geom g, Coeffs c, const double* __restrict__ s,
                                                          double* __restrict__ out4, double* __restrict__ part,
                                                          double* __restrict__ dens) {
    // blocks of (32, 4, 1): block gather mode, as rhs_kernel; every thread stays to the reduction
    __shared__ double red[8][128];
    __shared__ YzRows sh;
    const int lane = threadIdx.x;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int k = blockIdx.z;
    const bool live = i < g.nx && j < g.ny;
    yz_rows_fill(g, s, i, blockIdx.y * 4, threadIdx.y, k, lane, sh);
    __syncthreads();
    const int jc = min(j, g.ny + 2);
    const long long p = gidx(g, min(i, g.nx + 2) + NG, jc + NG, k + NG);
    PointIn in;
    double kos[NFIELDS];
    WarpRow wr;
    warp_row_halo(g, s, i - lane, jc, k, lane, wr);
    gather(g, s, p, in, kos, &wr, &sh, threadIdx.y);
    double vals[4] = {0.0, 0.0, 0.0, 0.0};
    if (live) {
        double r[NFIELDS];
        PointExtra ex;
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

void launch_rhs(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s, double* rhs,
                double ko, int* status) {
    rhs_kernel<<<grid, block, 0, st>>>(g, c, s, rhs, ko, status);
}
void launch_constraints(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s,
                        double* out4, double* part, double* dens) {
    constraints_kernel<<<grid, block, 0, st>>>(g, c, s, out4, part, dens);
}
}  // namespace grf
