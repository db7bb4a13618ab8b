// Single-state RHS and constraint kernels (4th-order scheme).
#include "grf_diag.cuh"
#include "grf_launch.h"

namespace grf {

// Launched with blocks of (32, 4, 1) threads (block gather mode, see stage_point). LOP: lopsided
// advection.
template <int LOP>
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
    double adv[LOP ? NFIELDS : 1];
    gather<LOP>(g, s, p, in, kos, &wr, &sh, threadIdx.y, adv);
    if (i >= g.nx || j >= g.ny) return;
    double r[NFIELDS];
    bool ok = true;
    point_rhs<double, double, -1, LOP>(c, in, r, nullptr, ok, adv);
    if (!ok) atomicOr(status, 1);
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) rhs[f * g.fstride + p] = r[f] + ko * kos[f];
}

void launch_rhs(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s, double* rhs,
                double ko, int* status) {
    if (g.ng == NG6) launch_rhs6(grid, block, st, g, c, s, rhs, ko, status);
    else if (c.advection) rhs_kernel<kLopsided><<<grid, block, 0, st>>>(g, c, s, rhs, ko, status);
    else rhs_kernel<0><<<grid, block, 0, st>>>(g, c, s, rhs, ko, status);
}
void launch_constraints(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s,
                        double* out4, double* part, double* dens, double* psi4, double3 origin, double* hyp) {
    if (g.ng == NG6) launch_constraints6(grid, block, st, g, c, s, out4, part, dens, psi4, origin, hyp);
    else if (psi4 || hyp) constraints_kernel<4, 1><<<grid, block, 0, st>>>(g, c, s, out4, part, dens, psi4, origin, hyp);
    else constraints_kernel<4, 0><<<grid, block, 0, st>>>(g, c, s, out4, part, dens, psi4, origin, hyp);
}
}  // namespace grf
