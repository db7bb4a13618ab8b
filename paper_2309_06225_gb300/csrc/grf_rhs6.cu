// Single-state RHS and constraint kernels of the 6th-order scheme (4 ghost layers).
#include "grf_diag.cuh"
#include "grf_launch.h"

namespace grf {

// Blocks of (32, 4, 1) threads, one point each. LOP: lopsided advection.
template <int LOP>
__global__ void __launch_bounds__(128) rhs6_kernel(Geom g, Coeffs c, const double* __restrict__ s,
                                                   double* __restrict__ rhs, double ko, int* status) {
    int i, j, k;
    if (!interior_thread(g, i, j, k)) return;
    const long long p = gidx(g, i + NG6, j + NG6, k + NG6);
    PointIn in;
    double kos[NFIELDS], adv[LOP ? NFIELDS : 1];
    gather6<LOP>(g, s, p, in, kos, adv);
    double r[NFIELDS];
    bool ok = true;
    point_rhs<double, double, -1, LOP>(c, in, r, nullptr, ok, adv);
    if (!ok) atomicOr(status, 1);
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) rhs[f * g.fstride + p] = r[f] + ko * kos[f];
}

void launch_rhs6(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s, double* rhs,
                 double ko, int* status) {
    if (c.advection) rhs6_kernel<kLopsided><<<grid, block, 0, st>>>(g, c, s, rhs, ko, status);
    else rhs6_kernel<0><<<grid, block, 0, st>>>(g, c, s, rhs, ko, status);
}

void launch_constraints6(dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const double* s,
                         double* out4, double* part, double* dens, double* psi4, double3 origin) {
    constraints_kernel<6><<<grid, block, 0, st>>>(g, c, s, out4, part, dens, psi4, origin);
}

}  // namespace grf
