// RK4 stage kernels of the 6th-order scheme with centred advection; the lopsided ones are in
// grf_stage6l.cu.
#include "grf_kernels6.cuh"
#include "grf_launch.h"

namespace grf {
void launch_stage6(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c,
                   const StageArgs& a) {
    if (c.advection) {
        launch_stage6_lopsided(stage, grid, block, st, g, c, a);
        return;
    }
    switch (stage) {
        case 0: rk4_stage6_kernel<0, 0><<<grid, block, 0, st>>>(g, c, a); break;
        case 1: rk4_stage6_kernel<1, 0><<<grid, block, 0, st>>>(g, c, a); break;
        case 2: rk4_stage6_kernel<2, 0><<<grid, block, 0, st>>>(g, c, a); break;
        default: rk4_stage6_kernel<3, 0><<<grid, block, 0, st>>>(g, c, a); break;
    }
}
}  // namespace grf
