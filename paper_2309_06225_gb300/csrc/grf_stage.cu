// RK4 stage kernels (the hot path): one instantiation per stage.
#include "grf_kernels.cuh"
#include "grf_launch.h"

namespace grf {
void launch_stage(int stage, dim3 grid, dim3 block, cudaStream_t st, const Geom& g, const Coeffs& c, const StageArgs& a) {
    if (g.ng != NG) {
        launch_stage6(stage, grid, block, st, g, c, a);
        return;
    }
    if (c.advection) {
        launch_stage_lopsided(stage, grid, block, st, g, c, a);
        return;
    }
    if (c.beta_kind == 2 || c.g3 != 0.0) {  // the exponential coupling or the cubic term: the general instantiation
        launch_stage_general(stage, grid, block, st, g, c, a);
        return;
    }
    if (a.fold != 32) {
        launch_stage_folded(stage, grid, block, st, g, c, a);
        return;
    }
    if (c.decoupled) {
        launch_stage_decoupled(stage, grid, block, st, g, c, a);
        return;
    }
    switch (stage) {
        case 0: rk4_stage_kernel<0, 0, 0, 0><<<grid, block, 0, st>>>(g, c, a); break;
        case 1: rk4_stage_kernel<1, 0, 0, 0><<<grid, block, 0, st>>>(g, c, a); break;
        case 2: rk4_stage_kernel<2, 0, 0, 0><<<grid, block, 0, st>>>(g, c, a); break;
        default: rk4_stage_kernel<3, 0, 0, 0><<<grid, block, 0, st>>>(g, c, a); break;
    }
}
}  // namespace grf
