// Batched RK4 over many boxes: the box and tile descriptors and the per-tile stage shared by the
// per-stage kernels (grf_batch.cu) and the persistent kernel (grf_batch_persistent.cu), which are
// compiled in separate translation units so that the library builds in parallel.
#pragma once

#include "grf.h"
#include "grf_kernels.cuh"

namespace grf {

struct BoxDesc {
    Geom g;
    Coeffs c;
    double* un;
    double* A;
    double* B;
    double* acc;
    double dt, ko, min_chi, min_lapse;
    int enforce;
    int pad_;
};

struct TileDesc {
    int box, i0, j0, k0;
    int w;  // x-points per row: blockDim.x (one row per warp), or 8 / 16 (a folded 32-wide tile:
            // each warp covers 32 / w rows of a narrow box)
};

// DEC: 0 full theory, 1 without backreaction, -1 read from the box's coefficients; LOP: lopsided
// advection.
template <int STAGE, int DEC, int LOP>
__device__ __forceinline__ void batch_tile(const BoxDesc* __restrict__ boxes, const TileDesc& td, int* status,
                                           YzRows& sh) {
    const BoxDesc& d = boxes[td.box];
    const bool folded = td.w != (int)blockDim.x;
    const int i = td.i0 + (folded ? (int)threadIdx.x % td.w : (int)threadIdx.x);
    const int j = td.j0 + (folded ? (int)threadIdx.y * ((int)blockDim.x / td.w) + (int)threadIdx.x / td.w : (int)threadIdx.y);
    const int k = td.k0 + threadIdx.z;
    // Tile shape -> gather mode (all modes give the same bits):
    //   32 x 4 x 1: block mode, d_y d_z through the shared rows; every thread stays to the barrier.
    //   width a multiple of 32: warp mode; whole warps stay for the shuffles.
    //   folded tiles and other shapes: per-thread mode.
    const int mode = folded ? GATHER_LOCAL
                     : ((blockDim.x == 32 && blockDim.y == 4 && blockDim.z == 1) ? GATHER_BLOCK
                        : ((blockDim.x & 31) == 0 ? GATHER_WARP : GATHER_LOCAL));
    StageArgs a;
    a.un = d.un;
    a.acc = d.acc;
    a.dt = d.dt;
    a.ko = d.ko;
    a.min_chi = d.min_chi;
    a.min_lapse = d.min_lapse;
    a.enforce = d.enforce;
    a.status = status;
    a.k0 = 0;
    a.fold = 32;
    a.src = (STAGE == 0) ? d.un : (STAGE == 1 ? d.A : (STAGE == 2 ? d.B : d.A));
    a.dst = (STAGE == 0) ? d.A : (STAGE == 1 ? d.B : (STAGE == 2 ? d.A : d.un));
    if (mode == GATHER_BLOCK) {
        if (k >= d.g.nz) return;  // the whole block (k = td.k0)
        __syncthreads();          // readers of the previous tile's rows are done
        yz_rows_fill(d.g, a.src, i, td.j0, threadIdx.y, k, threadIdx.x, sh);
        __syncthreads();
    } else if (j >= d.g.ny || k >= d.g.nz || (mode == GATHER_LOCAL && i >= d.g.nx)) {
        return;
    }
    stage_point<STAGE, DEC, LOP>(d.g, d.c, a, i, j, k, mode, &sh);
}

// Out-of-line copy of batch_tile for the persistent kernel: with the four stages inlined into one
// kernel, ptxas spilled 52 KB per thread; called, each stage is allocated on its own (13 KB).
template <int STAGE, int DEC, int LOP>
__device__ __noinline__ void batch_tile_call(const BoxDesc* __restrict__ boxes, const TileDesc& td, int* status,
                                             YzRows& sh) {
    batch_tile<STAGE, DEC, LOP>(boxes, td, status, sh);
}

// Shared with the split-box evolution (grf_patches.cu), in grf_batch.cu: the couplings check of
// one parameter set; a box descriptor (geometry, coefficients, dissipation, floors and dt; the
// buffers are left null); the x-points per row of a box's 32 x 4 x 1 tiles (32, or a folded 16 or 8);
// one stage launch over a tile list.
bool batch_params_ok(const grf_params* p);
void batch_box_desc(BoxDesc& d, const grf_box* b, const grf_params* p, double dt);
int batch_row_width(int nx);
void launch_batch_stage(int stage, long long ntiles, dim3 block, cudaStream_t st, const BoxDesc* boxes,
                        const TileDesc* tiles, int* status);

// The persistent cooperative launch (grf_batch_persistent.cu): its function attributes (loads the
// kernel), its resident blocks per SM for `nthreads` threads, and the launch.
cudaError_t batch_persistent_attributes();
cudaError_t batch_persistent_occupancy(int nthreads, int* per_sm);
cudaError_t launch_batch_persistent(dim3 grid, dim3 block, const BoxDesc* boxes, const TileDesc* tiles, int ntiles,
                                    int nsteps, unsigned* bar, int* status, long long timeout, cudaStream_t st);

}  // namespace grf
