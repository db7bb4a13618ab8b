// Tangent-linear RK4 evolution and the sphere-averaged scalar signal: the gradient of
//   L = sum_{n=1..N} dt * sum_p w_p phi(R x_p, t_n)
// (26-point degree-7 rule on the sphere of radius R, trilinear interpolation of phi, evaluated
// after every full RK4 step) with respect to three parameters, propagated forward exactly:
// every grid value carries its derivatives in three directions (grf_dual::D3) through the same
// pointwise RHS, stencils, dissipation, RK4 update and enforcement as the evolution itself.
// The three directions are seeded by the tangents of the initial state (e.g. with respect to
// the initial scalar amplitude) and by the tangents of the couplings lambda and g2.
#include <cmath>
#include <cstdint>

#include "grf.h"
#include "grf_dual.cuh"
#include "grf_kernels.cuh"
#include "grf_launch.h"
#include "grf_sphere.cuh"

namespace grf {

using grf_dual::D3;

struct TlmArgs {
    const double* src[4];  // value state and 3 tangent states whose RHS is evaluated
    const double* un[4];
    double* acc[4];
    double* dst[4];
    double dt, ko, min_chi, min_lapse;
    int enforce;
    int* status;
};

__device__ __forceinline__ void gather_d3(const Geom& g, const double* const* s, long long p, PointInT<D3>& in) {
    const double i12 = 1.0 / (12.0 * g.dx), i12s = 1.0 / (12.0 * g.dx * g.dx);
    const long long sx = 1, sy = g.pitch, sz = g.plane;
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        double v[4], d1[4][3], d2[4][6];
        const bool first = !(f >= F_B && f < F_B + 3);
        const bool second = has_d2(f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const double* u = s[c] + f * g.fstride;
            v[c] = __ldg(u + p);
            if (first) {
                d1[c][0] = fd1(u, p, sx, i12);
                d1[c][1] = fd1(u, p, sy, i12);
                d1[c][2] = second ? fd1_rounded(u, p, sz, i12) : fd1(u, p, sz, i12);  // as in gather()
            }
            if (second) {
                d2[c][0] = fd2(u, p, sx, v[c], i12s);
                d2[c][1] = mixed_local(u, p, sx, sy, i12);
                d2[c][2] = mixed_local(u, p, sx, sz, i12);
                d2[c][3] = fd2(u, p, sy, v[c], i12s);
                d2[c][4] = mixed_local(u, p, sy, sz, i12);
                d2[c][5] = fd2(u, p, sz, v[c], i12s);
            }
        }
        in.v[f] = D3(v[0], v[1], v[2], v[3]);
        if (first) {
            const int a = d1slot(f);
#pragma unroll
            for (int d = 0; d < 3; ++d) in.d1[a][d] = D3(d1[0][d], d1[1][d], d1[2][d], d1[3][d]);
        }
        if (second) {
            const int b = d2slot(f);
#pragma unroll
            for (int m = 0; m < 6; ++m) in.d2[b][m] = D3(d2[0][m], d2[1][m], d2[2][m], d2[3][m]);
        }
    }
}

__device__ __forceinline__ void enforce_point_d3(D3 u[NFIELDS], double min_chi, double min_lapse) {
    D3 hh[6], hi[6], id;
#pragma unroll
    for (int m = 0; m < 6; ++m) hh[m] = u[F_H + m];
    sym3_inv(hh, hi, id);
    const D3 tr = hi[0] * u[F_A] + hi[3] * u[F_A + 3] + hi[5] * u[F_A + 5]
                  + 2.0 * (hi[1] * u[F_A + 1] + hi[2] * u[F_A + 2] + hi[4] * u[F_A + 4]);
#pragma unroll
    for (int m = 0; m < 6; ++m) u[F_A + m] = u[F_A + m] - hh[m] * tr * (1.0 / 3.0);
    u[F_CHI] = grf_dual::fmax(u[F_CHI], min_chi);
    u[F_LAPSE] = grf_dual::fmax(u[F_LAPSE], min_lapse);
}

template <int STAGE>
__global__ void __launch_bounds__(128) tlm_stage_kernel(Geom g, CoeffsT<D3> c, TlmArgs a) {
    int i, j, k;
    if (!interior_thread(g, i, j, k)) return;
    const long long p = gidx(g, i + NG, j + NG, k + NG);
    PointInT<D3> in;
    gather_d3(g, a.src, p, in);
    D3 r[NFIELDS];
    bool ok = true;
    point_rhs<D3, D3>(c, in, r, nullptr, ok);
    if (!ok) atomicOr(a.status, 1);
    D3 out[NFIELDS];
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        double kf[4], unf[4], accf[4];
        const double rv[4] = {r[f].v, r[f].d0, r[f].d1, r[f].d2};
        const double inv[4] = {in.v[f].v, in.v[f].d0, in.v[f].d1, in.v[f].d2};
#pragma unroll
        for (int cmp = 0; cmp < 4; ++cmp) {
            kf[cmp] = rv[cmp] + a.ko * ko6(a.src[cmp] + f * g.fstride, p, g.pitch, g.plane);
            unf[cmp] = (STAGE == 0) ? inv[cmp] : a.un[cmp][f * g.fstride + p];
            if (STAGE == 0) accf[cmp] = kf[cmp];
            else if (STAGE == 3) accf[cmp] = a.acc[cmp][f * g.fstride + p] + kf[cmp];
            else accf[cmp] = a.acc[cmp][f * g.fstride + p] + 2.0 * kf[cmp];
            if (STAGE < 3) a.acc[cmp][f * g.fstride + p] = accf[cmp];
        }
        const double cs = (STAGE == 0 || STAGE == 1) ? 0.5 * a.dt : (STAGE == 2 ? a.dt : a.dt * (1.0 / 6.0));
        double o[4];
#pragma unroll
        for (int cmp = 0; cmp < 4; ++cmp) o[cmp] = (STAGE == 3) ? fma(cs, accf[cmp], unf[cmp]) : fma(cs, kf[cmp], unf[cmp]);
        out[f] = D3(o[0], o[1], o[2], o[3]);
    }
    if (a.enforce) enforce_point_d3(out, a.min_chi, a.min_lapse);
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        store_with_images(g, a.dst[0], f, i, j, k, out[f].v);
        store_with_images(g, a.dst[1], f, i, j, k, out[f].d0);
        store_with_images(g, a.dst[2], f, i, j, k, out[f].d1);
        store_with_images(g, a.dst[3], f, i, j, k, out[f].d2);
    }
}

// loss[c] += dt * sum_q w_q phi_c(centre + R x_q) for the value (c = 0) and the 3 tangents,
// trilinear interpolation on the interior points (x = x0 + i dx). One warp; fixed summation
// order, so the result is deterministic.
__global__ void sphere_signal_kernel(Geom g, double x0, double y0, double z0, double R, double cx, double cy, double cz,
                                     const double* s0, const double* s1, const double* s2, const double* s3, double dt,
                                     double* loss, int* status) {
    __shared__ double part[32][4];
    const int q = threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (q < 26) {
        double ux, uy, uz, w;
        sphere_point(q, ux, uy, uz, w);
        const double fx = (cx + R * ux - x0) / g.dx, fy = (cy + R * uy - y0) / g.dx, fz = (cz + R * uz - z0) / g.dx;
        int i0 = (int)floor(fx), j0 = (int)floor(fy), k0 = (int)floor(fz);
        if (i0 < 0 || j0 < 0 || k0 < 0 || i0 + 1 >= g.nx || j0 + 1 >= g.ny || k0 + 1 >= g.nz) {
            atomicOr(status, 4);  // sphere leaves the interior
        } else {
            const double tx = fx - i0, ty = fy - j0, tz = fz - k0;
            const double* arr[4] = {s0, s1, s2, s3};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double* u = arr[c] + F_PHI * g.fstride;
                double val = 0.0;
#pragma unroll
                for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            const double wt = (dx ? tx : 1.0 - tx) * (dy ? ty : 1.0 - ty) * (dz ? tz : 1.0 - tz);
                            val = fma(wt, u[gidx(g, i0 + dx + NG, j0 + dy + NG, k0 + dz + NG)], val);
                        }
                acc[c] = w * val;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) part[q][c] = acc[c];
    __syncwarp();
    if (q == 0)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int r = 0; r < 26; ++r) s += part[r][c];
            loss[c] = __fma_rn(dt, s, loss[c]);
        }
}

}  // namespace grf

using namespace grf;

namespace {

bool box_valid(const grf_box* b) {
    if (!b) return false;
    if (b->ng != 3 || b->nx < 2 || b->ny < 2 || b->nz < 2 || !(b->dx > 0.0)) return false;
    if (b->pitch < (long long)b->nx + 6) return false;
    if (b->bc != GRF_BC_PERIODIC && b->bc != GRF_BC_FROZEN) return false;
    if (b->bc == GRF_BC_PERIODIC && (b->nx < 3 || b->ny < 3 || b->nz < 3)) return false;
    return true;
}

Geom geom_from(const grf_box* b) {
    Geom g;
    g.nx = b->nx; g.ny = b->ny; g.nz = b->nz;
    g.NX = b->nx + 6; g.NY = b->ny + 6; g.NZ = b->nz + 6;
    g.ng = NG;
    g.pitch = b->pitch;
    g.plane = b->pitch * g.NY;
    g.fstride = g.plane * g.NZ;
    g.dx = b->dx;
    g.periodic = (b->bc == GRF_BC_PERIODIC);
    g.reflect = 0;  // mirror boxes are not accepted here
    return g;
}

size_t sbytes(const Geom& g) { return sizeof(double) * (size_t)NFIELDS * (size_t)g.fstride; }

__global__ void tlm_ghost_fill_kernel(Geom g, double* __restrict__ s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z;
    if (i >= g.NX || j >= g.NY) return;
    auto wrap = [](int a, int n) { int x = (a - NG) % n; if (x < 0) x += n; return x + NG; };
    const int wi = wrap(i, g.nx), wj = wrap(j, g.ny);
    const bool ghost_ij = (wi != i) || (wj != j);
    double* u = s + f * g.fstride;
    for (int k = 0; k < g.NZ; ++k) {
        const int wk = wrap(k, g.nz);
        if (!ghost_ij && wk == k) continue;
        u[gidx(g, i, j, k)] = u[gidx(g, wi, wj, wk)];
    }
}

}  // namespace

extern "C" {

size_t grf_tlm_workspace_bytes(const grf_box* box) {
    if (!box_valid(box)) return 0;
    return 12 * sbytes(geom_from(box)) + 256;
}

int grf_tlm_rk4(const grf_box* box, const grf_params* params, const double* dparams, double* state, double* tangents,
                double dt, int nsteps, const grf_sphere* sphere, double* loss, void* ws, size_t ws_bytes,
                grf_stream_t stream) {
    if (!box_valid(box) || !params || !dparams || !state || !tangents || !sphere || !loss || nsteps < 0)
        return GRF_EINVAL;
    if (params->beta_kind != GRF_BETA_LINEAR && params->beta_kind != GRF_BETA_QUADRATIC &&
        params->beta_kind != GRF_BETA_EXPONENTIAL)
        return GRF_EINVAL;
    if (params->beta_kind == GRF_BETA_EXPONENTIAL && !(params->beta_kappa >= 0.0 && params->beta_kappa < 1e300))
        return GRF_EINVAL;
    if (params->advection != 0) return GRF_EINVAL;  // centred advection only
    if (!(1.0 + params->a0 > 0.0) || !(1.0 + params->b0 > 0.0) || !(sphere->radius > 0.0)) return GRF_EINVAL;
    const Geom g = geom_from(box);
    const size_t sb = sbytes(g);
    if (!ws || ws_bytes < 12 * sb + 256 || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    if (nsteps == 0) return GRF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    int* status = (int*)base;
    double* bufs = (double*)(base + 256);
    auto buf = [&](int which, int comp) { return (double*)((char*)bufs + (size_t)(which * 4 + comp) * sb); };
    double* un[4] = {state, tangents, (double*)((char*)tangents + sb), (double*)((char*)tangents + 2 * sb)};
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e != cudaSuccess) return record_cuda_error(e);
    for (int c = 0; c < 4; ++c) {
        if (g.periodic) {
            dim3 blk(32, 8, 1), grd((g.NX + 31) / 32, (g.NY + 7) / 8, NFIELDS);
            tlm_ghost_fill_kernel<<<grd, blk, 0, st>>>(g, un[c]);
        } else {
            e = cudaMemcpyAsync(buf(0, c), un[c], sb, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(buf(1, c), un[c], sb, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return record_cuda_error(e);
        }
    }
    CoeffsT<D3> c;
    c.kappa1 = params->kappa1; c.kappa2 = params->kappa2; c.kappa3 = params->kappa3;
    c.shift_F = params->shift_F; c.eta = params->eta;
    c.lam = D3(params->lambda, dparams[0], dparams[2], dparams[4]);
    c.g2 = D3(params->g2, dparams[1], dparams[3], dparams[5]);
    c.g3 = params->g3;
    c.inv_1pa = 1.0 / (1.0 + params->a0);
    c.a_1pa = params->a0 / (1.0 + params->a0);
    c.bK = 3.0 * params->b0 / (4.0 * (1.0 + params->b0));
    c.bTh = 1.0 / (2.0 * (1.0 + params->b0));
    c.beta_kind = params->beta_kind;
    c.beta_kappa = params->beta_kappa;
    c.decoupled = params->decoupled;
    TlmArgs a;
    a.dt = dt;
    a.ko = params->sigma_ko / (64.0 * box->dx);
    a.min_chi = params->min_chi;
    a.min_lapse = params->min_lapse;
    a.enforce = params->enforce_algebraic;
    a.status = status;
    for (int cc = 0; cc < 4; ++cc) { a.un[cc] = un[cc]; a.acc[cc] = buf(2, cc); }
    const dim3 blk(32, 4, 1);
    const dim3 grd((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
    for (int n = 0; n < nsteps; ++n) {
        for (int s = 0; s < 4; ++s) {
            for (int cc = 0; cc < 4; ++cc) {
                a.src[cc] = (s == 0) ? un[cc] : (s == 2 ? buf(1, cc) : buf(0, cc));
                a.dst[cc] = (s == 3) ? un[cc] : (s == 1 ? buf(1, cc) : buf(0, cc));
            }
            switch (s) {
                case 0: tlm_stage_kernel<0><<<grd, blk, 0, st>>>(g, c, a); break;
                case 1: tlm_stage_kernel<1><<<grd, blk, 0, st>>>(g, c, a); break;
                case 2: tlm_stage_kernel<2><<<grd, blk, 0, st>>>(g, c, a); break;
                default: tlm_stage_kernel<3><<<grd, blk, 0, st>>>(g, c, a); break;
            }
        }
        sphere_signal_kernel<<<1, 32, 0, st>>>(g, box->x0, box->y0, box->z0, sphere->radius, sphere->cx, sphere->cy,
                                               sphere->cz, un[0], un[1], un[2], un[3], dt, loss, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    int h = 0;
    e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return record_cuda_error(e);
    if (h & 4) return GRF_EINVAL;
    if (h & 1) return GRF_ESINGULAR;
    return GRF_OK;
}

}  // extern "C"
