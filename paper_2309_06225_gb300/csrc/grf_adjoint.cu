// Discrete adjoint (reverse mode) of the RK4 evolution and of the sphere-averaged scalar signal
//   L = sum_{n=1..N} dt * sum_q w_q phi(c + R xhat_q, t_n)
// (26-point degree-7 rule, trilinear interpolation of phi, evaluated after every full RK4 step).
// Given the cotangent of L (and optionally of the final state), the reverse sweep returns the
// gradient of L with respect to the initial state (all 27 fields) and to the couplings lambda and
// g2 -- the vector-Jacobian product of the very discrete evolution the stage kernels compute.
//
// Forward: grf_signal_forward evolves the state with the production stage kernels, stores a
// checkpoint every `checkpoint_every` steps and accumulates L.
// Reverse, segment by segment from the last checkpoint: the segment's states are recomputed from
// its checkpoint (stored, one per step), and for every step, from last to first, the three stage
// states u_1, u_2, u_3 and the accumulator k_1 + 2 k_2 + 2 k_3 are recomputed; then the four
// stages are reversed. The RK4 step in the stage kernels' form is
//   u_s = E(u_n + c_s dt k_s)  (s = 1..3, c = 1/2, 1/2, 1),  u_{n+1} = E(u_n + dt/6 (acc + k_4)),
//   k_s = F(u_{s-1}) = f(u, D u, D^2 u; lambda, g2) + KO(u),   acc = k_1 + 2 k_2 + 2 k_3,
// with E the algebraic enforcement. Reversing stage s at a point p:
//   * adj_tape_kernel re-evaluates the pointwise map (f, the stage update and E) on the
//     reverse-mode scalar grf_rev::Rev, recording one tape per point, and seeds the adjoints of
//     the outputs (u_s, and the stage's contribution to acc);
//   * adj_sweep_kernel, a light kernel run at high occupancy, sweeps each tape backwards and
//     obtains the adjoints of the map's inputs: the values of u_{s-1}, u_n and acc at p, the
//     first and second derivatives and the KO sum of u_{s-1} at p, and lambda, g2. The two run
//     in waves of kAdjCols points, one tape column per point;
//   * adj_transpose_kernel applies the transposed stencils to the derivative and KO adjoints:
//     the first-difference stencil is antisymmetric (its transpose is -D), the second and mixed
//     ones and KO are symmetric, so u_{s-1}'s adjoint at q collects -D(G_d1) + D2(G_d2) + KO(G_ko)
//     at q. Periodic ghosts are images, so the adjoints at ghost points belong to their owners:
//     the derivative adjoints are written with their periodic images and the stencils read them
//     across the boundary. Frozen ghosts are constants, whose adjoints are dropped.
// The parameter adjoints are summed per thread in a fixed order and reduced in a fixed order at
// the end, so the gradient is deterministic.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "grf.h"
#include "grf_kernels.cuh"
#include "grf_launch.h"
#include "grf_rev.cuh"
#include "grf_sphere.cuh"

namespace grf {

using grf_rev::Rev;

// leaves of the pointwise map: values, first derivatives (24 slots x 3), second derivatives
// (12 slots x 6), KO sums, u_n, acc, lambda, g2
enum : int { kLV = 0, kLD1 = 27, kLD2 = 99, kLKO = 171, kLUN = 198, kLACC = 225, kLLAM = 252, kLG2 = 253, kNLeaf = 254 };
// tape entries per point and stage: the pointwise RHS records about 4,220, the stage update and
// enforcement about 130 more; an overflow is detected and reported
constexpr int kTapeCap = 5120;
constexpr int kAdjThreads = 128;
// tape columns (points per wave): 1024 per SM of a GB300, so that the sweep (at most 64 registers)
// has 32 warps per SM to hide its dependent memory operations; the taping kernel is held to 128
// registers for 16 warps per SM (more spills, but it ran faster than at 255 registers with 8)
constexpr long long kAdjCols = 152LL * 1024;
constexpr int kSweepThreads = 256;
// derivative and dissipation adjoints per point (slots of the G buffer): d1 72, d2 72, KO 27
constexpr int kGD2 = 72, kGKO = 144, kGSlots = 171;

struct AdjArgs {
    const double* src;    // u_{s-1} (ghosts valid)
    const double* un;     // u_n
    const double* acc;    // k_1 + 2 k_2 + 2 k_3 (stage 3)
    const double* ubar;   // adjoint of the stage output u_s
    double* abar;         // adjoint of the accumulator: written by stage 3, read by stages 0..2
    double* vbar;         // adjoint of the values of u_{s-1} (stages 1..3, written)
    double* unbar;        // adjoint of u_n (stage 3 writes it, stages 2..0 add)
    double* G;            // kGSlots derivative / KO adjoints, with periodic images
    double* pbar;         // per-column sums of the lambda and g2 adjoints
    int* count;           // tape entries of each column (written by the taping kernel)
    double dt, ko, min_chi, min_lapse;
    int enforce;
    int* status;
    long long npts;
};

template <typename T>
__device__ __forceinline__ void enforce_point_t(T u[NFIELDS], double min_chi, double min_lapse) {
    T hh[6], hi[6], id;
#pragma unroll
    for (int m = 0; m < 6; ++m) hh[m] = u[F_H + m];
    sym3_inv(hh, hi, id);
    const T tr = hi[0] * u[F_A] + hi[3] * u[F_A + 3] + hi[5] * u[F_A + 5]
                 + 2.0 * (hi[1] * u[F_A + 1] + hi[2] * u[F_A + 2] + hi[4] * u[F_A + 4]);
#pragma unroll
    for (int m = 0; m < 6; ++m) u[F_A + m] = u[F_A + m] - hh[m] * tr * (1.0 / 3.0);
    u[F_CHI] = fmax(u[F_CHI], T(min_chi));
    u[F_LAPSE] = fmax(u[F_LAPSE], T(min_lapse));
}

// Reverse sweep of this column's tape: node adjoints are consumed (reset to zero) as they are
// propagated, so the column is clean for its next point.
// The tape entries do not depend on the adjoints, so the next entry is loaded while the current
// one is applied.
__device__ __forceinline__ void rev_sweep(int entries, long long col) {
    const long long S = grf_rev::c_tape.stride;
    double* __restrict__ adj = grf_rev::c_tape.adj;
    const double2* __restrict__ w = grf_rev::c_tape.w;
    const ushort4* __restrict__ ix = grf_rev::c_tape.ix;
    if (entries <= 0) return;
    double2 pw = __ldcs(&w[(long long)(entries - 1) * S + col]);
    ushort4 o = __ldcs(&ix[(long long)(entries - 1) * S + col]);
#pragma unroll 1
    for (int n = entries - 1; n >= 0; --n) {
        const double2 pc = pw;
        const ushort4 oc = o;
        if (n > 0) {
            pw = __ldcs(&w[(long long)(n - 1) * S + col]);
            o = __ldcs(&ix[(long long)(n - 1) * S + col]);
        }
        const long long node = (long long)(kNLeaf + n) * S + col;
        const double g = adj[node];
        if (g == 0.0) continue;
        adj[node] = 0.0;
        if (oc.x != grf_rev::kNone) adj[(long long)oc.x * S + col] += pc.x * g;
        if (oc.y != grf_rev::kNone) adj[(long long)oc.y * S + col] += pc.y * g;
        if (oc.z != grf_rev::kNone) adj[(long long)oc.z * S + col] += g;
    }
}

// STAGE (0..3) is a run-time argument: one instantiation of the large pointwise map keeps the
// library's build time down (its four stage variants differ only in a few scalars and leaves).
// Thread col tapes point q0 + col of the wave into tape column col.
__global__ void __launch_bounds__(kAdjThreads, 4) adj_tape_kernel(Geom g, Coeffs c, AdjArgs a, int STAGE, long long q0) {
    const long long col = grf_rev::rev_col();
    const long long q = q0 + col;
    if (col >= grf_rev::c_tape.stride || q >= a.npts) return;
    const long long S = grf_rev::c_tape.stride;
    double* adj = grf_rev::c_tape.adj;
    const double cs = (STAGE == 0 || STAGE == 1) ? 0.5 * a.dt : (STAGE == 2 ? a.dt : a.dt * (1.0 / 6.0));
    const double wacc = (STAGE == 0) ? 1.0 : 2.0;  // weight of k_s in the accumulator (stages 0..2)
    const long long nxy = (long long)g.nx * g.ny;
    const int k = (int)(q / nxy);
    const long long rem = q - (long long)k * nxy;
    const int j = (int)(rem / g.nx), i = (int)(rem - (long long)j * g.nx);
    const long long p = gidx(g, i + NG, j + NG, k + NG);
    PointIn in;
    double kos[NFIELDS];
    gather<0>(g, a.src, p, in, kos, nullptr, nullptr, 0);
    grf_rev::s_count[threadIdx.x] = 0;
    PointInT<Rev> ir;
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) ir.v[f] = Rev(in.v[f], kLV + f);
#pragma unroll 1
    for (int m = 0; m < 24; ++m)
        for (int d = 0; d < 3; ++d) ir.d1[m][d] = Rev(in.d1[m][d], kLD1 + 3 * m + d);
#pragma unroll 1
    for (int b = 0; b < 12; ++b)
        for (int m = 0; m < 6; ++m) ir.d2[b][m] = Rev(in.d2[b][m], kLD2 + 6 * b + m);
    CoeffsT<Rev> cr;
    cr.kappa1 = c.kappa1; cr.kappa2 = c.kappa2; cr.kappa3 = c.kappa3; cr.shift_F = c.shift_F; cr.eta = c.eta;
    cr.lam = Rev(c.lam, kLLAM);
    cr.g3 = c.g3;
    cr.g2 = Rev(c.g2, kLG2);
    cr.inv_1pa = c.inv_1pa; cr.a_1pa = c.a_1pa; cr.bK = c.bK; cr.bTh = c.bTh;
    cr.beta_kind = c.beta_kind; cr.beta_kappa = c.beta_kappa; cr.decoupled = c.decoupled; cr.advection = 0;
    Rev r[NFIELDS];
    bool ok = true;
    point_rhs<Rev, Rev, -1, 0, 1>(cr, ir, r, nullptr, ok);
    if (!ok) atomicOr(a.status, 1);
    Rev out[NFIELDS];
    int knode[NFIELDS];
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        const long long o = f * g.fstride + p;
        const Rev kf = r[f] + a.ko * Rev(kos[f], kLKO + f);
        knode[f] = kf.i;
        const Rev unf = (STAGE == 0) ? ir.v[f] : Rev(a.un[o], kLUN + f);
        out[f] = (STAGE == 3) ? fma(Rev(cs), Rev(a.acc[o], kLACC + f) + kf, unf) : fma(Rev(cs), kf, unf);
    }
    if (a.enforce) enforce_point_t(out, a.min_chi, a.min_lapse);
    // seeds: the adjoint of the stage output, and (stages 0..2) of k_s through the accumulator
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        const long long o = f * g.fstride + p;
        const double sb = a.ubar[o];
        if (out[f].i >= 0 && sb != 0.0) adj[(long long)out[f].i * S + col] += sb;
        if (STAGE < 3) {
            const double ab = a.abar[o];
            if (knode[f] >= 0 && ab != 0.0) adj[(long long)knode[f] * S + col] += wacc * ab;
        }
    }
    a.count[col] = min(grf_rev::s_count[threadIdx.x], grf_rev::c_tape.cap);
}

// Sweeps tape column col (point q0 + col) and hands the leaves' adjoints to the stage's outputs:
// the values' to vbar / unbar / abar, the derivative and KO sums' to G (with periodic images),
// lambda's and g2's to the column's sums.
__global__ void __launch_bounds__(kSweepThreads, 4) adj_sweep_kernel(Geom g, AdjArgs a, int STAGE, long long q0) {
    const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long q = q0 + col;
    if (col >= grf_rev::c_tape.stride || q >= a.npts) return;
    const long long S = grf_rev::c_tape.stride;
    double* adj = grf_rev::c_tape.adj;
    auto take = [&](int leaf) {
        const long long o = (long long)leaf * S + col;
        const double x = adj[o];
        adj[o] = 0.0;
        return x;
    };
    rev_sweep(a.count[col], col);
    const long long nxy = (long long)g.nx * g.ny;
    const int k = (int)(q / nxy);
    const long long rem = q - (long long)k * nxy;
    const int j = (int)(rem / g.nx), i = (int)(rem - (long long)j * g.nx);
    const long long p = gidx(g, i + NG, j + NG, k + NG);
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        const long long o = f * g.fstride + p;
        const double vb = take(kLV + f);
        if (STAGE == 0) {
            a.unbar[o] += vb;
        } else {
            a.vbar[o] = vb;
            const double ub = take(kLUN + f);
            if (STAGE == 3) a.unbar[o] = ub;
            else a.unbar[o] += ub;
        }
        if (STAGE == 3) a.abar[o] = take(kLACC + f);
        store_with_images(g, a.G, kGKO + f, i, j, k, take(kLKO + f));
    }
#pragma unroll 1
    for (int m = 0; m < 72; ++m) store_with_images(g, a.G, m, i, j, k, take(kLD1 + m));
#pragma unroll 1
    for (int m = 0; m < 72; ++m) store_with_images(g, a.G, kGD2 + m, i, j, k, take(kLD2 + m));
    a.pbar[2 * col] += take(kLLAM);
    a.pbar[2 * col + 1] += take(kLG2);
}

// X(q) += transposed stencils of the derivative / KO adjoints at interior q:
// -D_d(G_d1) for the first derivatives, +D_dd(G) and the mixed D_a D_b(G) for the second, +KO(G_ko).
__global__ void __launch_bounds__(128) adj_transpose_kernel(Geom g, const double* __restrict__ G, double* __restrict__ X) {
    int i, j, k;
    if (!interior_thread(g, i, j, k)) return;
    const long long p = gidx(g, i + NG, j + NG, k + NG);
    const double i12 = 1.0 / (12.0 * g.dx), i12s = 1.0 / (12.0 * g.dx * g.dx);
    const long long st[3] = {1, g.pitch, g.plane};
    const long long fs = g.fstride;
#pragma unroll 1
    for (int f = 0; f < NFIELDS; ++f) {
        double acc = ko6(G + (long long)(kGKO + f) * fs, p, g.pitch, g.plane);
        if (!(f >= F_B && f < F_B + 3)) {
            const int a1 = d1slot(f);
#pragma unroll
            for (int d = 0; d < 3; ++d) acc -= fd1(G + (long long)(3 * a1 + d) * fs, p, st[d], i12);
        }
        if (has_d2(f)) {
            const double* Gb = G + (long long)(kGD2 + 6 * d2slot(f)) * fs;
            acc += fd2(Gb, p, st[0], __ldg(Gb + p), i12s);
            acc += mixed_local(Gb + fs, p, st[0], st[1], i12);
            acc += mixed_local(Gb + 2 * fs, p, st[0], st[2], i12);
            acc += fd2(Gb + 3 * fs, p, st[1], __ldg(Gb + 3 * fs + p), i12s);
            acc += mixed_local(Gb + 4 * fs, p, st[1], st[2], i12);
            acc += fd2(Gb + 5 * fs, p, st[2], __ldg(Gb + 5 * fs + p), i12s);
        }
        X[f * fs + p] += acc;
    }
}

// Trilinear sample of the sphere rule's point q: the 8 neighbours' offsets and trilinear
// weights, and the rule's weight w. Returns false if a neighbour leaves the interior.
__device__ __forceinline__ bool sphere_sample(const Geom& g, double x0, double y0, double z0, double R, double cx,
                                              double cy, double cz, int q, long long off[8], double wt[8], double& w) {
    double ux, uy, uz;
    sphere_point(q, ux, uy, uz, w);
    const double fx = (cx + R * ux - x0) / g.dx, fy = (cy + R * uy - y0) / g.dx, fz = (cz + R * uz - z0) / g.dx;
    const int i0 = (int)floor(fx), j0 = (int)floor(fy), k0 = (int)floor(fz);
    if (i0 < 0 || j0 < 0 || k0 < 0 || i0 + 1 >= g.nx || j0 + 1 >= g.ny || k0 + 1 >= g.nz) return false;
    const double tx = fx - i0, ty = fy - j0, tz = fz - k0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        off[c] = gidx(g, i0 + dx + NG, j0 + dy + NG, k0 + dz + NG);
        wt[c] = (dx ? tx : 1.0 - tx) * (dy ? ty : 1.0 - ty) * (dz ? tz : 1.0 - tz);
    }
    return true;
}

// loss += dt * sum_q w_q phi(sample q) (one thread, fixed order; the same roundings as the
// tangent-linear kernel's signal, so the two give the same bits)
__global__ void signal_kernel(Geom g, double x0, double y0, double z0, double R, double cx, double cy, double cz,
                              const double* __restrict__ s, double dt, double* loss, int* status) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double* u = s + F_PHI * g.fstride;
    double tot = 0.0;
    for (int q = 0; q < 26; ++q) {
        long long off[8];
        double wt[8], w;
        if (!sphere_sample(g, x0, y0, z0, R, cx, cy, cz, q, off, wt, w)) { atomicOr(status, 4); return; }
        double v = 0.0;
        for (int c = 0; c < 8; ++c) v = fma(wt[c], u[off[c]], v);
        tot += __dmul_rn(w, v);  // rounded product, then the sum: as the tangent kernel's signal
    }
    *loss = __fma_rn(dt, tot, *loss);
}

// ubar_phi += scale * d(sum_q w_q phi(sample q)) / d phi (one thread, fixed order)
__global__ void adj_signal_seed_kernel(Geom g, double x0, double y0, double z0, double R, double cx, double cy, double cz,
                                       double scale, double* ubar, int* status) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double* u = ubar + F_PHI * g.fstride;
    for (int q = 0; q < 26; ++q) {
        long long off[8];
        double wt[8], w;
        if (!sphere_sample(g, x0, y0, z0, R, cx, cy, cz, q, off, wt, w)) { atomicOr(status, 4); return; }
        for (int c = 0; c < 8; ++c) u[off[c]] += scale * w * wt[c];
    }
}

// out[0..1] = sum over columns of pbar (fixed order: strided partial sums, then in thread order)
__global__ void adj_param_reduce_kernel(const double* __restrict__ pbar, long long ncol, double* out) {
    __shared__ double sh[2][256];
    const int t = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (long long c = t; c < ncol; c += 256) { a += pbar[2 * c]; b += pbar[2 * c + 1]; }
    sh[0][t] = a;
    sh[1][t] = b;
    __syncthreads();
    if (t == 0) {
        double x = 0.0, y = 0.0;
        for (int r = 0; r < 256; ++r) { x += sh[0][r]; y += sh[1][r]; }
        out[0] = x;
        out[1] = y;
    }
}

// Deterministic dot product over interior points: per-block partial sums, then one block.
__global__ void dot_partial_kernel(Geom g, int f0, int f1, const double* __restrict__ x, const double* __restrict__ y,
                                   double* part) {
    __shared__ double sh[256];
    const long long n = (long long)g.nx * g.ny * g.nz * (f1 - f0);
    const long long nxy = (long long)g.nx * g.ny, nxyz = nxy * g.nz;
    double s = 0.0;
    for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
        const int f = f0 + (int)(q / nxyz);
        const long long r = q % nxyz;
        const int k = (int)(r / nxy), j = (int)((r % nxy) / g.nx), i = (int)(r % g.nx);
        const long long o = f * g.fstride + gidx(g, i + NG, j + NG, k + NG);
        s = fma(x[o], y[o], s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < 256; ++r) t += sh[r];
        part[blockIdx.x] = t;
    }
}

__global__ void dot_final_kernel(const double* part, int nb, double* out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[b];
    *out = t;
}

}  // namespace grf

using namespace grf;

namespace {

constexpr int kDotBlocks = 304;

bool adj_box_ok(const grf_box* b) {
    if (!b) return false;
    if (b->ng != NG || b->nx < 2 || b->ny < 2 || b->nz < 2 || !(b->dx > 0.0)) return false;
    if (b->pitch < (long long)b->nx + 2 * NG) return false;
    if (b->bc != GRF_BC_PERIODIC && b->bc != GRF_BC_FROZEN) return false;
    if (b->bc == GRF_BC_PERIODIC && (b->nx < NG || b->ny < NG || b->nz < NG)) return false;
    return true;
}

bool adj_params_ok(const grf_params* p) {
    if (!p) return false;
    if (p->beta_kind != GRF_BETA_LINEAR && p->beta_kind != GRF_BETA_QUADRATIC && p->beta_kind != GRF_BETA_EXPONENTIAL)
        return false;
    if (p->beta_kind == GRF_BETA_EXPONENTIAL && !(p->beta_kappa >= 0.0 && p->beta_kappa < 1e300)) return false;
    if (!(1.0 + p->a0 > 0.0) || !(1.0 + p->b0 > 0.0)) return false;
    return p->advection == 0;  // centred advection only
}

Geom adj_geom(const grf_box* b) {
    Geom g;
    g.nx = b->nx; g.ny = b->ny; g.nz = b->nz;
    g.NX = b->nx + 2 * NG; g.NY = b->ny + 2 * NG; g.NZ = b->nz + 2 * NG;
    g.ng = NG;
    g.pitch = b->pitch;
    g.plane = b->pitch * g.NY;
    g.fstride = g.plane * g.NZ;
    g.dx = b->dx;
    g.periodic = (b->bc == GRF_BC_PERIODIC);
    g.reflect = 0;
    return g;
}

Coeffs adj_coeffs(const grf_params* p) {
    Coeffs c = make_coeffs(p);
    c.advection = 0;  // centred advection only (checked by adj_params_ok)
    return c;
}

size_t sbytes(const Geom& g) { return sizeof(double) * (size_t)NFIELDS * (size_t)g.fstride; }

long long adj_cols(const Geom& g) {
    const long long npts = (long long)g.nx * g.ny * g.nz;
    const long long want = (npts + kSweepThreads - 1) / kSweepThreads * kSweepThreads;
    return want < kAdjCols ? want : kAdjCols;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout (every region 256-byte aligned):
//   status | stage region [U1 | U2 | ACC | U3] | adjoint states [W | UBn | Va | Vb | Abar] |
//   G (171 slots) | segment states (checkpoint_every) | tape partials | tape operands |
//   node adjoints | per-column parameter sums | per-column tape lengths | dot-product partials
struct Layout {
    size_t status, stage, adjs, G, seg, w, ix, adj, pbar, count, part, total;
};

Layout layout(const Geom& g, int ce) {
    const size_t sb = align256(sbytes(g));
    const long long cols = adj_cols(g);
    Layout L;
    size_t o = 0;
    L.status = o; o += 256;
    L.stage = o; o += 4 * sb;
    L.adjs = o; o += 5 * sb;
    L.G = o; o += align256(sizeof(double) * (size_t)kGSlots * (size_t)g.fstride);
    L.seg = o; o += (size_t)ce * sb;
    L.w = o; o += align256(sizeof(double2) * (size_t)kTapeCap * (size_t)cols);
    L.ix = o; o += align256(sizeof(ushort4) * (size_t)kTapeCap * (size_t)cols);
    L.adj = o; o += align256(sizeof(double) * (size_t)(kNLeaf + kTapeCap) * (size_t)cols);
    L.pbar = o; o += align256(sizeof(double) * 2 * (size_t)cols);
    L.count = o; o += align256(sizeof(int) * (size_t)cols);
    L.part = o; o += align256(sizeof(double) * kDotBlocks);
    L.total = o;
    return L;
}

bool sphere_ok(const grf_sphere* s) { return s && s->radius > 0.0 && std::isfinite(s->radius); }

int fail(cudaError_t e) { return grf::record_cuda_error(e); }

// status word of the workspace -> error code (synchronises)
int finish(int* status, cudaStream_t st) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e);
    if (h & 8) return GRF_EWORKSPACE;  // tape overflow
    if (h & 4) return GRF_EINVAL;      // sphere sample outside the interior
    if (h & 1) return GRF_ESINGULAR;
    return GRF_OK;
}

// The three stage states u_1, u_2, u_3 and the accumulator k_1 + 2 k_2 + 2 k_3 of the step from
// un, by the production stage kernels (same bits as grf_rk4_step's stages).
int recompute_stages(const grf_box* box, const Geom& g, const Coeffs& c, const grf_params* p, const double* un,
                     double* U1, double* U2, double* U3, double* ACC, double dt, int* status, cudaStream_t st) {
    const size_t sb = sbytes(g);
    if (!g.periodic) {  // the stage states carry the frozen ghosts
        for (double* U : {U1, U2, U3}) {
            cudaError_t e = cudaMemcpyAsync(U, un, sb, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return fail(e);
        }
    }
    StageArgs a;
    a.dt = dt;
    a.ko = p->sigma_ko / (64.0 * box->dx);
    a.min_chi = p->min_chi;
    a.min_lapse = p->min_lapse;
    a.enforce = p->enforce_algebraic;
    a.status = status;
    a.k0 = 0;
    a.fold = 32;
    a.un = un;
    a.acc = ACC;
    const dim3 blk(32, 4, 1), grd((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
    a.src = un; a.dst = U1;
    launch_stage(0, grd, blk, st, g, c, a);
    a.src = U1; a.dst = U2;
    launch_stage(1, grd, blk, st, g, c, a);
    a.src = U2; a.dst = U3;
    launch_stage(2, grd, blk, st, g, c, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRF_OK : fail(e);
}

}  // namespace

extern "C" {

size_t grf_adjoint_workspace_bytes(const grf_box* box, int checkpoint_every) {
    if (!adj_box_ok(box) || checkpoint_every < 1) return 0;
    return layout(adj_geom(box), checkpoint_every).total;
}

int grf_signal_forward(const grf_box* box, const grf_params* params, double* state, double dt, int nsteps,
                       const grf_sphere* sphere, int checkpoint_every, double* checkpoints, double* loss, void* ws,
                       size_t ws_bytes, grf_stream_t stream) {
    if (!adj_box_ok(box) || !adj_params_ok(params) || !state || !sphere_ok(sphere) || !loss || nsteps < 0 ||
        checkpoint_every < 1 || (nsteps > 0 && !checkpoints))
        return GRF_EINVAL;
    const Geom g = adj_geom(box);
    const Layout L = layout(g, checkpoint_every);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    int* status = (int*)(base + L.status);
    const size_t sb = sbytes(g);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), st);
    if (e != cudaSuccess) return fail(e);
    int r = grf_fill_ghosts(box, state, stream);
    if (r) return r;
    for (int n = 0; n < nsteps; ++n) {
        if (n % checkpoint_every == 0) {
            e = cudaMemcpyAsync((char*)checkpoints + (size_t)(n / checkpoint_every) * sb, state, sb,
                                cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return fail(e);
        }
        r = grf_rk4_step(box, params, state, dt, 1, base + L.stage, 3 * align256(sb), stream);
        if (r) return r;
        signal_kernel<<<1, 32, 0, st>>>(g, box->x0, box->y0, box->z0, sphere->radius, sphere->cx, sphere->cy, sphere->cz,
                                        state, dt, loss, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(e);
    }
    r = finish(status, st);
    if (r) return r;
    return grf_check_status(stream);
}

int grf_adjoint_rk4(const grf_box* box, const grf_params* params, const double* checkpoints, double dt, int nsteps,
                    const grf_sphere* sphere, int checkpoint_every, double loss_bar, double* state_bar,
                    double* param_bar, void* ws, size_t ws_bytes, grf_stream_t stream) {
    if (!adj_box_ok(box) || !adj_params_ok(params) || !sphere_ok(sphere) || !state_bar || !param_bar || nsteps < 0 ||
        checkpoint_every < 1 || (nsteps > 0 && !checkpoints) || !std::isfinite(loss_bar))
        return GRF_EINVAL;
    const Geom g = adj_geom(box);
    const Layout L = layout(g, checkpoint_every);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    const size_t sb = sbytes(g), sba = align256(sb);
    int* status = (int*)(base + L.status);
    double* U1 = (double*)(base + L.stage);
    double* U2 = (double*)(base + L.stage + sba);
    double* ACC = (double*)(base + L.stage + 2 * sba);
    double* U3 = (double*)(base + L.stage + 3 * sba);
    double* W = (double*)(base + L.adjs);
    double* UBn = (double*)(base + L.adjs + sba);
    double* Va = (double*)(base + L.adjs + 2 * sba);
    double* Vb = (double*)(base + L.adjs + 3 * sba);
    double* Abar = (double*)(base + L.adjs + 4 * sba);
    double* G = (double*)(base + L.G);
    auto seg = [&](int j) { return (double*)(base + L.seg + (size_t)j * sba); };
    const long long cols = adj_cols(g);
    double* pbar = (double*)(base + L.pbar);

    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + L.adj, 0, L.pbar - L.adj, st);  // node adjoints
    if (e == cudaSuccess) e = cudaMemsetAsync(pbar, 0, sizeof(double) * 2 * (size_t)cols, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)kGSlots * (size_t)g.fstride, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(W, state_bar, sb, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(e);
    grf_rev::Tape tape;
    tape.w = (double2*)(base + L.w);
    tape.ix = (ushort4*)(base + L.ix);
    tape.adj = (double*)(base + L.adj);
    tape.stride = cols;
    tape.cap = kTapeCap;
    tape.nleaf = kNLeaf;
    tape.status = status;
    e = cudaMemcpyToSymbolAsync(grf_rev::c_tape, &tape, sizeof(tape), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(e);

    const Coeffs c = adj_coeffs(params);
    AdjArgs a;
    a.dt = dt;
    a.ko = params->sigma_ko / (64.0 * box->dx);
    a.min_chi = params->min_chi;
    a.min_lapse = params->min_lapse;
    a.enforce = params->enforce_algebraic;
    a.status = status;
    a.npts = (long long)g.nx * g.ny * g.nz;
    a.G = G;
    a.pbar = pbar;
    a.abar = Abar;
    a.count = (int*)(base + L.count);
    const dim3 tgrd((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz), tblk(32, 4, 1);
    const int tblocks = (int)((cols + kAdjThreads - 1) / kAdjThreads);
    const int sblocks = (int)((cols + kSweepThreads - 1) / kSweepThreads);
    // one reversed stage: waves of `cols` points, each taped, then swept
    auto reverse_stage = [&](int stage) {
        for (long long q0 = 0; q0 < a.npts; q0 += cols) {
            adj_tape_kernel<<<tblocks, kAdjThreads, 0, st>>>(g, c, a, stage, q0);
            adj_sweep_kernel<<<sblocks, kSweepThreads, 0, st>>>(g, a, stage, q0);
        }
    };
    const double sx0 = box->x0, sy0 = box->y0, sz0 = box->z0;
    auto seed_signal = [&](double* ub) {
        if (loss_bar != 0.0)
            adj_signal_seed_kernel<<<1, 32, 0, st>>>(g, sx0, sy0, sz0, sphere->radius, sphere->cx, sphere->cy, sphere->cz,
                                                     loss_bar * dt, ub, status);
    };
    if (nsteps > 0) seed_signal(W);  // the signal at t_N

    const int nck = (nsteps + checkpoint_every - 1) / checkpoint_every;
    for (int ck = nck - 1; ck >= 0; --ck) {
        const int n0 = ck * checkpoint_every;
        const int n1 = (n0 + checkpoint_every < nsteps) ? n0 + checkpoint_every : nsteps;
        // the segment's states u_{n0} .. u_{n1-1}
        e = cudaMemcpyAsync(seg(0), (const char*)checkpoints + (size_t)ck * sb, sb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail(e);
        for (int jj = 1; jj < n1 - n0; ++jj) {
            e = cudaMemcpyAsync(seg(jj), seg(jj - 1), sb, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return fail(e);
            const int r = grf_rk4_step(box, params, seg(jj), dt, 1, U1, 3 * sba, stream);
            if (r) return r;
        }
        for (int n = n1 - 1; n >= n0; --n) {
            const double* un = seg(n - n0);
            int r = recompute_stages(box, g, c, params, un, U1, U2, U3, ACC, dt, status, st);
            if (r) return r;
            a.un = un;
            a.acc = ACC;
            // stage 3: u_{n+1} = E(u_n + dt/6 (acc + k_4)), k_4 = F(u_3)
            a.src = U3; a.ubar = W; a.vbar = Va; a.unbar = UBn;
            reverse_stage(3);
            adj_transpose_kernel<<<tgrd, tblk, 0, st>>>(g, G, Va);
            // stage 2: u_3 = E(u_n + dt k_3), k_3 = F(u_2)
            a.src = U2; a.ubar = Va; a.vbar = Vb;
            reverse_stage(2);
            adj_transpose_kernel<<<tgrd, tblk, 0, st>>>(g, G, Vb);
            // stage 1: u_2 = E(u_n + dt/2 k_2), k_2 = F(u_1)
            a.src = U1; a.ubar = Vb; a.vbar = Va;
            reverse_stage(1);
            adj_transpose_kernel<<<tgrd, tblk, 0, st>>>(g, G, Va);
            // stage 0: u_1 = E(u_n + dt/2 k_1), k_1 = F(u_n)
            a.src = un; a.ubar = Va; a.vbar = nullptr;
            reverse_stage(0);
            adj_transpose_kernel<<<tgrd, tblk, 0, st>>>(g, G, UBn);
            if (n >= 1) seed_signal(UBn);  // the signal at t_n
            e = cudaGetLastError();
            if (e != cudaSuccess) return fail(e);
            double* t = W; W = UBn; UBn = t;
        }
    }
    e = cudaMemcpyAsync(state_bar, W, sb, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(e);
    adj_param_reduce_kernel<<<1, 256, 0, st>>>(pbar, cols, param_bar);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e);
    const int r = finish(status, st);
    if (r) return r;
    return grf_check_status(stream);
}

int grf_state_dot(const grf_box* box, const double* x, const double* y, int field, double* out, void* ws,
                  size_t ws_bytes, grf_stream_t stream) {
    if (!adj_box_ok(box) || !x || !y || !out || field < -1 || field >= NFIELDS) return GRF_EINVAL;
    if (!ws || ws_bytes < sizeof(double) * kDotBlocks || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    const Geom g = adj_geom(box);
    cudaStream_t st = (cudaStream_t)stream;
    const int f0 = field < 0 ? 0 : field, f1 = field < 0 ? NFIELDS : field + 1;
    dot_partial_kernel<<<kDotBlocks, 256, 0, st>>>(g, f0, f1, x, y, (double*)ws);
    dot_final_kernel<<<1, 32, 0, st>>>((const double*)ws, kDotBlocks, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRF_OK : fail(e);
}

}  // extern "C"
