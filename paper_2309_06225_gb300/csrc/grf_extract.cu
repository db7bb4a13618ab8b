// Waveform extraction on spheres ("Diagnostics": tensor and scalar waveforms):
//   a_lm = integral over the sphere of f(c + R n) conj(sY_lm(theta, phi)) dOmega,
// theta from the z axis, phi from x towards y, spin weight s = 0 (scalar waveforms) or -2
// (tensor waveforms, from the Weyl scalar Psi_4), f = f_re + i f_im a field of the grid.
//
// Quadrature: Gauss-Legendre in cos(theta) (ntheta nodes) times nphi equally spaced phi, so
// a_lm = sum_i w_i A_lm(theta_i) F_m(theta_i) with the ring sums
//   F_m(theta) = (2 pi / nphi) sum_j f(theta, phi_j) e^{-i m phi_j}
// and sY_lm = A_lm(theta) e^{i m phi}. The field is interpolated with the tensor product of
// 4-point Lagrange polynomials (cubic, 4th order) on the points i0-1 .. i0+2 around the sample.
// Three launches, all sums in a fixed order: the Gauss-Legendre rule (one thread per node), the
// ring sums (one block per ring: the ring's samples into shared memory, then one thread per m),
// the modes (one thread per (l, m)).
#include <cstdint>

#include <math_constants.h>

#include "grf.h"
#include "grf_kernels.cuh"
#include "grf_launch.h"

namespace grf {

constexpr int kMaxNphi = 2048;
constexpr int kMaxLmax = 12;
constexpr int kMaxNtheta = 512;

// Node i of the n-point Gauss-Legendre rule: Newton's method on P_n from the asymptotic guess.
__global__ void gauss_legendre_kernel(int n, double* __restrict__ mu, double* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double z = cospi((i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double pn = p1, pm = n == 1 ? 1.0 : p0;  // P_n, P_{n-1}
        dp = n * (z * pn - pm) / (z * z - 1.0);
        const double dz = pn / dp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    mu[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
}

struct SphereArgs {
    double R, cx, cy, cz;
    double x0, y0, z0;  // coordinates of interior point (0, 0, 0)
    int ntheta, nphi, lmax, spin;
};

// Cubic Lagrange interpolant of one ghosted field at (x, y, z). The host has checked that the
// stencil lies in the box; the clamp only keeps a rounding at the edge inside the buffer.
__device__ __forceinline__ double interp4(const Geom& g, const double* __restrict__ f, const SphereArgs& s, double x,
                                          double y, double z) {
    const double p[3] = {(x - s.x0) / g.dx + g.ng, (y - s.y0) / g.dx + g.ng, (z - s.z0) / g.dx + g.ng};
    const int N[3] = {g.NX, g.NY, g.NZ};
    int i0[3];
    double L[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int c = (int)floor(p[d]);
        i0[d] = min(max(c, 1), N[d] - 3);
        const double t = p[d] - c;
        L[d][0] = -t * (t - 1.0) * (t - 2.0) * (1.0 / 6.0);
        L[d][1] = (t + 1.0) * (t - 1.0) * (t - 2.0) * 0.5;
        L[d][2] = -(t + 1.0) * t * (t - 2.0) * 0.5;
        L[d][3] = (t + 1.0) * t * (t - 1.0) * (1.0 / 6.0);
    }
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double vb = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const double* row = f + gidx(g, i0[0] - 1, i0[1] - 1 + b, i0[2] - 1 + c);
            const double va = L[0][0] * __ldg(row) + L[0][1] * __ldg(row + 1) + L[0][2] * __ldg(row + 2) +
                              L[0][3] * __ldg(row + 3);
            vb = fma(L[1][b], va, vb);
        }
        v = fma(L[2][c], vb, v);
    }
    return v;
}

// One block per ring theta_i: its nphi samples into shared memory, then F_m for m = -lmax .. lmax
// (thread lmax + m), written to F[i][lmax + m] (re, im).
__global__ void __launch_bounds__(256) ring_sums_kernel(Geom g, const double* __restrict__ fre,
                                                        const double* __restrict__ fim, SphereArgs s,
                                                        const double* __restrict__ mu, double* __restrict__ F) {
    __shared__ double sre[kMaxNphi], sim[kMaxNphi];
    const int i = blockIdx.x;
    const double ct = mu[i], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    for (int j = threadIdx.x; j < s.nphi; j += blockDim.x) {
        double sp, cp;
        sincospi(2.0 * j / s.nphi, &sp, &cp);
        const double x = s.cx + s.R * st * cp, y = s.cy + s.R * st * sp, z = s.cz + s.R * ct;
        sre[j] = interp4(g, fre, s, x, y, z);
        sim[j] = fim ? interp4(g, fim, s, x, y, z) : 0.0;
    }
    __syncthreads();
    const int nm = 2 * s.lmax + 1;
    if ((int)threadIdx.x >= nm) return;
    const int m = (int)threadIdx.x - s.lmax;
    double ar = 0.0, ai = 0.0;
    for (int j = 0; j < s.nphi; ++j) {
        double sp, cp;
        sincospi(2.0 * m * j / s.nphi, &sp, &cp);  // e^{-i m phi_j} = cp - i sp
        ar = fma(sre[j], cp, fma(sim[j], sp, ar));
        ai = fma(sim[j], cp, fma(-sre[j], sp, ai));
    }
    const double dphi = 2.0 * CUDART_PI / s.nphi;
    F[2 * ((long long)i * nm + m + s.lmax)] = ar * dphi;
    F[2 * ((long long)i * nm + m + s.lmax) + 1] = ai * dphi;
}

// A_lm(theta) of sY_lm = A_lm(theta) e^{i m phi} (Goldberg et al.'s sum, Condon-Shortley phase).
__device__ double sylm_theta(int s, int l, int m, double ct) {
    if (l < abs(s) || abs(m) > l) return 0.0;
    auto fact = [](int n) { double f = 1.0; for (int k = 2; k <= n; ++k) f *= k; return f; };
    auto binom = [&](int n, int k) { return (k < 0 || k > n) ? 0.0 : fact(n) / (fact(k) * fact(n - k)); };
    const double pre = ((m & 1) ? -1.0 : 1.0) *
                       sqrt(fact(l + m) * fact(l - m) * (2 * l + 1) / (4.0 * CUDART_PI * fact(l + s) * fact(l - s)));
    // sin^2(theta/2) = (1 - cos theta)/2, cot(theta/2) = sqrt((1 + cos theta)/(1 - cos theta))
    const double s2 = 0.5 * (1.0 - ct), cot = sqrt((1.0 + ct) / (1.0 - ct));
    double sum = 0.0;
    for (int r = 0; r <= l - s; ++r) {
        const double c = binom(l - s, r) * binom(l + s, r + s - m);
        if (c == 0.0) continue;
        sum += c * (((l - r - s) & 1) ? -1.0 : 1.0) * pow(cot, (double)(2 * r + s - m));
    }
    return pre * pow(s2, (double)l) * sum;
}

// a_lm = sum_i w_i A_lm(theta_i) F_m(theta_i); one thread per (l, m), q = l^2 + l + m.
__global__ void modes_kernel(SphereArgs s, const double* __restrict__ mu, const double* __restrict__ w,
                             const double* __restrict__ F, double* __restrict__ modes) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (s.lmax + 1) * (s.lmax + 1)) return;
    const int l = (int)sqrt((double)q + 0.5);
    const int m = q - l * l - l;
    const int nm = 2 * s.lmax + 1;
    double ar = 0.0, ai = 0.0;
    for (int i = 0; i < s.ntheta; ++i) {
        const double a = w[i] * sylm_theta(s.spin, l, m, mu[i]);
        ar = fma(a, F[2 * ((long long)i * nm + m + s.lmax)], ar);
        ai = fma(a, F[2 * ((long long)i * nm + m + s.lmax) + 1], ai);
    }
    modes[2 * q] = ar;
    modes[2 * q + 1] = ai;
}

}  // namespace grf

namespace {

using namespace grf;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct ExtractLayout {
    size_t mu, w, F, modes, total;
};

ExtractLayout extract_layout(int ntheta, int lmax) {
    ExtractLayout L;
    L.mu = 0;
    L.w = align256(sizeof(double) * ntheta);
    L.F = L.w + align256(sizeof(double) * ntheta);
    L.modes = L.F + align256(sizeof(double) * 2 * (size_t)ntheta * (2 * lmax + 1));
    L.total = L.modes + align256(sizeof(double) * 2 * (size_t)(lmax + 1) * (lmax + 1));
    return L;
}

bool extract_args_ok(int spin, int ntheta, int nphi, int lmax) {
    return (spin == 0 || spin == -2) && ntheta >= 1 && ntheta <= kMaxNtheta && nphi >= 1 && nphi <= kMaxNphi &&
           lmax >= 0 && lmax <= kMaxLmax;
}

}  // namespace

extern "C" size_t grf_extract_workspace_bytes(int ntheta, int lmax) {
    if (!extract_args_ok(0, ntheta, 1, lmax)) return 0;
    return extract_layout(ntheta, lmax).total;
}

namespace grf {

int extract_modes(const grf_box* box, const Geom& g, const double* f_re, const double* f_im, int spin,
                  const grf_sphere* sphere, int ntheta, int nphi, int lmax, double* modes_host, void* ws,
                  size_t ws_bytes, cudaStream_t st) {
    if (!f_re || !sphere || !modes_host || !extract_args_ok(spin, ntheta, nphi, lmax) || !(sphere->radius > 0.0))
        return GRF_EINVAL;
    // every sample's 4-point stencil inside the ghosted box: index-space bounds of the sphere's
    // bounding box within [1, N - 3], with a margin for rounding
    const double c[3] = {sphere->cx, sphere->cy, sphere->cz}, o[3] = {box->x0, box->y0, box->z0};
    const int N[3] = {g.NX, g.NY, g.NZ};
    for (int d = 0; d < 3; ++d) {
        const double lo = (c[d] - sphere->radius - o[d]) / box->dx + box->ng;
        const double hi = (c[d] + sphere->radius - o[d]) / box->dx + box->ng;
        if (!(lo >= 1.0 + 1e-9) || !(hi <= N[d] - 3 - 1e-9)) return GRF_EINVAL;
    }
    const ExtractLayout L = extract_layout(ntheta, lmax);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & 255)) return GRF_EWORKSPACE;
    char* base = (char*)ws;
    double* mu = (double*)(base + L.mu);
    double* w = (double*)(base + L.w);
    double* F = (double*)(base + L.F);
    double* modes = (double*)(base + L.modes);
    SphereArgs s;
    s.R = sphere->radius; s.cx = c[0]; s.cy = c[1]; s.cz = c[2];
    s.x0 = o[0]; s.y0 = o[1]; s.z0 = o[2];
    s.ntheta = ntheta; s.nphi = nphi; s.lmax = lmax; s.spin = spin;
    gauss_legendre_kernel<<<(ntheta + 127) / 128, 128, 0, st>>>(ntheta, mu, w);
    ring_sums_kernel<<<ntheta, 256, 0, st>>>(g, f_re, f_im, s, mu, F);
    const int nq = (lmax + 1) * (lmax + 1);
    modes_kernel<<<(nq + 63) / 64, 64, 0, st>>>(s, mu, w, F, modes);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(modes_host, modes, sizeof(double) * 2 * nq, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? GRF_OK : record_cuda_error(e);
}

}  // namespace grf
