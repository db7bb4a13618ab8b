// CPU oracle for the modified-CCZ4 + 4-derivative scalar-tensor (4dST) evolution.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this file:
// only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm use it.
// It shares no code, header, table or helper with the CUDA library.
//
// What it computes (GRFolres, arXiv:2309.06225, section "Key features": modified moving
// puncture gauge, 4dST theory, 4th-order Runge-Kutta with 4th-order finite differences,
// periodic boundaries, constraint monitoring). The paper prints no equations; the ones
// followed here are the modified-CCZ4 / 4dST equations of the works it cites, written out
// below and in the functions that evaluate them:
//   * fields: chi, h_ij, K, A_ij, Theta, Gamma^i, lapse, shift^i, B^i, phi, Pi (27 doubles)
//   * derivatives ("Accuracy": 4th and 6th order): the box's ghost width chooses the scheme,
//     ng = 3 -> centred 4th-order first, second and mixed differences, ng = 4 -> 6th order
//   * advection terms beta^k d_k u: centred differences (params.advection = 0) or lopsided
//     differences biased one point towards the side the shift points to (advection = 1;
//     4th order: offsets -1..3, 6th order: -2..4, mirrored for beta^k < 0)
//   * 4dST sources: built COVARIANTLY. At each point the 4D Riemann tensor is assembled in
//     the basis (n, d_i) from the Gauss, Codazzi and Ricci equations, the double dual P,
//     the Gauss-Bonnet invariant, the effective stress tensor
//        8 pi T_ab = 1/2 (1 + 2 g2 X) d_a phi d_b phi + 1/2 g_ab (X + g2 X^2)
//                    - 4 P_acbd nabla^c nabla^d beta(phi)
//     and the scalar equation
//        E = (1 + 2 g2 X) box(phi) - 2 g2 d^a phi d^b phi nabla_a nabla_b phi + beta'(phi) L_GB
//     are evaluated by plain index loops.
//   * the coupled unknowns v = (d_t K_ij (6), d_t Pi) enter the Riemann tensor (Ricci
//     equation) and nabla_n nabla_n phi. The residual of the equations is affine in v, so
//     it is evaluated at v = 0 and at the 7 scaled unit vectors and the 7x7 system is
//     solved by Gaussian elimination with FULL pivoting in long double.
//   * decoupled mode (params.decoupled = 1; "Key features": 4dST without backreaction onto the
//     metric, for comparison with decoupling-limit codes): T_ab is dropped from the metric
//     equations, which become vacuum CCZ4 in the same gauge, while the scalar evolves with the
//     full scalar equation on that metric
//   * Kreiss-Oliger dissipation on all fields: sigma/(64 dx) sum_d Delta^6_d u for the 4th-order
//     scheme, -sigma/(256 dx) sum_d Delta^8_d u for the 6th-order one (both damp the grid's
//     Nyquist mode at sigma/dx per direction)
//   * classical RK4 with post-stage algebraic enforcement (trace-free A, chi and lapse floors)
//
//   * the CCZ4 equations (K, A_ij, Theta, Gamma-hat) are the 3+1 projection of the covariant
//     damped Z4 system of the modified gauge,
//        G^ab + 2 Phat_c^{d ab} nabla_d Z^c - kappa1 [2 n^(a Z^b) + kappa2 (n.Z) g^ab] = 8 pi T^ab,
//        Phat_c^{d ab} = delta_c^(a gh^b)d - 1/2 delta_c^d gh^ab,   gh^ab = g^ab - b(x) n^a n^b,
//     with Theta = -n.Z and Gamma-hat^i = Gamma-tilde^i + 2 h^ij Z_j. The auxiliary metric gh
//     multiplies the time-derivative terms of the nn and ni components by (1 + b); solving for
//     them gives the b(x) terms of d_t K, d_t Theta and d_t Gamma-hat written in ccz4_rhs. The
//     other auxiliary metric, with a(x), enters only the lapse and shift conditions.
//
// Parity unpinned (no pin fixes these independently of the equations as read): the functional
// forms a(x) = a0, b(x) = b0 (constants) and the 1+log / Gamma-driver gauge coefficients. The
// gauge conditions' form is pinned by the linearised gauge waves; the b(x) terms and the damping
// terms by the covariant Z4 projection above (tests/test_oracle_pins.py).
//
// Plain loops, no blocking, FP64 (long double only inside the linear solve).
// Build: g++ -O2 -ffp-contract=off -fopenmp -shared -fPIC (see oracle/build.py).
//
// Layout: orc_types.h holds the C types, orc_core.inc the method (on a scalar type `real`), this
// file the plain double build and its C interface. grf_oracle_tlm.cpp instantiates the same core
// on dual numbers and on complex-step numbers for the tangent-linear model.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "orc_types.h"

namespace {

typedef double real;
typedef long double real_ld;
inline double vval(double x) { return x; }
inline double vabs(double x) { return std::fabs(x); }
inline long double vabsl(long double x) { return fabsl(x); }
inline double vmax(double x, double c) { return std::max(x, c); }
inline long double to_ld(double x) { return x; }
inline double from_ld(long double x) { return (double)x; }
using std::exp;
#define ORC_PLAIN 1

#include "orc_core.inc"

}  // namespace

extern "C" {

int orc_point_rhs(const orc_params* P, const double* v, const double* d1, const double* d2, double* rhs, double* diag) {
    return point_rhs(prm_of(*P), v, d1, d2, nullptr, rhs, diag);
}

// As orc_point_rhs with the 27 advection terms beta^k d_k u given (adv).
int orc_point_rhs_adv(const orc_params* P, const double* v, const double* d1, const double* d2, const double* adv,
                      double* rhs, double* diag) {
    return point_rhs(prm_of(*P), v, d1, d2, adv, rhs, diag);
}

void orc_point_constraints(const orc_params* P, const double* v, const double* d1, const double* d2, double* out4) {
    point_constraints(prm_of(*P), v, d1, d2, out4);
}

// Psi_4 at one point: the coupled system is solved as for the right-hand side, the Riemann tensor
// assembled with the solved d_t K_ij. xyz: coordinates relative to the origin of the triad.
void orc_point_psi4(const orc_params* P, const double* v, const double* d1, const double* d2, const double* xyz,
                    double* out2) {
    double rhs[NF], diag[64];
    point_rhs(prm_of(*P), v, d1, d2, nullptr, rhs, diag);
    static thread_local Conf c;
    conf_setup(v, d1, d2, nullptr, c);
    double u[3][3];
    for (int m = 0; m < 6; ++m) u[SYM_I[m]][SYM_J[m]] = u[SYM_J[m]][SYM_I[m]] = diag[11 + m];
    Src s;
    sources(prm_of(*P), c.p, c.G, u, diag[17], s);
    weyl_psi4(c.p, s, xyz, out2);
}

// Psi_4 at the interior points (ghosts of s valid): out[2][nz][ny][nx], coordinates
// x = x0 + i dx etc. relative to the origin.
void orc_psi4(const orc_box* b, const orc_params* P, const double* s, double* out) {
    Grid g(*b);
    const long long npt = (long long)b->nx * b->ny * b->nz;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < b->nz; ++k)
        for (int j = 0; j < b->ny; ++j)
            for (int i = 0; i < b->nx; ++i) {
                double v[NF], d1[NF * 3], d2[NF * 6], o[2];
                point_derivs(g, s, b->dx, i + g.ng, j + g.ng, k + g.ng, v, d1, d2);
                const double xyz[3] = {b->x0 + i * b->dx, b->y0 + j * b->dx, b->z0 + k * b->dx};
                orc_point_psi4(P, v, d1, d2, xyz, o);
                long long p = ((long long)k * b->ny + j) * b->nx + i;
                out[p] = o[0];
                out[npt + p] = o[1];
            }
}

// Physical 3+1 interface for the 4D brute-force checks. phys: g(6) dg(3x6) ddg(6x6)
// K(6) dK(3x6) alpha dalpha(3) ddalpha(6) beta(3) dbeta(3x3, [j][i] = d_j beta^i) phi dphi(3)
// ddphi(6) Pi dPi(3)  (120 doubles; symmetric pairs in the order 11,12,13,22,23,33).
// out: 8pi rho, 8pi S_i(3), 8pi S_ij(6), L_GB, E, R_ij(6), R  (19 doubles)
// With xyz_psi4 non-null, out[19], out[20] receive Psi_4 for the triad at those coordinates.
void orc_phys_sources_psi4(const orc_params* P, const double* phys, const double* u6, double w, const double* xyz_psi4,
                           double* out) {
    Phys p;
    const double* q = phys;
    for (int m = 0; m < 6; ++m) p.g[SYM_I[m]][SYM_J[m]] = p.g[SYM_J[m]][SYM_I[m]] = q[m];
    q += 6;
    for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 6; ++m) p.dg[k][SYM_I[m]][SYM_J[m]] = p.dg[k][SYM_J[m]][SYM_I[m]] = q[k * 6 + m];
    q += 18;
    for (int kl = 0; kl < 6; ++kl)
        for (int m = 0; m < 6; ++m) {
            double x = q[kl * 6 + m];
            int k = SYM_I[kl], l = SYM_J[kl], i = SYM_I[m], j = SYM_J[m];
            p.ddg[k][l][i][j] = p.ddg[k][l][j][i] = p.ddg[l][k][i][j] = p.ddg[l][k][j][i] = x;
        }
    q += 36;
    for (int m = 0; m < 6; ++m) p.K[SYM_I[m]][SYM_J[m]] = p.K[SYM_J[m]][SYM_I[m]] = q[m];
    q += 6;
    for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 6; ++m) p.dK[k][SYM_I[m]][SYM_J[m]] = p.dK[k][SYM_J[m]][SYM_I[m]] = q[k * 6 + m];
    q += 18;
    p.alpha = *q++;
    for (int k = 0; k < 3; ++k) p.dalpha[k] = *q++;
    for (int m = 0; m < 6; ++m) p.ddalpha[SYM_I[m]][SYM_J[m]] = p.ddalpha[SYM_J[m]][SYM_I[m]] = q[m];
    q += 6;
    for (int k = 0; k < 3; ++k) p.beta[k] = *q++;
    for (int j = 0; j < 3; ++j) for (int i = 0; i < 3; ++i) p.dbeta[j][i] = q[j * 3 + i];
    q += 9;
    p.phi = *q++;
    for (int k = 0; k < 3; ++k) p.dphi[k] = *q++;
    for (int m = 0; m < 6; ++m) p.ddphi[SYM_I[m]][SYM_J[m]] = p.ddphi[SYM_J[m]][SYM_I[m]] = q[m];
    q += 6;
    p.Pi = *q++;
    for (int k = 0; k < 3; ++k) p.dPi[k] = *q++;
    p.bdPi = 0;
    for (int k = 0; k < 3; ++k) p.bdPi += p.beta[k] * p.dPi[k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            p.bdK[i][j] = 0;
            for (int k = 0; k < 3; ++k) p.bdK[i][j] += p.beta[k] * p.dK[k][i][j];
        }
    Geo G;
    geometry(p, G);
    double u[3][3];
    for (int m = 0; m < 6; ++m) u[SYM_I[m]][SYM_J[m]] = u[SYM_J[m]][SYM_I[m]] = u6[m];
    Src s;
    sources(prm_of(*P), p, G, u, w, s);
    out[0] = s.rho8;
    for (int i = 0; i < 3; ++i) out[1 + i] = s.S8[i];
    for (int m = 0; m < 6; ++m) out[4 + m] = s.Sij8[SYM_I[m]][SYM_J[m]];
    out[10] = s.LGB;
    out[11] = s.E;
    for (int m = 0; m < 6; ++m) out[12 + m] = G.Ric[SYM_I[m]][SYM_J[m]];
    out[18] = G.Rs;
    if (xyz_psi4) weyl_psi4(p, s, xyz_psi4, out + 19);
}

void orc_phys_sources(const orc_params* P, const double* phys, const double* u6, double w, double* out) {
    orc_phys_sources_psi4(P, phys, u6, w, nullptr, out);
}

int orc_solve(int n, const double* M, const double* r, double* x) { return solve_full_pivot(n, M, r, x); }

void orc_fill_ghosts(const orc_box* b, double* s) {
    fill_bc(*b, Grid(*b), s);
}

// First and second derivatives of every field at every interior point:
// d1[f][d][k][j][i], d2[f][m][k][j][i] (interior indices, m in 11,12,13,22,23,33 order).
void orc_derivs(const orc_box* b, const double* s, double* d1out, double* d2out) {
    Grid g(*b);
    const long long npt = (long long)b->nx * b->ny * b->nz;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < b->nz; ++k)
        for (int j = 0; j < b->ny; ++j)
            for (int i = 0; i < b->nx; ++i) {
                double v[NF], d1[NF * 3], d2[NF * 6];
                point_derivs(g, s, b->dx, i + g.ng, j + g.ng, k + g.ng, v, d1, d2);
                long long p = ((long long)k * b->ny + j) * b->nx + i;
                for (int f = 0; f < NF; ++f) {
                    for (int d = 0; d < 3; ++d) d1out[(f * 3 + d) * npt + p] = d1[f * 3 + d];
                    for (int m = 0; m < 6; ++m) d2out[(f * 6 + m) * npt + p] = d2[f * 6 + m];
                }
            }
}

// Lopsided advection terms of every field at every interior point: adv[f][k][j][i].
void orc_adv_lopsided(const orc_box* b, const double* s, double* out) {
    Grid g(*b);
    const long long npt = (long long)b->nx * b->ny * b->nz;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < b->nz; ++k)
        for (int j = 0; j < b->ny; ++j)
            for (int i = 0; i < b->nx; ++i) {
                double a[NF];
                point_adv_lopsided(g, s, b->dx, i + g.ng, j + g.ng, k + g.ng, a);
                long long p = ((long long)k * b->ny + j) * b->nx + i;
                for (int f = 0; f < NF; ++f) out[f * npt + p] = a[f];
            }
}

// rhs (ghosted layout) <- right-hand side at interior points, including KO dissipation, and for
// Sommerfeld boxes the radiative right-hand side at every ghost point.
// The ghosts of s must be valid. Returns 0, or -5 if some point's linear solve was singular.
int orc_rhs(const orc_box* b, const orc_params* P, const double* s, double* rhs, int with_ko) {
    return rhs_box(*b, prm_of(*P), s, rhs, with_ko);
}

// rhs += the box's scheme's Kreiss-Oliger term on interior points (ghosts of s must be valid):
// sigma/(64 dx) sum_d Delta^6_d s (ng = 3) or -sigma/(256 dx) sum_d Delta^8_d s (ng = 4).
void orc_ko(const orc_box* b, double sigma, const double* s, double* rhs) {
    Grid g(*b);
    const double c = ko_factor(b->ng, sigma, b->dx);
#pragma omp parallel for collapse(2)
    for (int k = g.ng; k < g.ng + g.nz; ++k)
        for (int j = g.ng; j < g.ng + g.ny; ++j)
            for (int i = g.ng; i < g.ng + g.nx; ++i)
                for (int f = 0; f < NF; ++f) rhs[g.at(f, i, j, k)] += c * ko_point(g, s, f, i, j, k);
}

void orc_enforce(const orc_box* b, const orc_params* P, double* s) { enforce(Grid(*b), prm_of(*P), s); }

// Classical RK4 of the box (rk4_box above): nsteps steps in place, ghosts refilled by the box's
// boundary type. Returns 0, or -5 if some point's linear solve was singular.
int orc_rk4(const orc_box* b, const orc_params* P, double* s, double dt, int nsteps) {
    return rk4_box(*b, prm_of(*P), s, dt, nsteps, nullptr, nullptr);
}

// The same evolution with the sphere-averaged scalar signal: *L = sum over the steps of
// dt * sum_q w_q phi(c + R xhat_q) (sphere = {R, cx, cy, cz}). Returns -4 if a sample point's
// trilinear neighbours leave the interior.
int orc_rk4_signal(const orc_box* b, const orc_params* P, double* s, double dt, int nsteps, const double* sphere,
                   double* L) {
    const Sphere sp = {sphere[0], {sphere[1], sphere[2], sphere[3]}};
    *L = 0.0;
    return rk4_box(*b, prm_of(*P), s, dt, nsteps, &sp, L);
}

// ------------------------------------------------------------------------------------
// Waveform extraction on spheres ("Diagnostics": tensor and scalar waveforms): modes
//   a_lm = integral over the sphere of f(c + R n) conj(sY_lm(theta, phi)) dOmega,
// theta from the z axis, phi from x towards y, f = f_re + i f_im a field of the grid.
// Quadrature: Gauss-Legendre in cos(theta) (ntheta nodes) times nphi equally spaced phi.
// Interpolation: tensor product of 4-point Lagrange polynomials (cubic, 4th order) on the
// points i0-1 .. i0+2 around the sample along each axis.
// ------------------------------------------------------------------------------------

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n (three-term recurrence).
void orc_gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = z;  // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = n == 0 ? 1.0 : (n == 1 ? z : p1), pm = n == 1 ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Spin-weighted spherical harmonic sY_lm (Goldberg et al.'s sum formula, Condon-Shortley phase;
// s = 0 is the ordinary Y_lm):
//   sY_lm = (-1)^m sqrt((l+m)! (l-m)! (2l+1) / (4 pi (l+s)! (l-s)!)) sin^{2l}(theta/2)
//           sum_r C(l-s, r) C(l+s, r+s-m) (-1)^{l-r-s} cot^{2r+s-m}(theta/2) e^{i m phi}
void orc_sylm(int s, int l, int m, double theta, double phi, double* re, double* im) {
    auto fact = [](int n) { double f = 1; for (int k = 2; k <= n; ++k) f *= k; return f; };
    auto binom = [&](int n, int k) { return (k < 0 || k > n) ? 0.0 : fact(n) / (fact(k) * fact(n - k)); };
    if (l < std::abs(s) || std::abs(m) > l) { *re = *im = 0; return; }
    const double pre = ((m & 1) ? -1.0 : 1.0) *
                       std::sqrt(fact(l + m) * fact(l - m) * (2 * l + 1) / (4 * M_PI * fact(l + s) * fact(l - s)));
    const double ct = 1.0 / std::tan(0.5 * theta);
    double sum = 0;
    for (int r = 0; r <= l - s; ++r) {
        const double c = binom(l - s, r) * binom(l + s, r + s - m);
        if (c == 0) continue;
        sum += c * (((l - r - s) & 1) ? -1.0 : 1.0) * std::pow(ct, 2 * r + s - m);
    }
    const double a = pre * std::pow(std::sin(0.5 * theta), 2 * l) * sum;
    *re = a * std::cos(m * phi);
    *im = a * std::sin(m * phi);
}

// 4-point Lagrange interpolation of the field f (ghosted layout of box b) at point (x, y, z)
double interp_lagrange4(const orc_box& b, const Grid& g, const double* f, double x, double y, double z) {
    const double p[3] = {(x - b.x0) / b.dx + g.ng, (y - b.y0) / b.dx + g.ng, (z - b.z0) / b.dx + g.ng};
    int i0[3];
    double L[3][4];
    for (int d = 0; d < 3; ++d) {
        i0[d] = (int)std::floor(p[d]);
        const double t = p[d] - i0[d];
        L[d][0] = -t * (t - 1) * (t - 2) / 6.0;
        L[d][1] = (t + 1) * (t - 1) * (t - 2) / 2.0;
        L[d][2] = -(t + 1) * t * (t - 2) / 2.0;
        L[d][3] = (t + 1) * t * (t - 1) / 6.0;
    }
    double v = 0;
    for (int c = 0; c < 4; ++c)
        for (int bb = 0; bb < 4; ++bb)
            for (int a = 0; a < 4; ++a)
                v += L[0][a] * L[1][bb] * L[2][c] * f[g.at(0, i0[0] - 1 + a, i0[1] - 1 + bb, i0[2] - 1 + c)];
    return v;
}

// The interpolant of a single ghosted field at n points (xyz[3 n]).
void orc_interp(const orc_box* b, const double* f, int n, const double* xyz, double* out) {
    Grid g(*b);
    for (int q = 0; q < n; ++q) out[q] = interp_lagrange4(*b, g, f, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2]);
}

// modes[2 (l^2 + l + m) + {0, 1}] for l = 0 .. lmax, m = -l .. l (zero for l < |s|). f_im may be
// null (a real field). Returns -1 when a stencil would leave the ghosted box.
int orc_extract_modes(const orc_box* b, const double* f_re, const double* f_im, int spin, double R, double cx,
                      double cy, double cz, int ntheta, int nphi, int lmax, double* modes) {
    Grid g(*b);
    std::vector<double> mu(ntheta), w(ntheta);
    orc_gauss_legendre(ntheta, mu.data(), w.data());
    const int nm = (lmax + 1) * (lmax + 1);
    for (int q = 0; q < 2 * nm; ++q) modes[q] = 0;
    const int N[3] = {g.NX, g.NY, g.NZ};
    const double o[3] = {b->x0, b->y0, b->z0};
    for (int i = 0; i < ntheta; ++i) {
        const double th = std::acos(mu[i]);
        for (int j = 0; j < nphi; ++j) {
            const double ph = 2.0 * M_PI * j / nphi;
            const double x[3] = {cx + R * std::sin(th) * std::cos(ph), cy + R * std::sin(th) * std::sin(ph),
                                 cz + R * mu[i]};
            for (int d = 0; d < 3; ++d) {
                const int i0 = (int)std::floor((x[d] - o[d]) / b->dx + g.ng);
                if (i0 - 1 < 0 || i0 + 2 > N[d] - 1) return -1;
            }
            const double fr = interp_lagrange4(*b, g, f_re, x[0], x[1], x[2]);
            const double fi = f_im ? interp_lagrange4(*b, g, f_im, x[0], x[1], x[2]) : 0.0;
            const double dO = w[i] * 2.0 * M_PI / nphi;
            for (int l = 0; l <= lmax; ++l)
                for (int m = -l; m <= l; ++m) {
                    double yr, yi;
                    orc_sylm(spin, l, m, th, ph, &yr, &yi);
                    const int q = l * l + l + m;
                    // (fr + i fi) (yr - i yi)
                    modes[2 * q] += dO * (fr * yr + fi * yi);
                    modes[2 * q + 1] += dO * (fi * yr - fr * yi);
                }
        }
    }
    return 0;
}

// Hamiltonian and momentum constraints at interior points: out[4][nz][ny][nx] (ghosts valid).
void orc_point_energy(const orc_params* P, const double* v, const double* d1, const double* d2, double* out3) {
    point_energy(prm_of(*P), v, d1, d2, out3);
}

// Energy densities of the three scalar terms at interior points: out[3][nz][ny][nx] (ghosts valid).
void orc_energy_densities(const orc_box* b, const orc_params* P, const double* s, double* out) {
    Grid g(*b);
    const long long npt = (long long)b->nx * b->ny * b->nz;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < b->nz; ++k)
        for (int j = 0; j < b->ny; ++j)
            for (int i = 0; i < b->nx; ++i) {
                double v[NF], d1[NF * 3], d2[NF * 6], o[3];
                point_derivs(g, s, b->dx, i + g.ng, j + g.ng, k + g.ng, v, d1, d2);
                point_energy(prm_of(*P), v, d1, d2, o);
                long long p = ((long long)k * b->ny + j) * b->nx + i;
                for (int m = 0; m < 3; ++m) out[m * npt + p] = o[m];
            }
}

// Hyperbolicity diagnostics at one point (point_hyperbolicity) and at every interior point:
// out[4][nz][ny][nx] (the ghosts of s must be valid).
void orc_point_hyperbolicity(const orc_params* P, const double* v, const double* d1, const double* d2, double* out4) {
    point_hyperbolicity(prm_of(*P), v, d1, d2, out4);
}

// The normalised 7 x 7 matrix of the coupled system at one point (row-major, 49 doubles).
void orc_point_system(const orc_params* P, const double* v, const double* d1, const double* d2, double* out49) {
    point_system(prm_of(*P), v, d1, d2, out49);
}

void orc_hyperbolicity(const orc_box* b, const orc_params* P, const double* s, double* out) {
    Grid g(*b);
    const long long npt = (long long)b->nx * b->ny * b->nz;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < b->nz; ++k)
        for (int j = 0; j < b->ny; ++j)
            for (int i = 0; i < b->nx; ++i) {
                double v[NF], d1[NF * 3], d2[NF * 6], o[4];
                point_derivs(g, s, b->dx, i + g.ng, j + g.ng, k + g.ng, v, d1, d2);
                point_hyperbolicity(prm_of(*P), v, d1, d2, o);
                long long p = ((long long)k * b->ny + j) * b->nx + i;
                for (int m = 0; m < 4; ++m) out[m * npt + p] = o[m];
            }
}

void orc_constraints(const orc_box* b, const orc_params* P, const double* s, double* out) {
    Grid g(*b);
    const long long npt = (long long)b->nx * b->ny * b->nz;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < b->nz; ++k)
        for (int j = 0; j < b->ny; ++j)
            for (int i = 0; i < b->nx; ++i) {
                double v[NF], d1[NF * 3], d2[NF * 6], o[4];
                point_derivs(g, s, b->dx, i + g.ng, j + g.ng, k + g.ng, v, d1, d2);
                point_constraints(prm_of(*P), v, d1, d2, o);
                long long p = ((long long)k * b->ny + j) * b->nx + i;
                for (int m = 0; m < 4; ++m) out[m * npt + p] = o[m];
            }
}

}  // extern "C"
