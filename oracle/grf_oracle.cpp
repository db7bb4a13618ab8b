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

#include <cmath>
#include <cstring>
#include <cstdlib>
#include <vector>
#include <algorithm>

extern "C" {

typedef struct {
    double kappa1, kappa2, kappa3;
    double shift_F, eta;
    double a0, b0;
    double lam, g2;
    double sigma_ko, min_chi, min_lapse;
    int beta_kind;          // 0: beta = lam*phi ; 1: beta = lam*phi^2/2 ;
                            // 2: beta = lam/(2 kappa) (1 - exp(-kappa phi^2))
    int enforce_algebraic;  // 1: trace-free A, chi/lapse floors after every RK stage
    int decoupled;          // 1: no backreaction: the metric evolves by vacuum CCZ4, the scalar on it
    int advection;          // 0: centred advection derivatives; 1: lopsided (upwind-biased)
    double beta_kappa;      // kappa of the exponential coupling (beta_kind 2)
} orc_params;

typedef struct {
    int nx, ny, nz, ng;     // interior points per axis, ghost layers (3: 4th order, 4: 6th order)
    double dx;
    double x0, y0, z0;      // coordinate of interior point 0 (unused by the operator itself)
    int bc;                 // 0 periodic (ghosts refilled by wrap), 1 frozen (ghosts kept),
                            // 2 mirror planes at the three low faces (high-face ghosts kept),
                            // 3 extrapolating (ghosts refilled by linear extrapolation),
                            // 4 Sommerfeld (ghosts evolved by the radiative condition),
                            // 5 mirror planes at the low faces, Sommerfeld at the high faces
    int pad_;
} orc_box;

}  // extern "C"

namespace {

const int NF = 27;
const int F_CHI = 0, F_H = 1, F_K = 7, F_A = 8, F_TH = 14, F_GAM = 15, F_LAPSE = 18,
          F_SHIFT = 19, F_B = 22, F_PHI = 25, F_PI = 26;
const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
const int SYM_I[6] = {0, 0, 0, 1, 1, 2};
const int SYM_J[6] = {0, 1, 2, 1, 2, 2};

void inv3(const double a[3][3], double out[3][3]) {
    double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
    double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
    double id = 1.0 / det;
    out[0][0] = c00 * id;
    out[1][0] = c01 * id;
    out[2][0] = c02 * id;
    out[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
    out[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
    out[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * id;
    out[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
    out[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
    out[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
}

// Gaussian elimination with full pivoting, long double. Returns 0, or -1 if singular.
int solve_full_pivot(int n, const double* M, const double* r, double* x) {
    long double A[8][9];
    int col[8];
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) A[i][j] = M[i * n + j];
        A[i][n] = r[i];
        col[i] = i;
    }
    long double scale = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) scale = std::max(scale, fabsl(A[i][j]));
    for (int k = 0; k < n; ++k) {
        int pi = k, pj = k;
        long double best = -1;
        for (int i = k; i < n; ++i)
            for (int j = k; j < n; ++j)
                if (fabsl(A[i][j]) > best) { best = fabsl(A[i][j]); pi = i; pj = j; }
        if (!(best > 1e-300L * scale) || best == 0) return -1;
        if (pi != k)
            for (int j = 0; j <= n; ++j) std::swap(A[k][j], A[pi][j]);
        if (pj != k) {
            for (int i = 0; i < n; ++i) std::swap(A[i][k], A[i][pj]);
            std::swap(col[k], col[pj]);
        }
        for (int i = k + 1; i < n; ++i) {
            long double f = A[i][k] / A[k][k];
            for (int j = k; j <= n; ++j) A[i][j] -= f * A[k][j];
        }
    }
    long double y[8];
    for (int i = n - 1; i >= 0; --i) {
        long double s = A[i][n];
        for (int j = i + 1; j < n; ++j) s -= A[i][j] * y[j];
        y[i] = s / A[i][i];
    }
    for (int i = 0; i < n; ++i) x[col[i]] = (double)y[i];
    return 0;
}

// ------------------------------------------------------------------------------------
// Physical 3+1 data at one point and the geometry derived from it.
// ------------------------------------------------------------------------------------
struct Phys {
    double g[3][3], dg[3][3][3], ddg[3][3][3][3];  // dg[k][i][j] = d_k g_ij, ddg[k][l][i][j]
    double K[3][3], dK[3][3][3];                   // dK[k][i][j] = d_k K_ij
    double alpha, dalpha[3], ddalpha[3][3];
    double beta[3], dbeta[3][3];                   // dbeta[j][i] = d_j beta^i
    double phi, dphi[3], ddphi[3][3];
    double Pi, dPi[3];
    double bdK[3][3], bdPi;                        // advection derivatives beta^k d_k K_ij, beta^k d_k Pi
};

struct Geo {
    double gi[3][3];
    double Gam[3][3][3];       // Gamma^k_ij  -> Gam[k][i][j]
    double Riem[3][3][3][3];   // 3D Riemann, all indices down
    double Ric[3][3], Rs;      // 3D Ricci, scalar
    double DK[3][3][3];        // D_k K_ij -> DK[k][i][j]
    double DDa[3][3], DDphi[3][3];
    double LbK[3][3];          // Lie derivative of K_ij along the shift
    double Kud[3][3];          // K^i_j
};

void geometry(const Phys& p, Geo& G) {
    inv3(p.g, G.gi);
    double G1[3][3][3];  // Christoffel of the first kind, G1[l][i][j] = Gamma_lij
    for (int l = 0; l < 3; ++l)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                G1[l][i][j] = 0.5 * (p.dg[i][l][j] + p.dg[j][l][i] - p.dg[l][i][j]);
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int l = 0; l < 3; ++l) s += G.gi[k][l] * G1[l][i][j];
                G.Gam[k][i][j] = s;
            }
    // derivative of the inverse metric and of Gamma^k_ij
    double dgi[3][3][3];
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
                double s = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) s -= G.gi[k][a] * p.dg[m][a][b] * G.gi[b][l];
                dgi[m][k][l] = s;
            }
    double dGam[3][3][3][3];  // dGam[m][k][i][j] = d_m Gamma^k_ij
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0;
                    for (int l = 0; l < 3; ++l) {
                        double dG1 = 0.5 * (p.ddg[m][i][l][j] + p.ddg[m][j][l][i] - p.ddg[m][l][i][j]);
                        s += dgi[m][k][l] * G1[l][i][j] + G.gi[k][l] * dG1;
                    }
                    dGam[m][k][i][j] = s;
                }
    // R^i_jkl = d_k Gamma^i_lj - d_l Gamma^i_kj + Gamma^i_km Gamma^m_lj - Gamma^i_lm Gamma^m_kj
    double Rud[3][3][3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double s = dGam[k][i][l][j] - dGam[l][i][k][j];
                    for (int m = 0; m < 3; ++m)
                        s += G.Gam[i][k][m] * G.Gam[m][l][j] - G.Gam[i][l][m] * G.Gam[m][k][j];
                    Rud[i][j][k][l] = s;
                }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double s = 0;
                    for (int m = 0; m < 3; ++m) s += p.g[i][m] * Rud[m][j][k][l];
                    G.Riem[i][j][k][l] = s;
                }
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) {
            double s = 0;
            for (int i = 0; i < 3; ++i) s += Rud[i][j][i][l];
            G.Ric[j][l] = s;
        }
    G.Rs = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G.Rs += G.gi[i][j] * G.Ric[i][j];
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = p.dK[k][i][j];
                for (int l = 0; l < 3; ++l) s -= G.Gam[l][k][i] * p.K[l][j] + G.Gam[l][k][j] * p.K[i][l];
                G.DK[k][i][j] = s;
            }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double sa = p.ddalpha[i][j], sp = p.ddphi[i][j];
            for (int k = 0; k < 3; ++k) {
                sa -= G.Gam[k][i][j] * p.dalpha[k];
                sp -= G.Gam[k][i][j] * p.dphi[k];
            }
            G.DDa[i][j] = sa;
            G.DDphi[i][j] = sp;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = p.bdK[i][j];
            for (int k = 0; k < 3; ++k) s += p.K[k][j] * p.dbeta[i][k] + p.K[i][k] * p.dbeta[j][k];
            G.LbK[i][j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += G.gi[i][k] * p.K[k][j];
            G.Kud[i][j] = s;
        }
}

// ------------------------------------------------------------------------------------
// 4dST sources by covariant assembly in the basis e_0 = n, e_i = d_i (g_ab = diag(-1, g_ij)).
// u[i][j] = d_t K_ij and w = d_t Pi are the coupled unknowns.
// ------------------------------------------------------------------------------------
struct Src {
    double rho8, S8[3], Sij8[3][3], LGB, E;  // 8 pi rho, 8 pi S_i, 8 pi S_ij, L_GB, scalar eq.
    double rho8_parts[3];  // 8 pi rho of the X, g2 X^2 and beta(phi) L_GB terms (with backreaction or not)
    double R4[4][4][4][4];  // the 4D Riemann tensor in the basis (n, d_i), all indices down
    double Ric4[4][4], R4s;  // its Ricci tensor and scalar
};

// beta'(phi), beta''(phi) of the Gauss-Bonnet coupling. The exponential kind ("Statement of
// Need": spin-induced scalarisation with an exponential coupling) is
//   beta = lam/(2 kappa) (1 - e^{-kappa phi^2}):  beta' = lam phi e^{-kappa phi^2},
//   beta'' = lam e^{-kappa phi^2} (1 - 2 kappa phi^2),
// which tends to the quadratic kind as kappa -> 0.
void beta_derivs(const orc_params& P, double phi, double& b1, double& b2) {
    if (P.beta_kind == 1) { b1 = P.lam * phi; b2 = P.lam; }
    else if (P.beta_kind == 2) {
        const double e = std::exp(-P.beta_kappa * phi * phi);
        b1 = P.lam * phi * e;
        b2 = P.lam * e * (1.0 - 2.0 * P.beta_kappa * phi * phi);
    } else { b1 = P.lam; b2 = 0.0; }
}

void sources(const orc_params& P, const Phys& p, const Geo& G, const double u[3][3], double w, Src& s) {
    double g4[4][4] = {{0}}, g4i[4][4] = {{0}};
    g4[0][0] = -1; g4i[0][0] = -1;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { g4[i + 1][j + 1] = p.g[i][j]; g4i[i + 1][j + 1] = G.gi[i][j]; }

    static thread_local double R4[4][4][4][4];
    std::memset(R4, 0, sizeof(R4));
    // Gauss: R_ijkl = 3R_ijkl + K_ik K_jl - K_il K_jk
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                    R4[i + 1][j + 1][k + 1][l + 1] =
                        G.Riem[i][j][k][l] + p.K[i][k] * p.K[j][l] - p.K[i][l] * p.K[j][k];
    // Codazzi: R_{n k i j} = D_i K_kj - D_j K_ki
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double b = G.DK[i][k][j] - G.DK[j][k][i];
                R4[0][k + 1][i + 1][j + 1] = b;
                R4[k + 1][0][i + 1][j + 1] = -b;
                R4[i + 1][j + 1][0][k + 1] = b;
                R4[i + 1][j + 1][k + 1][0] = -b;
            }
    // Ricci equation: R_{n i n j} = (d_t K_ij - L_beta K_ij + D_i D_j alpha)/alpha + K_ik K^k_j
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double kk = 0;
            for (int k = 0; k < 3; ++k) kk += p.K[i][k] * G.Kud[k][j];
            double c = (u[i][j] - G.LbK[i][j] + G.DDa[i][j]) / p.alpha + kk;
            R4[0][i + 1][0][j + 1] = c;
            R4[i + 1][0][j + 1][0] = c;
            R4[0][i + 1][j + 1][0] = -c;
            R4[i + 1][0][0][j + 1] = -c;
        }
    // raise all indices
    static thread_local double T1[4][4][4][4], T2[4][4][4][4], R4u[4][4][4][4];
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d) {
        double x = 0; for (int e = 0; e < 4; ++e) x += g4i[a][e] * R4[e][b][c][d]; T1[a][b][c][d] = x; }
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d) {
        double x = 0; for (int e = 0; e < 4; ++e) x += g4i[b][e] * T1[a][e][c][d]; T2[a][b][c][d] = x; }
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d) {
        double x = 0; for (int e = 0; e < 4; ++e) x += g4i[c][e] * T2[a][b][e][d]; T1[a][b][c][d] = x; }
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d) {
        double x = 0; for (int e = 0; e < 4; ++e) x += g4i[d][e] * T1[a][b][c][e]; R4u[a][b][c][d] = x; }
    double Ric4[4][4], Ric4u[4][4], R4s = 0;
    for (int b = 0; b < 4; ++b)
        for (int d = 0; d < 4; ++d) {
            double x = 0;
            for (int a = 0; a < 4; ++a) for (int c = 0; c < 4; ++c) x += g4i[a][c] * R4[a][b][c][d];
            Ric4[b][d] = x;
        }
    for (int b = 0; b < 4; ++b) for (int d = 0; d < 4; ++d) R4s += g4i[b][d] * Ric4[b][d];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double x = 0;
            for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d) x += g4i[a][c] * g4i[b][d] * Ric4[c][d];
            Ric4u[a][b] = x;
        }
    std::memcpy(s.R4, R4, sizeof(R4));
    std::memcpy(s.Ric4, Ric4, sizeof(Ric4));
    s.R4s = R4s;
    double riem2 = 0, ric2 = 0;
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d)
        riem2 += R4[a][b][c][d] * R4u[a][b][c][d];
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) ric2 += Ric4[a][b] * Ric4u[a][b];
    s.LGB = riem2 - 4.0 * ric2 + R4s * R4s;

    // double dual P_abcd
    static thread_local double Pd[4][4][4][4];
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d)
        Pd[a][b][c][d] = R4[a][b][c][d] - g4[a][c] * Ric4[b][d] + g4[a][d] * Ric4[b][c]
                         + g4[b][c] * Ric4[a][d] - g4[b][d] * Ric4[a][c]
                         + 0.5 * R4s * (g4[a][c] * g4[b][d] - g4[a][d] * g4[b][c]);

    // nabla phi and nabla nabla phi in the basis
    double dph[4] = {p.Pi, p.dphi[0], p.dphi[1], p.dphi[2]};
    double H[4][4];
    {
        double dadp = 0;
        for (int k = 0; k < 3; ++k) for (int l = 0; l < 3; ++l) dadp += G.gi[k][l] * p.dalpha[k] * p.dphi[l];
        H[0][0] = (w - p.bdPi - dadp) / p.alpha;
        for (int i = 0; i < 3; ++i) {
            double kd = 0;
            for (int k = 0; k < 3; ++k) kd += G.Kud[k][i] * p.dphi[k];  // K_i^k d_k phi
            H[0][i + 1] = H[i + 1][0] = p.dPi[i] + kd;
            for (int j = 0; j < 3; ++j) H[i + 1][j + 1] = G.DDphi[i][j] + p.K[i][j] * p.Pi;
        }
    }
    double b1, b2;
    beta_derivs(P, p.phi, b1, b2);
    double Phi[4][4], Phiu[4][4];
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) Phi[a][b] = b1 * H[a][b] + b2 * dph[a] * dph[b];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double x = 0;
            for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d) x += g4i[a][c] * g4i[b][d] * Phi[c][d];
            Phiu[a][b] = x;
        }
    double X = 0;
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) X -= 0.5 * g4i[a][b] * dph[a] * dph[b];
    const double g2 = P.g2;
    double T8[4][4];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double x = 0.5 * (1.0 + 2.0 * g2 * X) * dph[a] * dph[b] + 0.5 * g4[a][b] * (X + g2 * X * X);
            for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d) x -= 4.0 * Pd[a][c][b][d] * Phiu[c][d];
            T8[a][b] = x;
        }
    // energy densities of the three scalar terms of the action ("Diagnostics"): the n-n components
    // of the three parts of 8 pi T_ab
    {
        double gb = 0;
        for (int c = 0; c < 4; ++c) for (int d = 0; d < 4; ++d) gb -= 4.0 * Pd[0][c][0][d] * Phiu[c][d];
        s.rho8_parts[0] = 0.5 * dph[0] * dph[0] + 0.5 * g4[0][0] * X;
        s.rho8_parts[1] = g2 * X * dph[0] * dph[0] + 0.5 * g4[0][0] * g2 * X * X;
        s.rho8_parts[2] = gb;
    }
    // Without backreaction ("Key features": 4dST without backreaction onto the metric) the
    // scalar's stress-energy is left out of the metric equations; the scalar equation below still
    // uses the full 4D curvature of the evolving metric.
    const double keep = P.decoupled ? 0.0 : 1.0;
    s.rho8 = keep * T8[0][0];
    for (int i = 0; i < 3; ++i) {
        s.S8[i] = -keep * T8[i + 1][0];
        for (int j = 0; j < 3; ++j) s.Sij8[i][j] = keep * T8[i + 1][j + 1];
    }
    double dphu[4];
    for (int a = 0; a < 4; ++a) { double x = 0; for (int b = 0; b < 4; ++b) x += g4i[a][b] * dph[b]; dphu[a] = x; }
    double boxphi = 0, ddd = 0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) { boxphi += g4i[a][b] * H[a][b]; ddd += dphu[a] * dphu[b] * H[a][b]; }
    s.E = (1.0 + 2.0 * g2 * X) * boxphi - 2.0 * g2 * ddd + b1 * s.LGB;
}

// ------------------------------------------------------------------------------------
// Conformal (CCZ4) variables at one point.
// ------------------------------------------------------------------------------------
struct Conf {
    double chi, h[3][3], K, A[3][3], Th, Gam[3], alpha, beta[3], B[3], phi, Pi;
    double d1[NF][3];
    double d2[NF][6];
    double adv[NF];  // advection terms beta^k d_k u of every field
    // derived
    double hi[3][3], dh[3][3][3], Gt[3][3][3], Gtc[3], dGtc[3][3];  // Gt[k][i][j], dGtc[m][k]
    double Zl[3], Zu[3], RZ[3][3], RZs, divZ, Ric[3][3], Rs, Au[3][3], Aud[3][3], AA, DDa[3][3], DDa_tr, divb;
    double Kphys[3][3];
    Phys p;
    Geo G;
};

// Sets the shift-contracted derivatives of the physical data: from the advection terms `adv`
// (beta^k d_k of every conformal field; the chain rule of K_ij = (A_ij + h_ij K/3)/chi), or,
// when adv is null, as beta^k times the centred derivatives.
void advection_terms(const double* adv, Conf& c) {
    Phys& p = c.p;
    for (int f = 0; f < NF; ++f)
        c.adv[f] = adv ? adv[f] : c.beta[0] * c.d1[f][0] + c.beta[1] * c.d1[f][1] + c.beta[2] * c.d1[f][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            p.bdK[i][j] = (c.adv[F_A + SYM[i][j]] + c.adv[F_H + SYM[i][j]] * c.K / 3.0 + c.h[i][j] * c.adv[F_K] / 3.0) / c.chi
                          - p.K[i][j] * c.adv[F_CHI] / c.chi;
    p.bdPi = c.adv[F_PI];
}

void conf_setup(const double* v, const double* d1, const double* d2, const double* adv, Conf& c) {
    c.chi = v[F_CHI];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { c.h[i][j] = v[F_H + SYM[i][j]]; c.A[i][j] = v[F_A + SYM[i][j]]; }
    c.K = v[F_K]; c.Th = v[F_TH];
    for (int i = 0; i < 3; ++i) {
        c.Gam[i] = v[F_GAM + i]; c.beta[i] = v[F_SHIFT + i]; c.B[i] = v[F_B + i];
    }
    c.alpha = v[F_LAPSE]; c.phi = v[F_PHI]; c.Pi = v[F_PI];
    std::memcpy(c.d1, d1, sizeof(double) * NF * 3);
    std::memcpy(c.d2, d2, sizeof(double) * NF * 6);

    // physical data: g_ij = h_ij/chi and its derivatives (chain rule on the FD derivatives)
    Phys& p = c.p;
    const double chi = c.chi;
    double dchi[3], ddchi[3][3];
    for (int k = 0; k < 3; ++k) dchi[k] = d1[F_CHI * 3 + k];
    for (int k = 0; k < 3; ++k) for (int l = 0; l < 3; ++l) ddchi[k][l] = d2[F_CHI * 6 + SYM[k][l]];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int f = F_H + SYM[i][j];
            p.g[i][j] = c.h[i][j] / chi;
            for (int k = 0; k < 3; ++k) {
                c.dh[k][i][j] = d1[f * 3 + k];
                p.dg[k][i][j] = d1[f * 3 + k] / chi - c.h[i][j] * dchi[k] / (chi * chi);
            }
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                    p.ddg[k][l][i][j] = d2[f * 6 + SYM[k][l]] / chi
                                        - (d1[f * 3 + k] * dchi[l] + d1[f * 3 + l] * dchi[k]) / (chi * chi)
                                        - c.h[i][j] * ddchi[k][l] / (chi * chi)
                                        + 2.0 * c.h[i][j] * dchi[k] * dchi[l] / (chi * chi * chi);
        }
    // K_ij = (A_ij + h_ij K / 3) / chi
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int fa = F_A + SYM[i][j];
            c.Kphys[i][j] = p.K[i][j] = (c.A[i][j] + c.h[i][j] * c.K / 3.0) / chi;
            for (int k = 0; k < 3; ++k)
                p.dK[k][i][j] = (d1[fa * 3 + k] + c.dh[k][i][j] * c.K / 3.0 + c.h[i][j] * d1[F_K * 3 + k] / 3.0) / chi
                                - p.K[i][j] * dchi[k] / chi;
        }
    p.alpha = c.alpha;
    for (int k = 0; k < 3; ++k) p.dalpha[k] = d1[F_LAPSE * 3 + k];
    for (int k = 0; k < 3; ++k) for (int l = 0; l < 3; ++l) p.ddalpha[k][l] = d2[F_LAPSE * 6 + SYM[k][l]];
    for (int i = 0; i < 3; ++i) {
        p.beta[i] = c.beta[i];
        for (int j = 0; j < 3; ++j) p.dbeta[j][i] = d1[(F_SHIFT + i) * 3 + j];
    }
    p.phi = c.phi;
    for (int k = 0; k < 3; ++k) p.dphi[k] = d1[F_PHI * 3 + k];
    for (int k = 0; k < 3; ++k) for (int l = 0; l < 3; ++l) p.ddphi[k][l] = d2[F_PHI * 6 + SYM[k][l]];
    p.Pi = c.Pi;
    for (int k = 0; k < 3; ++k) p.dPi[k] = d1[F_PI * 3 + k];
    advection_terms(adv, c);

    geometry(p, c.G);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) c.Ric[i][j] = c.G.Ric[i][j];
    c.Rs = c.G.Rs;

    // conformal connection of h and its contraction, with derivatives (chain rule)
    inv3(c.h, c.hi);
    double Gt1[3][3][3];
    for (int l = 0; l < 3; ++l)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Gt1[l][i][j] = 0.5 * (c.dh[i][l][j] + c.dh[j][l][i] - c.dh[l][i][j]);
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int l = 0; l < 3; ++l) s += c.hi[k][l] * Gt1[l][i][j];
                c.Gt[k][i][j] = s;
            }
    for (int k = 0; k < 3; ++k) {
        double s = 0;
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) s += c.hi[i][j] * c.Gt[k][i][j];
        c.Gtc[k] = s;
    }
    double dhi[3][3][3];
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
                double s = 0;
                for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) s -= c.hi[k][a] * c.dh[m][a][b] * c.hi[b][l];
                dhi[m][k][l] = s;
            }
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k) {
            double s = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double dGt = 0;  // d_m Gt^k_ij
                    for (int l = 0; l < 3; ++l) {
                        double dG1 = 0.5 * (d2[(F_H + SYM[l][j]) * 6 + SYM[m][i]] + d2[(F_H + SYM[l][i]) * 6 + SYM[m][j]]
                                            - d2[(F_H + SYM[i][j]) * 6 + SYM[m][l]]);
                        dGt += dhi[m][k][l] * Gt1[l][i][j] + c.hi[k][l] * dG1;
                    }
                    s += dhi[m][i][j] * c.Gt[k][i][j] + c.hi[i][j] * dGt;
                }
            c.dGtc[m][k] = s;
        }
    // Z_i = h_ij (Gamma-hat^j - Gamma-tilde^j)/2 (physical covariant Z), D_j Z_i physical
    double dZ[3], ddZ[3][3];
    for (int k = 0; k < 3; ++k) dZ[k] = c.Gam[k] - c.Gtc[k];
    for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k) ddZ[j][k] = d1[(F_GAM + k) * 3 + j] - c.dGtc[j][k];
    double dZl[3][3];
    for (int i = 0; i < 3; ++i) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += c.h[i][k] * dZ[k];
        c.Zl[i] = 0.5 * s;
        for (int j = 0; j < 3; ++j) {
            double t = 0;
            for (int k = 0; k < 3; ++k) t += c.dh[j][i][k] * dZ[k] + c.h[i][k] * ddZ[j][k];
            dZl[j][i] = 0.5 * t;
        }
    }
    double DZ[3][3];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            double s = dZl[j][i];
            for (int k = 0; k < 3; ++k) s -= c.G.Gam[k][j][i] * c.Zl[k];
            DZ[j][i] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c.RZ[i][j] = c.Ric[i][j] + DZ[i][j] + DZ[j][i];
    c.RZs = 0;
    c.divZ = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { c.RZs += c.G.gi[i][j] * c.RZ[i][j]; c.divZ += c.G.gi[i][j] * DZ[i][j]; }
    for (int i = 0; i < 3; ++i) {
        double s = 0;
        for (int j = 0; j < 3; ++j) s += c.G.gi[i][j] * c.Zl[j];
        c.Zu[i] = s;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0, t = 0;
            for (int k = 0; k < 3; ++k) {
                t += c.hi[i][k] * c.A[k][j];
                for (int l = 0; l < 3; ++l) s += c.hi[i][k] * c.hi[j][l] * c.A[k][l];
            }
            c.Au[i][j] = s;
            c.Aud[i][j] = t;
        }
    c.AA = 0;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) c.AA += c.A[i][j] * c.Au[i][j];
    c.DDa_tr = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { c.DDa[i][j] = c.G.DDa[i][j]; c.DDa_tr += c.G.gi[i][j] * c.DDa[i][j]; }
    c.divb = d1[(F_SHIFT + 0) * 3 + 0] + d1[(F_SHIFT + 1) * 3 + 1] + d1[(F_SHIFT + 2) * 3 + 2];
}

// CCZ4 right-hand side in the modified puncture gauge, given the matter sources.
// rhs[F_PI] is left untouched (it is the solved unknown w).
void ccz4_rhs(const orc_params& P, const Conf& c, const Src& s, double* rhs) {
    const double al = c.alpha, chi = c.chi, K = c.K, Th = c.Th;
    const double a = P.a0, b = P.b0;
    auto adv = [&](int f) { return c.adv[f]; };
    auto db = [&](int j, int i) { return c.d1[F_SHIFT + i][j]; };  // d_j beta^i
    double S8tr = 0;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) S8tr += c.G.gi[i][j] * s.Sij8[i][j];

    rhs[F_CHI] = adv(F_CHI) + (2.0 / 3.0) * chi * (al * K - c.divb);
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            double x = adv(F_H + SYM[i][j]) - (2.0 / 3.0) * c.h[i][j] * c.divb - 2.0 * al * c.A[i][j];
            for (int k = 0; k < 3; ++k) x += c.h[i][k] * db(j, k) + c.h[j][k] * db(i, k);
            rhs[F_H + SYM[i][j]] = x;
        }
    // The modified gauge's b(x) enters through the auxiliary metric of the Z terms (see the header):
    // Hb = H - 16 pi rho - 2 kappa1 (2 + kappa2) Theta, with the plain H = R + K^2 - K_ij K^ij.
    const double Hb = c.Rs - c.AA + (2.0 / 3.0) * K * K - 2.0 * s.rho8 - 2.0 * P.kappa1 * (2.0 + P.kappa2) * Th;
    rhs[F_K] = adv(F_K) + al * (c.RZs + K * (K - 2.0 * Th)) - 3.0 * al * P.kappa1 * (1.0 + P.kappa2) * Th
               - c.DDa_tr + 0.5 * al * (S8tr - 3.0 * s.rho8) - (3.0 * al * b / (4.0 * (1.0 + b))) * Hb;
    {
        double X[3][3], trX = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) X[i][j] = -c.DDa[i][j] + al * (c.RZ[i][j] - s.Sij8[i][j]);
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) trX += c.hi[i][j] * X[i][j];
        for (int i = 0; i < 3; ++i)
            for (int j = i; j < 3; ++j) {
                double x = adv(F_A + SYM[i][j]) + chi * (X[i][j] - c.h[i][j] * trX / 3.0)
                           + al * (K - 2.0 * Th) * c.A[i][j] - (2.0 / 3.0) * c.A[i][j] * c.divb;
                for (int k = 0; k < 3; ++k)
                    x += -2.0 * al * c.A[i][k] * c.Aud[k][j] + c.A[i][k] * db(j, k) + c.A[j][k] * db(i, k);
                rhs[F_A + SYM[i][j]] = x;
            }
    }
    {
        double zda = 0;
        for (int i = 0; i < 3; ++i) zda += c.Zu[i] * c.d1[F_LAPSE][i];
        rhs[F_TH] = adv(F_TH) + al * (c.divZ - Th * K) - zda + (al / (2.0 * (1.0 + b))) * Hb;
    }
    double rhsG[3];
    for (int i = 0; i < 3; ++i) {
        double t1 = 0, t2 = 0, t3 = 0;
        for (int j = 0; j < 3; ++j) {
            for (int k = 0; k < 3; ++k) t1 += c.Gt[i][j][k] * c.Au[j][k];
            t2 += c.Au[i][j] * c.d1[F_CHI][j];
            t3 += c.hi[i][j] * c.d1[F_K][j];
        }
        double x = adv(F_GAM + i) + 2.0 * al * (t1 - (3.0 / (2.0 * chi)) * t2 - (2.0 / 3.0) * t3);
        for (int k = 0; k < 3; ++k)
            x += 2.0 * c.hi[k][i] * (al * c.d1[F_TH][k] - Th * c.d1[F_LAPSE][k] - (2.0 / 3.0) * al * K * c.Zl[k]);
        for (int j = 0; j < 3; ++j) x -= 2.0 * c.Au[i][j] * c.d1[F_LAPSE][j];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) x += c.hi[j][k] * c.d2[F_SHIFT + i][SYM[j][k]];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) x += c.hi[i][j] * c.d2[F_SHIFT + k][SYM[j][k]] / 3.0;
        x += (2.0 / 3.0) * c.Gtc[i] * c.divb;
        for (int k = 0; k < 3; ++k) x -= c.Gtc[k] * db(k, i);
        double hz = 0, hzdb = 0, hs = 0;
        for (int j = 0; j < 3; ++j) {
            hz += c.hi[i][j] * c.Zl[j];
            hs += c.hi[i][j] * s.S8[j];
            for (int k = 0; k < 3; ++k) hzdb += c.hi[j][k] * c.Zl[j] * db(k, i);
        }
        x += 2.0 * P.kappa3 * ((2.0 / 3.0) * hz * c.divb - hzdb) - 2.0 * al * P.kappa1 * hz - 2.0 * al * hs;
        // b(x) part of d_t Z_j: -(b/(1+b)) alpha (M_j + d_j Theta - K_j^k Z_k - kappa1 Z_j), with the
        // momentum constraint M_j = D_k K^k_j - D_j K - 8 pi S_j; Gamma-hat^i carries 2 h^ij Z_j
        double zb = 0;
        for (int j = 0; j < 3; ++j) {
            double m = -s.S8[j], kz = 0;
            for (int a2 = 0; a2 < 3; ++a2) {
                kz += c.Kphys[j][a2] * c.Zu[a2];
                for (int b2 = 0; b2 < 3; ++b2) m += c.G.gi[a2][b2] * (c.G.DK[a2][b2][j] - c.G.DK[j][a2][b2]);
            }
            zb += c.hi[i][j] * (m + c.d1[F_TH][j] - kz - P.kappa1 * c.Zl[j]);
        }
        x -= (2.0 * al * b / (1.0 + b)) * zb;
        rhsG[i] = x;
        rhs[F_GAM + i] = x;
    }
    rhs[F_LAPSE] = adv(F_LAPSE) - 2.0 * al * (K - 2.0 * Th) / (1.0 + a);
    for (int i = 0; i < 3; ++i) {
        double hda = 0;
        for (int j = 0; j < 3; ++j) hda += c.hi[i][j] * c.d1[F_LAPSE][j];
        rhs[F_SHIFT + i] = P.shift_F * c.B[i] / (1.0 + a) - (a / (1.0 + a)) * al * chi * hda;
        rhs[F_B + i] = rhsG[i] - P.eta * c.B[i];
    }
    rhs[F_PHI] = al * c.Pi + adv(F_PHI);
}

// d_t K_ij implied by the conformal right-hand sides (chain rule of K_ij = (A_ij + h_ij K/3)/chi)
void kdot_from_rhs(const Conf& c, const double* rhs, double u[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            u[i][j] = (rhs[F_A + SYM[i][j]] + rhs[F_H + SYM[i][j]] * c.K / 3.0 + c.h[i][j] * rhs[F_K] / 3.0) / c.chi
                      - c.Kphys[i][j] * rhs[F_CHI] / c.chi;
}

// Residual of the coupled equations at v = (u_11,u_12,u_13,u_22,u_23,u_33, w).
void residual(const orc_params& P, const Conf& c, const double* v, double* R, Src* s_out, double* rhs_out) {
    double u[3][3];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) u[i][j] = v[SYM[i][j]];
    Src s;
    sources(P, c.p, c.G, u, v[6], s);
    double rhs[NF];
    ccz4_rhs(P, c, s, rhs);
    double up[3][3];
    kdot_from_rhs(c, rhs, up);
    for (int m = 0; m < 6; ++m) R[m] = up[SYM_I[m]][SYM_J[m]] - v[m];
    R[6] = -c.alpha * s.E;
    if (s_out) *s_out = s;
    if (rhs_out) { std::memcpy(rhs_out, rhs, sizeof(rhs)); rhs_out[F_PI] = v[6]; }
}

// Tensor-waveform source ("Diagnostics": tensor gravitational waveforms): the Weyl scalar
//   Psi_4 = C_abcd n^a mbar^b n^c mbar^d,  n = (u - e_r)/sqrt(2),  m = (e_theta + i e_phi)/sqrt(2),
// u the unit normal of the slice, (e_r, e_theta, e_phi) the orthonormal triad (Gram-Schmidt with
// respect to gamma, in that order) of the coordinate directions (x, y, z), (x z, y z, -(x^2 + y^2))
// and (-y, x, 0) at the point's coordinates xyz relative to the origin. C is the 4D Weyl tensor
//   C_abcd = R_abcd - 1/2 (g_ac R_bd - g_ad R_bc - g_bc R_ad + g_bd R_ac) + R/6 (g_ac g_bd - g_ad g_bc)
// of the Riemann tensor assembled as for the sources (with the solved d_t K_ij). Psi_4 = 0 on the
// polar axis (x = y = 0), where the triad is not defined.
void weyl_psi4(const Phys& p, const Src& s, const double xyz[3], double out[2]) {
    out[0] = out[1] = 0;
    const double x = xyz[0], y = xyz[1], z = xyz[2];
    if (x * x + y * y == 0.0) return;
    double g4[4][4] = {{0}};
    g4[0][0] = -1;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) g4[i + 1][j + 1] = p.g[i][j];
    auto dot = [&](const double* a, const double* b) {
        double d = 0;
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) d += p.g[i][j] * a[i] * b[j];
        return d;
    };
    double e[3][3] = {{x, y, z}, {x * z, y * z, -(x * x + y * y)}, {-y, x, 0}};  // r, theta, phi
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < a; ++b) {
            const double d = dot(e[a], e[b]);
            for (int i = 0; i < 3; ++i) e[a][i] -= d * e[b][i];
        }
        const double nrm = std::sqrt(dot(e[a], e[a]));
        for (int i = 0; i < 3; ++i) e[a][i] /= nrm;
    }
    // tetrad components in the basis (n, d_i)
    const double h = 1.0 / std::sqrt(2.0);
    double nv[4] = {h, -h * e[0][0], -h * e[0][1], -h * e[0][2]};
    double mr[4] = {0, h * e[1][0], h * e[1][1], h * e[1][2]};   // Re mbar
    double mi[4] = {0, -h * e[2][0], -h * e[2][1], -h * e[2][2]};  // Im mbar
    double re = 0, im = 0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c)
                for (int d = 0; d < 4; ++d) {
                    const double C = s.R4[a][b][c][d]
                                     - 0.5 * (g4[a][c] * s.Ric4[b][d] - g4[a][d] * s.Ric4[b][c]
                                              - g4[b][c] * s.Ric4[a][d] + g4[b][d] * s.Ric4[a][c])
                                     + s.R4s / 6.0 * (g4[a][c] * g4[b][d] - g4[a][d] * g4[b][c]);
                    const double nn = nv[a] * nv[c] * C;
                    // mbar^b mbar^d = (mr + i mi)^b (mr + i mi)^d
                    re += nn * (mr[b] * mr[d] - mi[b] * mi[d]);
                    im += nn * (mr[b] * mi[d] + mi[b] * mr[d]);
                }
    out[0] = re;
    out[1] = im;
}

// Pointwise right-hand side (no dissipation). diag (optional, 64 doubles) receives:
// [0] 8pi rho [1..3] 8pi S_i [4..9] 8pi S_ij [10] L_GB [11..16] d_t K_ij [17] d_t Pi
// [18] |residual| after solve [19] solve status [20..25] R_ij + 2 D_(i Z_j) [26] its trace
// [27] R [28..33] R_ij [34..36] Z^i [37] D^i D_i lapse [38..44] solve matrix diagonal
// adv (optional): the advection terms beta^k d_k u of the 27 fields; null: centred, from d1.
int point_rhs(const orc_params& P, const double* v, const double* d1, const double* d2, const double* adv, double* rhs,
              double* diag) {
    static thread_local Conf c;
    conf_setup(v, d1, d2, adv, c);
    double zero[7] = {0, 0, 0, 0, 0, 0, 0}, R0[7], J[49], x[7];
    residual(P, c, zero, R0, nullptr, nullptr);
    double sc = 1.0;
    for (int m = 0; m < 7; ++m) sc = std::max(sc, std::fabs(R0[m]));
    for (int k = 0; k < 7; ++k) {
        double e[7] = {0, 0, 0, 0, 0, 0, 0}, Rk[7];
        e[k] = sc;
        residual(P, c, e, Rk, nullptr, nullptr);
        for (int m = 0; m < 7; ++m) J[m * 7 + k] = (Rk[m] - R0[m]) / sc;
    }
    double mr[7];
    for (int m = 0; m < 7; ++m) mr[m] = -R0[m];
    int st = solve_full_pivot(7, J, mr, x);
    Src s;
    double Rf[7];
    residual(P, c, x, Rf, &s, rhs);
    if (diag) {
        diag[0] = s.rho8;
        for (int i = 0; i < 3; ++i) diag[1 + i] = s.S8[i];
        for (int m = 0; m < 6; ++m) diag[4 + m] = s.Sij8[SYM_I[m]][SYM_J[m]];
        diag[10] = s.LGB;
        for (int m = 0; m < 7; ++m) diag[11 + m] = x[m];
        double rr = 0;
        for (int m = 0; m < 7; ++m) rr = std::max(rr, std::fabs(Rf[m]));
        diag[18] = rr;
        diag[19] = st;
        for (int m = 0; m < 6; ++m) diag[20 + m] = c.RZ[SYM_I[m]][SYM_J[m]];
        diag[26] = c.RZs;
        diag[27] = c.Rs;
        for (int m = 0; m < 6; ++m) diag[28 + m] = c.Ric[SYM_I[m]][SYM_J[m]];
        for (int i = 0; i < 3; ++i) diag[34 + i] = c.Zu[i];
        diag[37] = c.DDa_tr;
        for (int m = 0; m < 7; ++m) diag[38 + m] = J[m * 7 + m];
    }
    return st;
}

// Hamiltonian and momentum constraints in their physical form:
//   H = R + K^2 - K_ij K^ij - 16 pi rho,  M_i = D_j K^j_i - D_i K - 8 pi S_i
void point_constraints(const orc_params& P, const double* v, const double* d1, const double* d2, double* out4) {
    static thread_local Conf c;
    conf_setup(v, d1, d2, nullptr, c);
    double u[3][3] = {{0}};
    Src s;
    sources(P, c.p, c.G, u, 0.0, s);
    const double (*gi)[3] = c.G.gi;
    double tr = 0, kk = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            tr += gi[i][j] * c.p.K[i][j];
            double kij = 0;
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) kij += gi[i][a] * gi[j][b] * c.p.K[a][b];
            kk += c.p.K[i][j] * kij;
        }
    out4[0] = c.Rs + tr * tr - kk - 2.0 * s.rho8;
    for (int i = 0; i < 3; ++i) {
        double m = 0;
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) m += gi[j][k] * (c.G.DK[j][k][i] - c.G.DK[i][j][k]);
        out4[1 + i] = m - s.S8[i];
    }
}

// 8 pi rho of the X, g2 X^2 and Gauss-Bonnet terms at one point (independent of d_t K_ij, d_t Pi).
void point_energy(const orc_params& P, const double* v, const double* d1, const double* d2, double* out3) {
    static thread_local Conf c;
    conf_setup(v, d1, d2, nullptr, c);
    double u[3][3] = {{0}};
    Src s;
    sources(P, c.p, c.G, u, 0.0, s);
    for (int m = 0; m < 3; ++m) out3[m] = s.rho8_parts[m];
}

// ------------------------------------------------------------------------------------
// Grid operations
// ------------------------------------------------------------------------------------
struct Grid {
    int nx, ny, nz, ng, NX, NY, NZ;
    long long fstride;
    explicit Grid(const orc_box& b) : nx(b.nx), ny(b.ny), nz(b.nz), ng(b.ng) {
        NX = nx + 2 * ng; NY = ny + 2 * ng; NZ = nz + 2 * ng;
        fstride = (long long)NX * NY * NZ;
    }
    long long at(int f, int i, int j, int k) const {  // ghosted indices
        return f * fstride + ((long long)k * NY + j) * NX + i;
    }
};

// Difference weights of the two schemes ("Accuracy": 4th and 6th order), on offsets -r..r
// (centred) or lo..lo+n-1 (lopsided, for beta >= 0), each sum divided by den dx (den dx^2 for the
// second derivative). The box's ghost width chooses the scheme: ng = 3 -> 4th, ng = 4 -> 6th.
struct Scheme {
    int r;             // half-width of the centred stencils
    double c1[7], c2[7], den1, den2;
    int lo, nl;        // lopsided stencil: first offset and length
    double cl[7], denl;
    int rko;           // Kreiss-Oliger half-width; weights binomial, factor ko_sign sigma / (4^rko dx)
    double cko[9], ko_sign, ko_div;
};

Scheme scheme(int ng) {
    Scheme q;
    if (ng == 4) {
        q = {3, {-1, 9, -45, 0, 45, -9, 1}, {2, -27, 270, -490, 270, -27, 2}, 60.0, 180.0,
             -2, 7, {2, -24, -35, 80, -30, 8, -1}, 60.0,
             4, {1, -8, 28, -56, 70, -56, 28, -8, 1}, -1.0, 256.0};
    } else {
        q = {2, {1, -8, 0, 8, -1}, {-1, 16, -30, 16, -1}, 12.0, 12.0,
             -1, 5, {-3, -10, 18, -6, 1}, 12.0,
             3, {1, -6, 15, -20, 15, -6, 1}, 1.0, 64.0};
    }
    return q;
}

// centred stencils of the box's scheme at ghosted point (i,j,k); mixed derivatives are the
// tensor product of two first-derivative stencils
void point_derivs(const Grid& g, const double* s, double dx, int i, int j, int k, double* v, double* d1, double* d2) {
    const Scheme q = scheme(g.ng);
    const int n = 2 * q.r + 1;
    const double i1 = 1.0 / (q.den1 * dx), i2 = 1.0 / (q.den2 * dx * dx), imx = 1.0 / (q.den1 * q.den1 * dx * dx);
    for (int f = 0; f < NF; ++f) {
        auto U = [&](int a, int b, int cc) { return s[g.at(f, i + a, j + b, k + cc)]; };
        v[f] = U(0, 0, 0);
        int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int d = 0; d < 3; ++d) {
            double x = 0, y = 0;
            for (int m = 0; m < n; ++m) {
                const int o = m - q.r;
                x += q.c1[m] * U(o * e[d][0], o * e[d][1], o * e[d][2]);
                y += q.c2[m] * U(o * e[d][0], o * e[d][1], o * e[d][2]);
            }
            d1[f * 3 + d] = x * i1;
            d2[f * 6 + SYM[d][d]] = y * i2;
        }
        for (int d = 0; d < 3; ++d)
            for (int p = d + 1; p < 3; ++p) {
                double x = 0;
                for (int m = 0; m < n; ++m)
                    for (int l = 0; l < n; ++l) {
                        int o[3] = {0, 0, 0};
                        o[d] += m - q.r;
                        o[p] += l - q.r;
                        x += q.c1[m] * q.c1[l] * U(o[0], o[1], o[2]);
                    }
                d2[f * 6 + SYM[d][p]] = x * imx;
            }
    }
}

// Lopsided advection terms adv[f] = sum_d beta^d D_d u_f at ghosted point (i,j,k): D_d is the
// lopsided stencil of the box's scheme, biased towards +d where beta^d >= 0 and mirrored (offsets
// negated, sum negated) where beta^d < 0.
void point_adv_lopsided(const Grid& g, const double* s, double dx, int i, int j, int k, double* adv) {
    const Scheme q = scheme(g.ng);
    double beta[3];
    for (int d = 0; d < 3; ++d) beta[d] = s[g.at(F_SHIFT + d, i, j, k)];
    for (int f = 0; f < NF; ++f) {
        double a = 0;
        for (int d = 0; d < 3; ++d) {
            const int sg = beta[d] >= 0.0 ? 1 : -1;
            double x = 0;
            for (int m = 0; m < q.nl; ++m) {
                const int o = sg * (q.lo + m);
                x += q.cl[m] * s[g.at(f, i + (d == 0 ? o : 0), j + (d == 1 ? o : 0), k + (d == 2 ? o : 0))];
            }
            a += beta[d] * (sg * x / (q.denl * dx));
        }
        adv[f] = a;
    }
}

// Kreiss-Oliger difference sum_d Delta^(2 rko)_d u (unscaled)
double ko_point(const Grid& g, const double* s, int f, int i, int j, int k) {
    const Scheme q = scheme(g.ng);
    double t = 0;
    for (int m = 0; m < 2 * q.rko + 1; ++m) {
        int o = m - q.rko;
        t += q.cko[m] * (s[g.at(f, i + o, j, k)] + s[g.at(f, i, j + o, k)] + s[g.at(f, i, j, k + o)]);
    }
    return t;
}

// sigma times the Kreiss-Oliger factor of the box's scheme
double ko_factor(int ng, double sigma, double dx) {
    const Scheme q = scheme(ng);
    return q.ko_sign * sigma / (q.ko_div * dx);
}

void fill_periodic(const Grid& g, double* s) {
    auto wrap = [](int a, int n, int ng) { int x = (a - ng) % n; if (x < 0) x += n; return x + ng; };
    for (int f = 0; f < NF; ++f)
        for (int k = 0; k < g.NZ; ++k)
            for (int j = 0; j < g.NY; ++j)
                for (int i = 0; i < g.NX; ++i) {
                    bool ghost = i < g.ng || i >= g.ng + g.nx || j < g.ng || j >= g.ng + g.ny || k < g.ng || k >= g.ng + g.nz;
                    if (!ghost) continue;
                    s[g.at(f, i, j, k)] = s[g.at(f, wrap(i, g.nx, g.ng), wrap(j, g.ny, g.ng), wrap(k, g.nz, g.ng))];
                }
}

// Parity of field f under the reflection x_d -> -x_d: -1 for components with an odd number of
// indices along d (the d-component of Gamma-hat, shift and B; h_de and A_de with exactly one
// index d), +1 for scalars and the rest.
double parity(int f, int d) {
    if (f >= F_GAM && f < F_GAM + 3) return (f - F_GAM == d) ? -1.0 : 1.0;
    if (f >= F_SHIFT && f < F_SHIFT + 3) return (f - F_SHIFT == d) ? -1.0 : 1.0;
    if (f >= F_B && f < F_B + 3) return (f - F_B == d) ? -1.0 : 1.0;
    int m = -1;
    if (f >= F_H && f < F_H + 6) m = f - F_H;
    if (f >= F_A && f < F_A + 6) m = f - F_A;
    if (m >= 0) return ((SYM_I[m] == d) != (SYM_J[m] == d)) ? -1.0 : 1.0;
    return 1.0;
}

// Mirror planes half a cell below the first interior point on the three low faces: a ghost point
// whose coordinates are interior or low ghosts (at least one) takes the value of its mirror image
// in the interior, times the field's parity under each reflected axis. Ghosts on the high faces
// (any coordinate past the interior) are left as given.
// With all = true every ghost with a low coordinate is an image, also those beyond a high face
// in another axis (mirror planes combined with evolved high-face ghosts).
void fill_reflect(const Grid& g, double* s, bool all = false) {
    const int ex = all ? g.NX : g.ng + g.nx, ey = all ? g.NY : g.ng + g.ny, ez = all ? g.NZ : g.ng + g.nz;
    for (int f = 0; f < NF; ++f)
        for (int k = 0; k < ez; ++k)
            for (int j = 0; j < ey; ++j)
                for (int i = 0; i < ex; ++i) {
                    if (i >= g.ng && j >= g.ng && k >= g.ng) continue;
                    double sign = 1.0;
                    int a = i, b = j, c = k;
                    if (i < g.ng) { a = 2 * g.ng - 1 - i; sign *= parity(f, 0); }
                    if (j < g.ng) { b = 2 * g.ng - 1 - j; sign *= parity(f, 1); }
                    if (k < g.ng) { c = 2 * g.ng - 1 - k; sign *= parity(f, 2); }
                    s[g.at(f, i, j, k)] = sign * s[g.at(f, a, b, c)];
                }
}

// Extrapolating boundaries ("Boundary Conditions": extrapolating): every ghost point takes the
// linear extrapolation, along one axis, of the last two points before it,
//   u(last + m) = u(last) + m (u(last) - u(last - 1)),  m = 1 .. ng,
// axis by axis: x-ghosts on rows of interior (y, z), then y-ghosts on rows of any x and interior
// z, then z-ghosts on rows of any x and y, so edges and corners extrapolate values already set.
void fill_extrapolate(const Grid& g, double* s) {
    const int n[3] = {g.nx, g.ny, g.nz};
    const int N[3] = {g.NX, g.NY, g.NZ};
    for (int ax = 0; ax < 3; ++ax) {
        const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
        for (int f = 0; f < NF; ++f)
            for (int c2 = 0; c2 < N[a2]; ++c2)
                for (int c1 = 0; c1 < N[a1]; ++c1) {
                    // the transverse coordinates range over what earlier axes have filled
                    auto inside = [&](int a, int c) { return a < ax || (c >= g.ng && c < g.ng + n[a]); };
                    if (!inside(a1, c1) || !inside(a2, c2)) continue;
                    auto at = [&](int c) {
                        int ijk[3];
                        ijk[ax] = c; ijk[a1] = c1; ijk[a2] = c2;
                        return g.at(f, ijk[0], ijk[1], ijk[2]);
                    };
                    const int lo = g.ng, hi = g.ng + n[ax] - 1;
                    for (int m = 1; m <= g.ng; ++m) {
                        s[at(hi + m)] = s[at(hi)] + m * (s[at(hi)] - s[at(hi - 1)]);
                        s[at(lo - m)] = s[at(lo)] + m * (s[at(lo)] - s[at(lo + 1)]);
                    }
                }
    }
}

void fill_bc(const orc_box& b, const Grid& g, double* s) {
    if (b.bc == 0) fill_periodic(g, s);
    else if (b.bc == 2) fill_reflect(g, s);
    else if (b.bc == 3) fill_extrapolate(g, s);
    else if (b.bc == 5) fill_reflect(g, s, true);
}

// Sommerfeld (radiative) boundaries ("Boundary Conditions": Sommerfeld): every ghost point of the
// box is evolved with
//   d_t u = - v (u - u_inf) / r - v (x^i / r) d_i u,   v = 1, r = |x| (centre at the origin),
// u_inf the flat values (chi = h_11 = h_22 = h_33 = lapse = 1, all else 0). Along an axis on
// which the point lies beyond the interior, d_i is the 2nd-order one-sided difference pointing
// into the box ((3 u - 4 u_-1 + u_-2) / (2 dx) past the high face, (-3 u + 4 u_1 - u_2) / (2 dx)
// past the low face); along the other axes the centred 2nd-order difference. At r = 0 the right
// side is taken as 0.
double u_inf(int f) {
    return (f == F_CHI || f == F_H + 0 || f == F_H + 3 || f == F_H + 5 || f == F_LAPSE) ? 1.0 : 0.0;
}

bool is_ghost(const Grid& g, int i, int j, int k) {
    return i < g.ng || i >= g.ng + g.nx || j < g.ng || j >= g.ng + g.ny || k < g.ng || k >= g.ng + g.nz;
}

// The ghosts a box evolves with the radiative condition: all of them (bc 4), or, behind mirror
// planes (bc 5), those beyond a high face with no coordinate below the box.
bool is_sommerfeld_point(const orc_box& b, const Grid& g, int i, int j, int k) {
    if (b.bc == 4) return is_ghost(g, i, j, k);
    if (b.bc != 5) return false;
    return i >= g.ng && j >= g.ng && k >= g.ng && is_ghost(g, i, j, k);
}

double sommerfeld_rhs(const orc_box& b, const Grid& g, const double* s, int f, int i, int j, int k) {
    const int idx[3] = {i, j, k};
    const int n[3] = {g.nx, g.ny, g.nz};
    const double x[3] = {b.x0 + (i - g.ng) * b.dx, b.y0 + (j - g.ng) * b.dx, b.z0 + (k - g.ng) * b.dx};
    const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    if (r == 0.0) return 0.0;
    auto U = [&](int d, int o) {
        int q[3] = {i, j, k};
        q[d] += o;
        return s[g.at(f, q[0], q[1], q[2])];
    };
    double adv = 0;
    for (int d = 0; d < 3; ++d) {
        double du;
        if (idx[d] >= g.ng + n[d]) du = (3.0 * U(d, 0) - 4.0 * U(d, -1) + U(d, -2)) / (2.0 * b.dx);
        else if (idx[d] < g.ng) du = (-3.0 * U(d, 0) + 4.0 * U(d, 1) - U(d, 2)) / (2.0 * b.dx);
        else du = (U(d, 1) - U(d, -1)) / (2.0 * b.dx);
        adv += x[d] * du;
    }
    return -(U(0, 0) - u_inf(f)) / r - adv / r;
}

// rhs at every ghost point of a Sommerfeld box
void sommerfeld_box(const orc_box& b, const Grid& g, const double* s, double* rhs) {
#pragma omp parallel for collapse(2)
    for (int f = 0; f < NF; ++f)
        for (int k = 0; k < g.NZ; ++k)
            for (int j = 0; j < g.NY; ++j)
                for (int i = 0; i < g.NX; ++i)
                    if (is_sommerfeld_point(b, g, i, j, k)) rhs[g.at(f, i, j, k)] = sommerfeld_rhs(b, g, s, f, i, j, k);
}

int rhs_box(const orc_box& b, const orc_params& P, const double* s, double* rhs, int with_ko) {
    Grid g(b);
    int bad = 0;
    const double ko = ko_factor(b.ng, P.sigma_ko, b.dx);
#pragma omp parallel for collapse(2) schedule(dynamic) reduction(+ : bad)
    for (int k = g.ng; k < g.ng + g.nz; ++k)
        for (int j = g.ng; j < g.ng + g.ny; ++j)
            for (int i = g.ng; i < g.ng + g.nx; ++i) {
                double v[NF], d1[NF * 3], d2[NF * 6], r[NF], adv[NF];
                point_derivs(g, s, b.dx, i, j, k, v, d1, d2);
                if (P.advection) point_adv_lopsided(g, s, b.dx, i, j, k, adv);
                if (point_rhs(P, v, d1, d2, P.advection ? adv : nullptr, r, nullptr) != 0) bad++;
                for (int f = 0; f < NF; ++f) {
                    double x = r[f];
                    if (with_ko) x += ko * ko_point(g, s, f, i, j, k);
                    rhs[g.at(f, i, j, k)] = x;
                }
            }
    if (b.bc == 4 || b.bc == 5) sommerfeld_box(b, g, s, rhs);
    return bad ? -5 : 0;
}

void enforce(const Grid& g, const orc_params& P, double* s) {
#pragma omp parallel for collapse(2)
    for (int k = g.ng; k < g.ng + g.nz; ++k)
        for (int j = g.ng; j < g.ng + g.ny; ++j)
            for (int i = g.ng; i < g.ng + g.nx; ++i) {
                double h[3][3], hi[3][3], A[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) {
                        h[a][c] = s[g.at(F_H + SYM[a][c], i, j, k)];
                        A[a][c] = s[g.at(F_A + SYM[a][c], i, j, k)];
                    }
                inv3(h, hi);
                double tr = 0;
                for (int a = 0; a < 3; ++a) for (int c = 0; c < 3; ++c) tr += hi[a][c] * A[a][c];
                for (int m = 0; m < 6; ++m)
                    s[g.at(F_A + m, i, j, k)] = A[SYM_I[m]][SYM_J[m]] - h[SYM_I[m]][SYM_J[m]] * tr / 3.0;
                double& chi = s[g.at(F_CHI, i, j, k)];
                chi = std::max(chi, P.min_chi);
                double& al = s[g.at(F_LAPSE, i, j, k)];
                al = std::max(al, P.min_lapse);
            }
}

}  // namespace

extern "C" {

int orc_point_rhs(const orc_params* P, const double* v, const double* d1, const double* d2, double* rhs, double* diag) {
    return point_rhs(*P, v, d1, d2, nullptr, rhs, diag);
}

// As orc_point_rhs with the 27 advection terms beta^k d_k u given (adv).
int orc_point_rhs_adv(const orc_params* P, const double* v, const double* d1, const double* d2, const double* adv,
                      double* rhs, double* diag) {
    return point_rhs(*P, v, d1, d2, adv, rhs, diag);
}

void orc_point_constraints(const orc_params* P, const double* v, const double* d1, const double* d2, double* out4) {
    point_constraints(*P, v, d1, d2, out4);
}

// Psi_4 at one point: the coupled system is solved as for the right-hand side, the Riemann tensor
// assembled with the solved d_t K_ij. xyz: coordinates relative to the origin of the triad.
void orc_point_psi4(const orc_params* P, const double* v, const double* d1, const double* d2, const double* xyz,
                    double* out2) {
    double rhs[NF], diag[64];
    point_rhs(*P, v, d1, d2, nullptr, rhs, diag);
    static thread_local Conf c;
    conf_setup(v, d1, d2, nullptr, c);
    double u[3][3];
    for (int m = 0; m < 6; ++m) u[SYM_I[m]][SYM_J[m]] = u[SYM_J[m]][SYM_I[m]] = diag[11 + m];
    Src s;
    sources(*P, c.p, c.G, u, diag[17], s);
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
    sources(*P, p, G, u, w, s);
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
    return rhs_box(*b, *P, s, rhs, with_ko);
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

void orc_enforce(const orc_box* b, const orc_params* P, double* s) { enforce(Grid(*b), *P, s); }

// Classical RK4: k_s = RHS(u_{s-1}) (with KO); u_1 = u_n + dt/2 k_1, u_2 = u_n + dt/2 k_2,
// u_3 = u_n + dt k_3, u_{n+1} = u_n + dt/6 (k_1 + 2k_2 + 2k_3 + k_4); every written state is
// passed through the algebraic enforcement (interior points) when enabled. Periodic, mirror and
// extrapolating boxes refill ghosts before every RHS evaluation; frozen boxes keep the ghosts of
// the input state; Sommerfeld boxes evolve their ghosts with the same RK4 stages.
int orc_rk4(const orc_box* b, const orc_params* P, double* s, double dt, int nsteps) {
    Grid g(*b);
    const long long n = NF * g.fstride;
    std::vector<double> us(s, s + n), k(n, 0.0), acc(n, 0.0);
    const double c[3] = {0.5, 0.5, 1.0};
    int st = 0;
    for (int step = 0; step < nsteps; ++step) {
        fill_bc(*b, g, s);
        std::copy(s, s + n, us.begin());
        for (int stage = 0; stage < 4; ++stage) {
            const double* src = (stage == 0) ? s : us.data();
            int r = rhs_box(*b, *P, src, k.data(), 1);
            if (r) st = r;
            // the evolved points: the interior, and the Sommerfeld ghosts (all ghosts for bc 4,
            // those with no coordinate below the box for bc 5)
            const bool som = b->bc == 4 || b->bc == 5;
            const int e0 = b->bc == 4 ? 0 : g.ng;
            const int ex = som ? g.NX : g.ng + g.nx, ey = som ? g.NY : g.ng + g.ny, ez = som ? g.NZ : g.ng + g.nz;
#pragma omp parallel for collapse(3)
            for (int f = 0; f < NF; ++f)
                for (int kk = e0; kk < ez; ++kk)
                    for (int j = e0; j < ey; ++j)
                        for (int i = e0; i < ex; ++i) {
                            long long q = g.at(f, i, j, kk);
                            double w = (stage == 0 || stage == 3) ? 1.0 : 2.0;
                            acc[q] = (stage == 0 ? 0.0 : acc[q]) + w * k[q];
                            if (stage < 3) us[q] = s[q] + c[stage] * dt * k[q];
                        }
            if (stage < 3) {
                if (P->enforce_algebraic) enforce(g, *P, us.data());
                fill_bc(*b, g, us.data());
            }
        }
        const bool som = b->bc == 4 || b->bc == 5;
        const int e0 = b->bc == 4 ? 0 : g.ng;
        const int ex = som ? g.NX : g.ng + g.nx, ey = som ? g.NY : g.ng + g.ny, ez = som ? g.NZ : g.ng + g.nz;
#pragma omp parallel for collapse(3)
        for (int f = 0; f < NF; ++f)
            for (int kk = e0; kk < ez; ++kk)
                for (int j = e0; j < ey; ++j)
                    for (int i = e0; i < ex; ++i) {
                        long long q = g.at(f, i, j, kk);
                        s[q] = s[q] + dt / 6.0 * acc[q];
                    }
        if (P->enforce_algebraic) enforce(g, *P, s);
        fill_bc(*b, g, s);
    }
    return st;
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
    point_energy(*P, v, d1, d2, out3);
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
                point_energy(*P, v, d1, d2, o);
                long long p = ((long long)k * b->ny + j) * b->nx + i;
                for (int m = 0; m < 3; ++m) out[m * npt + p] = o[m];
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
                point_constraints(*P, v, d1, d2, o);
                long long p = ((long long)k * b->ny + j) * b->nx + i;
                for (int m = 0; m < 4; ++m) out[m * npt + p] = o[m];
            }
}

}  // extern "C"
