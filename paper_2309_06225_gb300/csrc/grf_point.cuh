// Pointwise right-hand side of the modified CCZ4 + 4dST system (FP64, one grid point per
// thread, everything in registers / local memory).
//
// The 4dST sources are written in explicit 3+1 form. With the basis (n, d_i) the 4D
// Riemann tensor splits into
//     S_ij  = gamma^kl R_kilj           = R_ij + K K_ij - K_ik K^k_j          (Gauss block)
//     B_kij = R_{n k i j}               = D_i K_kj - D_j K_ki                (Codazzi block)
//     C_ij  = R_{n i n j}               = (d_t K_ij - L_beta K_ij + D_i D_j lapse)/lapse
//                                          + K_ik K^k_j                        (Ricci equation)
// and the double dual P has the closed form
//     P_ninj = S_ij - gamma_ij S / 2,   P_nkij = B_kij - gamma_ki B_j + gamma_kj B_i,
//     P_ijkl = gamma_ik C_jl - gamma_il C_jk - gamma_jk C_il + gamma_jl C_ik - C (g_ik g_jl - g_il g_jk),
// with B_j = gamma^ab B_abj. Then
//     L_GB   = 8 G_S^ij C_ij - 4 B_kij B^kij + 8 B_i B^i            (G_S = S - gamma S/2)
//     8 pi rho  = rho1 - 4 G_S^ij Phi_ij
//     8 pi S_i  = S1_i + 4 [G_S ik Phi_n^k + B_kil Phi^kl - Phi_i^l B_l + tr(Phi) B_i]
//     8 pi S_ij = S1_ij - 4 [G_S ij Phi_nn + Y_ij + Q_ij(C)]
// where Phi_ab = nabla_a nabla_b beta(phi) and the first-order (X, X^2) parts rho1, S1 are
// those of (1/16 pi)(X + g2 X^2). C_ij (through d_t K_ij) and Phi_nn (through d_t Pi) are
// the only places the unknowns enter, affinely: the 7x7 system M v = r for v = (d_t K_ij, d_t Pi)
// is assembled from these expressions and solved by LU with partial pivoting.
#pragma once

#include <cuda_runtime.h>

namespace grf {

// d1 slots: fields 0..21 keep their index, phi -> 22, Pi -> 23 (B^i has no derivative)
__host__ __device__ constexpr int d1slot(int f) { return f < 22 ? f : (f == 25 ? 22 : 23); }
// d2 slots: chi 0, h 1..6, lapse 7, shift 8..10, phi 11
__host__ __device__ constexpr int d2slot(int f) { return f < 7 ? f : (f == 18 ? 7 : (f < 22 ? f - 11 : 11)); }
__host__ __device__ constexpr int sidx(int i, int j) {
    return i <= j ? (i == 0 ? j : (i == 1 ? 2 + j : 5)) : (j == 0 ? i : (j == 1 ? 2 + i : 5));
}

enum { F_CHI = 0, F_H = 1, F_K = 7, F_A = 8, F_TH = 14, F_GAM = 15, F_LAPSE = 18, F_SHIFT = 19,
       F_B = 22, F_PHI = 25, F_PI = 26, NFIELDS = 27 };

struct Coeffs {
    double kappa1, kappa2, kappa3, shift_F, eta, lam, g2;
    double inv_1pa, a_1pa;        // 1/(1+a), a/(1+a)
    double bK, bTh;               // 3b/(4(1+b)), 1/(2(1+b))
    int beta_kind;
};

struct PointIn {
    double v[NFIELDS];
    double d1[24][3];
    double d2[12][6];
};

// Output diagnostics besides the RHS (constraints come out as by-products).
struct PointExtra {
    double ham;      // H = S - 2 (8 pi rho)
    double mom[3];   // M_i = B_i - 8 pi S_i
};

__device__ __forceinline__ double sym3_det(const double h[6]) {
    return h[0] * (h[3] * h[5] - h[4] * h[4]) - h[1] * (h[1] * h[5] - h[4] * h[2])
           + h[2] * (h[1] * h[4] - h[3] * h[2]);
}

// symmetric inverse; returns determinant
__device__ __forceinline__ double sym3_inv(const double h[6], double hi[6]) {
    const double c00 = h[3] * h[5] - h[4] * h[4];
    const double c01 = h[2] * h[4] - h[1] * h[5];
    const double c02 = h[1] * h[4] - h[2] * h[3];
    const double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    const double id = 1.0 / det;
    hi[0] = c00 * id;
    hi[1] = c01 * id;
    hi[2] = c02 * id;
    hi[3] = (h[0] * h[5] - h[2] * h[2]) * id;
    hi[4] = (h[1] * h[2] - h[0] * h[4]) * id;
    hi[5] = (h[0] * h[3] - h[1] * h[1]) * id;
    return det;
}

// 7x7 LU with partial pivoting (row swaps by compare-and-exchange, so every index stays a
// compile-time constant and the matrix stays in registers). Returns false on a pivot
// smaller than 1e-300 times the largest entry.
__device__ __forceinline__ bool solve7(double M[7][8]) {
    double mx = 0.0;
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int j = 0; j < 7; ++j) mx = fmax(mx, fabs(M[i][j]));
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
#pragma unroll
        for (int i = k + 1; i < 7; ++i) {
            const bool sw = fabs(M[i][k]) > fabs(M[k][k]);
#pragma unroll
            for (int j = k; j < 8; ++j) {
                const double a = M[k][j], b = M[i][j];
                M[k][j] = sw ? b : a;
                M[i][j] = sw ? a : b;
            }
        }
        ok = ok && (fabs(M[k][k]) > 1e-300 * mx);
        const double ip = 1.0 / M[k][k];
#pragma unroll
        for (int i = k + 1; i < 7; ++i) {
            const double f = M[i][k] * ip;
#pragma unroll
            for (int j = k + 1; j < 8; ++j) M[i][j] = fma(-f, M[k][j], M[i][j]);
        }
        M[k][7] *= ip;
#pragma unroll
        for (int j = k + 1; j < 7; ++j) M[k][j] *= ip;
    }
#pragma unroll
    for (int k = 6; k >= 0; --k) {
#pragma unroll
        for (int j = k + 1; j < 7; ++j) M[k][7] = fma(-M[k][j], M[j][7], M[k][7]);
    }
    return ok;
}

// L(Q(u)) for a symmetric u (6 components): the linear part of the 4dST S_ij in d_t K_ij,
// traced-reversed as it enters d_t K_ij. gd: gamma_ij, Phm: Phi_i^k (mixed, row i),
// Phu: Phi^{ij}, Phd: Phi_ij, trP = gamma^ij Phi_ij, gu: gamma^ij.
__device__ __forceinline__ void apply_LQ(const double u[6], const double gd[6], const double gu[6],
                                         const double Phd[6], const double Phu[6], const double Phm[3][3],
                                         double trP, double out[6]) {
    double uP = 0.0, tru = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uP = fma(u[sidx(i, j)], Phu[sidx(i, j)], uP);
            tru = fma(u[sidx(i, j)], gu[sidx(i, j)], tru);
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double pu = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) pu += Phm[i][k] * u[sidx(k, j)] + Phm[j][k] * u[sidx(i, k)];
            out[sidx(i, j)] = 0.5 * gd[sidx(i, j)] * (uP - tru * trP) - pu + trP * u[sidx(i, j)] + tru * Phd[sidx(i, j)];
        }
}

__device__ __forceinline__ void point_rhs(const Coeffs& c, const PointIn& in, double rhs[NFIELDS],
                                          PointExtra* extra, bool& ok) {
    const double* v = in.v;
    const double chi = v[F_CHI], K = v[F_K], Th = v[F_TH], al = v[F_LAPSE], phi = v[F_PHI], Pi = v[F_PI];
    double h[6], A[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) { h[m] = v[F_H + m]; A[m] = v[F_A + m]; }
    double hi[6];
    const double deth = sym3_inv(h, hi);
    const double ichi = 1.0 / chi;
    const double ial = 1.0 / al;

    // ---- derivatives (aliases)
#define D1(f, k) in.d1[d1slot(f)][k]
#define D2(f, m) in.d2[d2slot(f)][m]
    double dh[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 6; ++m) dh[k][m] = D1(F_H + m, k);
    double dchi[3], dal[3], dK[3], dTh[3], dphi[3], dPi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dchi[k] = D1(F_CHI, k); dal[k] = D1(F_LAPSE, k); dK[k] = D1(F_K, k);
        dTh[k] = D1(F_TH, k); dphi[k] = D1(F_PHI, k); dPi[k] = D1(F_PI, k);
    }
    double db[3][3];  // db[j][i] = d_j beta^i
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) db[j][i] = D1(F_SHIFT + i, j);
    const double divb = db[0][0] + db[1][1] + db[2][2];
    const double bx = v[F_SHIFT], by = v[F_SHIFT + 1], bz = v[F_SHIFT + 2];
#define ADV(f) (bx * D1(f, 0) + by * D1(f, 1) + bz * D1(f, 2))

    // ---- conformal Christoffels: G1[l][ij] = Gt_{l ij}, G2[k][ij] = Gt^k_ij, Gtc^k
    double G1[3][6], G2[3][6], Gtc[3];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j)
                G1[l][sidx(i, j)] = 0.5 * (dh[i][sidx(l, j)] + dh[j][sidx(l, i)] - dh[l][sidx(i, j)]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 6; ++m)
            G2[k][m] = hi[sidx(k, 0)] * G1[0][m] + hi[sidx(k, 1)] * G1[1][m] + hi[sidx(k, 2)] * G1[2][m];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        Gtc[k] = hi[0] * G2[k][0] + hi[3] * G2[k][3] + hi[5] * G2[k][5]
                 + 2.0 * (hi[1] * G2[k][1] + hi[2] * G2[k][2] + hi[4] * G2[k][4]);

    // ---- d_m Gt^k (chain rule through h^-1 and d2 h)
    double dGtc[3][3];
    {
        double Gl[3];  // G_l = h^ij Gt_lij
#pragma unroll
        for (int l = 0; l < 3; ++l)
            Gl[l] = hi[0] * G1[l][0] + hi[3] * G1[l][3] + hi[5] * G1[l][5]
                    + 2.0 * (hi[1] * G1[l][1] + hi[2] * G1[l][2] + hi[4] * G1[l][4]);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            // d_m h^ab = -h^ac d_m h_cd h^db
            double T[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    T[a][d] = hi[sidx(a, 0)] * dh[m][sidx(0, d)] + hi[sidx(a, 1)] * dh[m][sidx(1, d)]
                              + hi[sidx(a, 2)] * dh[m][sidx(2, d)];
            double dhi[6];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = a; b < 3; ++b)
                    dhi[sidx(a, b)] = -(T[a][0] * hi[sidx(0, b)] + T[a][1] * hi[sidx(1, b)] + T[a][2] * hi[sidx(2, b)]);
            double dGl[3];
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        // d_m Gt_lij = 1/2 (d_m d_i h_lj + d_m d_j h_li - d_m d_l h_ij)
                        const double dG1 = 0.5 * (D2(F_H + sidx(l, j), sidx(m, i)) + D2(F_H + sidx(l, i), sidx(m, j))
                                                  - D2(F_H + sidx(i, j), sidx(m, l)));
                        s += dhi[sidx(i, j)] * G1[l][sidx(i, j)] + hi[sidx(i, j)] * dG1;
                    }
                dGl[l] = s;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k)
                dGtc[m][k] = dhi[sidx(k, 0)] * Gl[0] + dhi[sidx(k, 1)] * Gl[1] + dhi[sidx(k, 2)] * Gl[2]
                             + hi[sidx(k, 0)] * dGl[0] + hi[sidx(k, 1)] * dGl[1] + hi[sidx(k, 2)] * dGl[2];
        }
    }

    // ---- physical Christoffels Gp^k_ij = Gt^k_ij - (d_i chi delta^k_j + d_j chi delta^k_i - h_ij h^kl d_l chi)/(2 chi)
    double hidchi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) hidchi[k] = hi[sidx(k, 0)] * dchi[0] + hi[sidx(k, 1)] * dchi[1] + hi[sidx(k, 2)] * dchi[2];
    double Gp[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                double t = -h[sidx(i, j)] * hidchi[k];
                if (k == j) t += dchi[i];
                if (k == i) t += dchi[j];
                Gp[k][sidx(i, j)] = G2[k][sidx(i, j)] - 0.5 * ichi * t;
            }

    // ---- plain Ricci tensor of gamma = h/chi (conformal decomposition)
    double Ric[6];
    {
        double DDchi[6];
#pragma unroll
        for (int m = 0; m < 6; ++m)
            DDchi[m] = D2(F_CHI, m) - G2[0][m] * dchi[0] - G2[1][m] * dchi[1] - G2[2][m] * dchi[2];
        const double lapchi = hi[0] * DDchi[0] + hi[3] * DDchi[3] + hi[5] * DDchi[5]
                              + 2.0 * (hi[1] * DDchi[1] + hi[2] * DDchi[2] + hi[4] * DDchi[4]);
        const double dchi2 = dchi[0] * hidchi[0] + dchi[1] * hidchi[1] + dchi[2] * hidchi[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                double r = 0.0;
#pragma unroll
                for (int l = 0; l < 3; ++l)
#pragma unroll
                    for (int m = 0; m < 3; ++m) r -= 0.5 * hi[sidx(l, m)] * D2(F_H + sidx(i, j), sidx(l, m));
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    r += 0.5 * (h[sidx(k, i)] * dGtc[j][k] + h[sidx(k, j)] * dGtc[i][k]);
                    r += 0.5 * Gtc[k] * (G1[i][sidx(j, k)] + G1[j][sidx(i, k)]);
#pragma unroll
                    for (int l = 0; l < 3; ++l)
#pragma unroll
                        for (int m = 0; m < 3; ++m)
                            r += hi[sidx(l, m)] * (G2[k][sidx(l, i)] * G1[j][sidx(k, m)] + G2[k][sidx(l, j)] * G1[i][sidx(k, m)]
                                                   + G2[k][sidx(i, m)] * G1[k][sidx(l, j)]);
                }
                r += 0.5 * ichi * (DDchi[sidx(i, j)] + h[sidx(i, j)] * lapchi)
                     - 0.25 * ichi * ichi * (dchi[i] * dchi[j] + 3.0 * h[sidx(i, j)] * dchi2);
                Ric[sidx(i, j)] = r;
            }
    }
    // gamma^ij = chi h^ij, gamma_ij = h_ij / chi
    double gu[6], gd[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) { gu[m] = chi * hi[m]; gd[m] = h[m] * ichi; }
#define TRU(X) (gu[0] * (X)[0] + gu[3] * (X)[3] + gu[5] * (X)[5] + 2.0 * (gu[1] * (X)[1] + gu[2] * (X)[2] + gu[4] * (X)[4]))
    const double Rs = TRU(Ric);

    // ---- Z terms: Zl_i = h_ik (Gamma-hat^k - Gt^k)/2 ; R^Z_ij = R_ij + D_i Z_j + D_j Z_i
    double dG[3], Zl[3], Zu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dG[k] = v[F_GAM + k] - Gtc[k];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Zl[i] = 0.5 * (h[sidx(i, 0)] * dG[0] + h[sidx(i, 1)] * dG[1] + h[sidx(i, 2)] * dG[2]);
        Zu[i] = 0.5 * chi * dG[i];
    }
    double RZ[6];
    {
        double dZ[3][3];  // dZ[j][i] = d_j Zl_i
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < 3; ++k) s += dh[j][sidx(i, k)] * dG[k] + h[sidx(i, k)] * (D1(F_GAM + k, j) - dGtc[j][k]);
                dZ[j][i] = 0.5 * s;
            }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                const double gz = Gp[0][sidx(i, j)] * Zl[0] + Gp[1][sidx(i, j)] * Zl[1] + Gp[2][sidx(i, j)] * Zl[2];
                RZ[sidx(i, j)] = Ric[sidx(i, j)] + dZ[i][j] + dZ[j][i] - 2.0 * gz;
            }
    }
    const double RZs = TRU(RZ);

    // ---- D_i D_j lapse, D_i D_j phi (physical)
    double DDa[6], DDp[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        DDa[m] = D2(F_LAPSE, m) - Gp[0][m] * dal[0] - Gp[1][m] * dal[1] - Gp[2][m] * dal[2];
        DDp[m] = D2(F_PHI, m) - Gp[0][m] * dphi[0] - Gp[1][m] * dphi[1] - Gp[2][m] * dphi[2];
    }
    const double lapal = TRU(DDa);

    // ---- extrinsic curvature K_ij = (A_ij + h_ij K/3)/chi and friends
    double Kp[6], Aud[3][3], Kud[3][3];
#pragma unroll
    for (int m = 0; m < 6; ++m) Kp[m] = (A[m] + h[m] * K * (1.0 / 3.0)) * ichi;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Aud[i][j] = hi[sidx(i, 0)] * A[sidx(0, j)] + hi[sidx(i, 1)] * A[sidx(1, j)] + hi[sidx(i, 2)] * A[sidx(2, j)];
            Kud[i][j] = Aud[i][j] + (i == j ? K * (1.0 / 3.0) : 0.0);
        }
    const double trK = K + Aud[0][0] + Aud[1][1] + Aud[2][2];
    double Au[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            Au[sidx(i, j)] = Aud[i][0] * hi[sidx(0, j)] + Aud[i][1] * hi[sidx(1, j)] + Aud[i][2] * hi[sidx(2, j)];
    const double AA = A[0] * Au[0] + A[3] * Au[3] + A[5] * Au[5] + 2.0 * (A[1] * Au[1] + A[2] * Au[2] + A[4] * Au[4]);
    double KK[6];  // K_ik K^k_j
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            KK[sidx(i, j)] = Kp[sidx(i, 0)] * Kud[0][j] + Kp[sidx(i, 1)] * Kud[1][j] + Kp[sidx(i, 2)] * Kud[2][j];

    // d_k K_ij, D_k K_ij, L_beta K_ij
    double dKp[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 6; ++m)
            dKp[k][m] = (D1(F_A + m, k) + (dh[k][m] * K + h[m] * dK[k]) * (1.0 / 3.0) - Kp[m] * dchi[k]) * ichi;
    double LbK[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double s = bx * dKp[0][sidx(i, j)] + by * dKp[1][sidx(i, j)] + bz * dKp[2][sidx(i, j)];
#pragma unroll
            for (int k = 0; k < 3; ++k) s += Kp[sidx(k, j)] * db[i][k] + Kp[sidx(i, k)] * db[j][k];
            LbK[sidx(i, j)] = s;
        }
    // Codazzi block: Bc[k][i][j] = D_i K_kj - D_j K_ki
    double Bc[3][3][3];
    {
        double DK[3][6];  // DK[k][ij] = D_k K_ij
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = i; j < 3; ++j) {
                    double s = dKp[k][sidx(i, j)];
#pragma unroll
                    for (int l = 0; l < 3; ++l) s -= Gp[l][sidx(k, i)] * Kp[sidx(l, j)] + Gp[l][sidx(k, j)] * Kp[sidx(i, l)];
                    DK[k][sidx(i, j)] = s;
                }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Bc[k][i][j] = (i == j) ? 0.0 : DK[i][sidx(k, j)] - DK[j][sidx(k, i)];
    }
    double Bv[3];  // B_j = gamma^ab B_abj
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) s += gu[sidx(a, b)] * Bc[a][b][j];
        Bv[j] = s;
    }

    // ---- Gauss block and its Einstein tensor
    double S[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) S[m] = Ric[m] + trK * Kp[m] - KK[m];
    const double Ss = TRU(S);
    double GS[6], GSu[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) GS[m] = S[m] - 0.5 * gd[m] * Ss;
    // raise both indices: GSu = gu GS gu
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) s += gu[sidx(i, a)] * GS[sidx(a, b)] * gu[sidx(b, j)];
            GSu[sidx(i, j)] = s;
        }

    // ---- scalar: nabla nabla phi blocks, Phi = nabla nabla beta(phi)
    double b1, b2;
    if (c.beta_kind == 1) { b1 = c.lam * phi; b2 = c.lam; } else { b1 = c.lam; b2 = 0.0; }
    double dphiu[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dphiu[i] = gu[sidx(i, 0)] * dphi[0] + gu[sidx(i, 1)] * dphi[1] + gu[sidx(i, 2)] * dphi[2];
    const double dphi2 = dphi[0] * dphiu[0] + dphi[1] * dphiu[1] + dphi[2] * dphiu[2];
    const double X = 0.5 * (Pi * Pi - dphi2);
    const double g2 = c.g2;
    double Hij[6], Hn[3];
#pragma unroll
    for (int m = 0; m < 6; ++m) Hij[m] = DDp[m] + Kp[m] * Pi;
#pragma unroll
    for (int i = 0; i < 3; ++i) Hn[i] = dPi[i] + Kud[0][i] * dphi[0] + Kud[1][i] * dphi[1] + Kud[2][i] * dphi[2];
    double Phd[6], Phn[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Phn[i] = b1 * Hn[i] + b2 * Pi * dphi[i];
#pragma unroll
        for (int j = i; j < 3; ++j) Phd[sidx(i, j)] = b1 * Hij[sidx(i, j)] + b2 * dphi[i] * dphi[j];
    }
    double Phm[3][3], Phu[6], Phnu[3];  // Phi_i^k, Phi^ij, Phi_n^k
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            Phm[i][k] = Phd[sidx(i, 0)] * gu[sidx(0, k)] + Phd[sidx(i, 1)] * gu[sidx(1, k)] + Phd[sidx(i, 2)] * gu[sidx(2, k)];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = i; j < 3; ++j)
            Phu[sidx(i, j)] = gu[sidx(i, 0)] * Phm[0][j] + gu[sidx(i, 1)] * Phm[1][j] + gu[sidx(i, 2)] * Phm[2][j];
        Phnu[i] = gu[sidx(i, 0)] * Phn[0] + gu[sidx(i, 1)] * Phn[1] + gu[sidx(i, 2)] * Phn[2];
    }
    const double trP = Phm[0][0] + Phm[1][1] + Phm[2][2];

    // ---- sources that do not depend on the unknowns
    const double fX = 1.0 + 2.0 * g2 * X;
    double rho8 = 0.5 * fX * Pi * Pi - 0.5 * (X + g2 * X * X);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) rho8 -= 4.0 * GS[sidx(i, j)] * Phu[sidx(i, j)];
    double S8[3];
    const double BPn = Bv[0] * Phnu[0] + Bv[1] * Phnu[1] + Bv[2] * Phnu[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double s = GS[sidx(i, 0)] * Phnu[0] + GS[sidx(i, 1)] * Phnu[1] + GS[sidx(i, 2)] * Phnu[2]
                   - (Phm[i][0] * Bv[0] + Phm[i][1] * Bv[1] + Phm[i][2] * Bv[2]) + trP * Bv[i];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) s += Bc[k][i][l] * Phu[sidx(k, l)];
        S8[i] = -0.5 * fX * Pi * dphi[i] + 4.0 * s;
    }
    // first-order S_ij and the Y_ij (mixed-block) part of the Gauss-Bonnet S_ij
    double S1[6], Y[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            S1[sidx(i, j)] = 0.5 * fX * dphi[i] * dphi[j] + 0.5 * gd[sidx(i, j)] * (X + g2 * X * X);
            double y = 0.0;
#pragma unroll
            for (int l = 0; l < 3; ++l) y += (Bc[i][j][l] + Bc[j][i][l]) * Phnu[l];
            Y[sidx(i, j)] = y - 2.0 * gd[sidx(i, j)] * BPn + Bv[j] * Phn[i] + Bv[i] * Phn[j];
        }
    // C0 = C at d_t K_ij = 0
    double C0[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) C0[m] = (DDa[m] - LbK[m]) * ial + KK[m];
    const double bdPi = bx * dPi[0] + by * dPi[1] + bz * dPi[2];
    const double dadp = dal[0] * dphiu[0] + dal[1] * dphiu[1] + dal[2] * dphiu[2];
    const double Phnn0 = b1 * (-bdPi - dadp) * ial + b2 * Pi * Pi;
    // L_GB at d_t K_ij = 0
    double L0;
    {
        double gc = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) gc += GSu[sidx(i, j)] * C0[sidx(i, j)];
        // B_kij B^kij through the dual b_k^m = B_k,(m+1)(m+2):  = 2 chi^3/det(h) h^kk' h_mm' b_k^m b_k'^m'
        double bb[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) { bb[k][0] = Bc[k][1][2]; bb[k][1] = Bc[k][2][0]; bb[k][2] = Bc[k][0][1]; }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                double t = 0.0;
#pragma unroll
                for (int m = 0; m < 3; ++m)
#pragma unroll
                    for (int mm = 0; mm < 3; ++mm) t += h[sidx(m, mm)] * bb[k][m] * bb[kk][mm];
                s += hi[sidx(k, kk)] * t;
            }
        const double BB = 2.0 * chi * chi * chi / deth * s;
        const double BvBv = Bv[0] * (gu[0] * Bv[0] + gu[1] * Bv[1] + gu[2] * Bv[2])
                            + Bv[1] * (gu[1] * Bv[0] + gu[3] * Bv[1] + gu[4] * Bv[2])
                            + Bv[2] * (gu[2] * Bv[0] + gu[4] * Bv[1] + gu[5] * Bv[2]);
        L0 = 8.0 * gc - 4.0 * BB + 8.0 * BvBv;
    }

    // ---- CCZ4 right-hand sides without S_ij (rho and S_i included)
    rhs[F_CHI] = ADV(F_CHI) + (2.0 / 3.0) * chi * (al * K - divb);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double x = ADV(F_H + sidx(i, j)) - (2.0 / 3.0) * h[sidx(i, j)] * divb - 2.0 * al * A[sidx(i, j)];
#pragma unroll
            for (int k = 0; k < 3; ++k) x += h[sidx(i, k)] * db[j][k] + h[sidx(j, k)] * db[i][k];
            rhs[F_H + sidx(i, j)] = x;
        }
    const double Kdot0 = ADV(F_K) + al * (RZs + K * (K - 2.0 * Th)) - 3.0 * al * c.kappa1 * (1.0 + c.kappa2) * Th
                         - lapal - 1.5 * al * rho8
                         - c.bK * al * (Rs - AA + (2.0 / 3.0) * K * K - 2.0 * rho8);
    double Adot0[6];
    {
        double Xa[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) Xa[m] = -DDa[m] + al * RZ[m];
        const double trX = hi[0] * Xa[0] + hi[3] * Xa[3] + hi[5] * Xa[5] + 2.0 * (hi[1] * Xa[1] + hi[2] * Xa[2] + hi[4] * Xa[4]);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                double x = ADV(F_A + sidx(i, j)) + chi * (Xa[sidx(i, j)] - h[sidx(i, j)] * trX * (1.0 / 3.0))
                           + al * (K - 2.0 * Th) * A[sidx(i, j)] - (2.0 / 3.0) * A[sidx(i, j)] * divb;
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    x += -2.0 * al * A[sidx(i, k)] * Aud[k][j] + A[sidx(i, k)] * db[j][k] + A[sidx(j, k)] * db[i][k];
                Adot0[sidx(i, j)] = x;
            }
    }
    rhs[F_TH] = ADV(F_TH) + c.bTh * al * (RZs - AA + (2.0 / 3.0) * K * K - 2.0 * Th * K - 2.0 * rho8)
                - (Zu[0] * dal[0] + Zu[1] * dal[1] + Zu[2] * dal[2]) - al * c.kappa1 * (2.0 + c.kappa2) * Th;
    {
        double hZ[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) hZ[i] = hi[sidx(i, 0)] * Zl[0] + hi[sidx(i, 1)] * Zl[1] + hi[sidx(i, 2)] * Zl[2];
        double ddbk[3];  // sum_k d_j d_k beta^k
#pragma unroll
        for (int j = 0; j < 3; ++j) ddbk[j] = D2(F_SHIFT, sidx(j, 0)) + D2(F_SHIFT + 1, sidx(j, 1)) + D2(F_SHIFT + 2, sidx(j, 2));
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0, t5 = 0.0, t6 = 0.0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    t1 += G2[i][sidx(j, k)] * Au[sidx(j, k)];
                    t5 += hi[sidx(j, k)] * D2(F_SHIFT + i, sidx(j, k));
                    t6 += hi[sidx(j, k)] * Zl[j] * db[k][i];
                }
                t2 += Au[sidx(i, j)] * dchi[j];
                t3 += hi[sidx(i, j)] * dK[j];
                t4 += Au[sidx(i, j)] * dal[j];
            }
            double x = ADV(F_GAM + i) + 2.0 * al * (t1 - 1.5 * ichi * t2 - (2.0 / 3.0) * t3) - 2.0 * t4 + t5;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                x += 2.0 * hi[sidx(k, i)] * (al * dTh[k] - Th * dal[k] - (2.0 / 3.0) * al * K * Zl[k]);
                x += (1.0 / 3.0) * hi[sidx(i, k)] * ddbk[k] - Gtc[k] * db[k][i];
            }
            x += (2.0 / 3.0) * Gtc[i] * divb + 2.0 * c.kappa3 * ((2.0 / 3.0) * hZ[i] * divb - t6)
                 - 2.0 * al * c.kappa1 * hZ[i]
                 - 2.0 * al * (hi[sidx(i, 0)] * S8[0] + hi[sidx(i, 1)] * S8[1] + hi[sidx(i, 2)] * S8[2]);
            rhs[F_GAM + i] = x;
            rhs[F_B + i] = x - c.eta * v[F_B + i];
            rhs[F_SHIFT + i] = c.shift_F * v[F_B + i] * c.inv_1pa
                               - c.a_1pa * al * chi * (hi[sidx(i, 0)] * dal[0] + hi[sidx(i, 1)] * dal[1] + hi[sidx(i, 2)] * dal[2]);
        }
    }
    rhs[F_LAPSE] = ADV(F_LAPSE) - 2.0 * al * (K - 2.0 * Th) * c.inv_1pa;
    rhs[F_PHI] = al * Pi + ADV(F_PHI);

    // ---- coupled system for v = (d_t K_ij, d_t Pi)
    double Msys[7][8];
    {
        // U0_ij: d_t K_ij implied by the S_ij-free right-hand sides
        const double chid = rhs[F_CHI];
        double LGS[6], rr[6], QC0[6], LS1[6], LY[6];
        const double trS1 = TRU(S1), trY = TRU(Y);
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            LGS[m] = S[m] - 0.25 * gd[m] * Ss;
            LS1[m] = S1[m] - 0.5 * gd[m] * trS1;
            LY[m] = Y[m] - 0.5 * gd[m] * trY;
        }
        apply_LQ(C0, gd, gu, Phd, Phu, Phm, trP, QC0);  // = L(Q(C0))
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const double U0 = (Adot0[m] + (rhs[F_H + m] * K + h[m] * Kdot0) * (1.0 / 3.0) - Kp[m] * chid) * ichi;
            rr[m] = U0 - al * LS1[m] + 4.0 * al * (LGS[m] * Phnn0 + LY[m] + QC0[m]);
        }
        // u-rows: u - 4 L(Q(u)) - 4 b1 L(G_S) w = r
#pragma unroll
        for (int col = 0; col < 6; ++col) {
            double e[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            e[col] = 1.0;
            double q[6];
            apply_LQ(e, gd, gu, Phd, Phu, Phm, trP, q);
#pragma unroll
            for (int row = 0; row < 6; ++row) Msys[row][col] = (row == col ? 1.0 : 0.0) - 4.0 * q[row];
        }
#pragma unroll
        for (int row = 0; row < 6; ++row) {
            Msys[row][6] = -4.0 * b1 * LGS[row];
            Msys[row][7] = rr[row];
        }
        // w-row: w - (8 b1 / D) G_S^ij u_ij = r_w
        const double Dphi = fX + 2.0 * g2 * Pi * Pi;
        const double iD = 1.0 / Dphi;
#pragma unroll
        for (int col = 0; col < 6; ++col) {
            const bool off = (col == 1 || col == 2 || col == 4);
            Msys[6][col] = -8.0 * b1 * iD * GSu[col] * (off ? 2.0 : 1.0);
        }
        Msys[6][6] = 1.0;
        const double trH = TRU(Hij);
        double Hnd = 0.0, Hdd = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Hnd += dphiu[i] * Hn[i];
#pragma unroll
            for (int j = 0; j < 3; ++j) Hdd += dphiu[i] * dphiu[j] * Hij[sidx(i, j)];
        }
        Msys[6][7] = bdPi + dadp + al * iD * (fX * trH + 4.0 * g2 * Pi * Hnd - 2.0 * g2 * Hdd + b1 * L0);
    }
    ok = solve7(Msys);
    double u[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) u[m] = Msys[m][7];
    const double w = Msys[6][7];

    // ---- full S_ij at the solution and the final K, A_ij, Pi right-hand sides
    {
        double Cs[6], QC[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) Cs[m] = C0[m] + u[m] * ial;
        // Q(C) itself (not trace-reversed): Q = L(Q) + gamma tr(Q)/2 ... compute directly
        double CP = 0.0, trC = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                CP += Cs[sidx(i, j)] * Phu[sidx(i, j)];
                trC += Cs[sidx(i, j)] * gu[sidx(i, j)];
            }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                double pc = 0.0;
#pragma unroll
                for (int k = 0; k < 3; ++k) pc += Phm[i][k] * Cs[sidx(k, j)] + Phm[j][k] * Cs[sidx(i, k)];
                QC[sidx(i, j)] = gd[sidx(i, j)] * CP - pc + trP * Cs[sidx(i, j)] - trC * (gd[sidx(i, j)] * trP - Phd[sidx(i, j)]);
            }
        const double Phnn = Phnn0 + b1 * w * ial;
        double S8ij[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) S8ij[m] = S1[m] - 4.0 * (GS[m] * Phnn + Y[m] + QC[m]);
        const double Ss8 = TRU(S8ij);
        rhs[F_K] = Kdot0 + 0.5 * al * Ss8;
        const double trh = hi[0] * S8ij[0] + hi[3] * S8ij[3] + hi[5] * S8ij[5]
                           + 2.0 * (hi[1] * S8ij[1] + hi[2] * S8ij[2] + hi[4] * S8ij[4]);
#pragma unroll
        for (int m = 0; m < 6; ++m) rhs[F_A + m] = Adot0[m] - al * chi * (S8ij[m] - h[m] * trh * (1.0 / 3.0));
        rhs[F_PI] = w;
    }
    if (extra) {
        extra->ham = Ss - 2.0 * rho8;
#pragma unroll
        for (int i = 0; i < 3; ++i) extra->mom[i] = Bv[i] - S8[i];
    }
#undef D1
#undef D2
#undef ADV
#undef TRU
}

}  // namespace grf
