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
//
// The cubic Horndeski term (1/16 pi) g3 X box(phi) (general instantiation, COUP = 1) adds, with
// H = nabla nabla phi in the same basis (H_nn holding d_t Pi, H_ni, H_ij = D_i D_j phi + K_ij Pi),
//     8 pi rho3  = g3/2 (Pi^2 tr H - H(dphi, dphi))
//     8 pi S3_i  = -g3/2 [(Pi tr H - H_n(dphi)) d_i phi + Pi^2 H_ni - Pi H_ik d^k phi]
//     8 pi S3_ij = g3 [1/2 H_nn (Pi^2 gamma_ij - d_i phi d_j phi) + 1/2 tr H d_i phi d_j phi
//                      + Pi H_n(i d_j) phi - H_(i|k d^k phi d_|j) phi + gamma_ij (H(dphi, dphi)/2 - Pi H_n(dphi))]
// to the metric equations, and to the scalar equation
//     g3 [box(phi)^2 - H_ab H^ab - R_ab d^a phi d^b phi],
// in which H_nn^2 cancels: -2 H_nn tr H + (tr H)^2 + 2 H_n.H_n - H_ij H^ij
// - (Pi^2 gamma^kl - d^k phi d^l phi) C_kl - 2 Pi B^i d_i phi - S_ij d^i phi d^j phi
// (4D Ricci: R_nn = tr C, R_ni = -B_i, R_ij = S_ij - C_ij). The system stays affine in the unknowns.
#pragma once

#include <type_traits>

#ifdef __CUDACC__
#include <cuda_runtime.h>
#define GRF_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define GRF_HD inline
#define __host__
#define __device__
#endif

// Section markers: no-ops in the CUDA build; the host operation-counting build defines them
// to attribute FP64 operations to the parts of the algorithm.
#ifndef GRF_SECTION
#define GRF_SECTION(id)
#endif
// Marks a value as data (not a known constant) in the counting build: compare-and-exchange
// pivoting turns every swapped entry into a runtime value.
#ifndef GRF_OPAQUE
#define GRF_OPAQUE(x)
#endif

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

// Per-launch coefficients. P is the type of the two couplings (double, or a dual number when
// their tangents are propagated).
template <typename P>
struct CoeffsT {
    double kappa1, kappa2, kappa3, shift_F, eta;
    P lam, g2;
    double inv_1pa, a_1pa;        // 1/(1+a), a/(1+a)
    double bK, bTh;               // 3b/(4(1+b)), 1/(2(1+b))
    int beta_kind;
    double beta_kappa;  // kappa of the exponential coupling (beta_kind 2)
    int decoupled;  // 1: the scalar's stress-energy is left out of the metric equations
    int advection;  // 1: lopsided advection derivatives (kernels instantiated with LOP = 1)
    double g3;      // cubic Horndeski coupling (read only by COUP = 1 instances)
};
using Coeffs = CoeffsT<double>;

template <typename T>
struct PointInT {
    T v[NFIELDS];
    T d1[24][3];
    T d2[12][6];
};
using PointIn = PointInT<double>;

// Output diagnostics besides the RHS (constraints come out as by-products).
template <typename T>
struct PointExtraT {
    T ham;      // H = S - 2 (8 pi rho)
    T mom[3];   // M_i = B_i - 8 pi S_i
    T rho8[3];  // 8 pi rho of the X, g2 X^2 and beta(phi) L_GB terms of the action (their sum is
                // the 8 pi rho of the equations when g3 = 0; reported with and without backreaction)
    // Weyl scalar Psi_4 (double instances only), computed when want_psi4 is set: xyz are the
    // point's coordinates relative to the origin of the tetrad's triad.
    int want_psi4 = 0;
    double xyz[3];
    T psi4[2];
    // Hyperbolicity diagnostics (double instances only), computed when want_hyp is set:
    //   hyp[0] = det M of the coupled system for (d_t K_ij, d_t Pi), normalised so that each
    //            unknown's own coefficient is 1 (M = identity without coupling); where it
    //            vanishes the equations no longer determine the time derivatives;
    //   hyp[1] = det(g_eff^ab) / det(g^ab) of the scalar equation's principal symbol
    //            g_eff^ab = (1 + 2 g2 X) g^ab - 2 g2 d^a phi d^b phi + 2 g3 (box(phi) g^ab - H^ab);
    //            for g3 = 0, by the matrix determinant lemma, (1 + 2 g2 X)^3 (1 + 6 g2 X);
    //   hyp[2] = -g_eff^nn = 1 + 2 g2 X + 2 g2 Pi^2 + 2 g3 tr H (the coefficient of d_t Pi; the
    //            normal is timelike for the scalar's characteristic cone while it is positive);
    //   hyp[3] = the smallest pivot of partial-pivoting elimination of M over its largest entry.
    int want_hyp = 0;
    double hyp[4];
};
using PointExtra = PointExtraT<double>;

template <typename T>
GRF_HD T sym3_det(const T h[6]) {
    return h[0] * (h[3] * h[5] - h[4] * h[4]) - h[1] * (h[1] * h[5] - h[4] * h[2])
           + h[2] * (h[1] * h[4] - h[3] * h[2]);
}

// symmetric inverse; returns determinant
template <typename T>
GRF_HD T sym3_inv(const T h[6], T hi[6], T& id) {
    const T c00 = h[3] * h[5] - h[4] * h[4];
    const T c01 = h[2] * h[4] - h[1] * h[5];
    const T c02 = h[1] * h[4] - h[2] * h[3];
    const T det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    id = 1.0 / det;
    hi[0] = c00 * id;
    hi[1] = c01 * id;
    hi[2] = c02 * id;
    hi[3] = (h[0] * h[5] - h[2] * h[2]) * id;
    hi[4] = (h[1] * h[2] - h[0] * h[4]) * id;
    hi[5] = (h[0] * h[3] - h[1] * h[1]) * id;
    return det;
}

// |a| > |b|, and the largest |M_ij| of the 7x7 block. For doubles on the device both run on the
// integer pipe: with the sign bit cleared, the bit patterns of non-NaN doubles order like their
// magnitudes (a NaN entry makes the maximum a NaN, which then fails every pivot test).
template <typename T>
GRF_HD bool abs_gt(const T& a, const T& b) { return fabs(a) > fabs(b); }
template <typename T>
GRF_HD T abs_max7(const T M[7][8]) {
    T mx = 0.0;
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int j = 0; j < 7; ++j) mx = fmax(mx, fabs(M[i][j]));
    return mx;
}
#ifdef __CUDA_ARCH__
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }
__device__ __forceinline__ bool abs_gt(double a, double b) { return abs_bits(a) > abs_bits(b); }
__device__ __forceinline__ double abs_max7(const double M[7][8]) {
    long long m = 0;
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int j = 0; j < 7; ++j) m = max(m, abs_bits(M[i][j]));
    return __longlong_as_double(m);
}
#endif

// Determinant of the 7x7 block of M (a copy, Gaussian elimination with partial pivoting and the
// sign of each row exchange), and in *ratio the smallest pivot magnitude over the block's largest
// entry magnitude. Diagnostics only.
GRF_HD double det7(const double M[7][8], double* ratio) {
    double A[7][7], mx = 0.0, mn = -1.0;
    for (int i = 0; i < 7; ++i)
        for (int j = 0; j < 7; ++j) { A[i][j] = M[i][j]; mx = fmax(mx, fabs(A[i][j])); }
    *ratio = 0.0;
    double det = 1.0;
    for (int k = 0; k < 7; ++k) {
        int piv = k;
        for (int i = k + 1; i < 7; ++i)
            if (fabs(A[i][k]) > fabs(A[piv][k])) piv = i;
        const double pm = fabs(A[piv][k]);
        mn = (mn < 0.0 || pm < mn) ? pm : mn;
        if (A[piv][k] == 0.0) return 0.0;
        if (piv != k) {
            for (int j = 0; j < 7; ++j) {
                const double t = A[k][j];
                A[k][j] = A[piv][j];
                A[piv][j] = t;
            }
            det = -det;
        }
        det *= A[k][k];
        for (int i = k + 1; i < 7; ++i) {
            const double f = A[i][k] / A[k][k];
            for (int j = k + 1; j < 7; ++j) A[i][j] -= f * A[k][j];
        }
    }
    *ratio = mx > 0.0 ? mn / mx : 0.0;
    return det;
}

// 7x7 LU with partial pivoting (row swaps by compare-and-exchange, so every index stays a
// compile-time constant and the matrix stays in registers); the pivot rows are not normalised,
// the back substitution multiplies by the stored pivot reciprocals. Returns false on a pivot
// not larger than 1e-300 times the largest entry.
template <typename T>
GRF_HD bool solve7(T M[7][8]) {
    const T thr = 1e-300 * abs_max7(M);
    bool ok = true;
    T ipv[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
#pragma unroll
        for (int i = k + 1; i < 7; ++i) {
            const bool sw = abs_gt(M[i][k], M[k][k]);
#pragma unroll
            for (int j = k; j < 8; ++j) {
                const T a = M[k][j], b = M[i][j];
                M[k][j] = sw ? b : a;
                M[i][j] = sw ? a : b;
                GRF_OPAQUE(M[k][j]);
                GRF_OPAQUE(M[i][j]);
            }
        }
        ok = ok && abs_gt(M[k][k], thr);
        const T ip = 1.0 / M[k][k];
        ipv[k] = ip;
#pragma unroll
        for (int i = k + 1; i < 7; ++i) {
            const T f = M[i][k] * ip;
#pragma unroll
            for (int j = k + 1; j < 8; ++j) M[i][j] = fma(-f, M[k][j], M[i][j]);
        }
    }
#pragma unroll
    for (int k = 6; k >= 0; --k) {
        T x = M[k][7];
#pragma unroll
        for (int j = k + 1; j < 7; ++j) x = fma(-M[k][j], M[j][7], x);
        M[k][7] = x * ipv[k];
    }
    return ok;
}

// sum_ij a_ij b^ij for symmetric a, b stored as 6 components, with `bw` = b with the three
// off-diagonal components pre-multiplied by 2.
template <typename T>
GRF_HD T sdotw(const T a[6], const T bw[6]) {
    return a[0] * bw[0] + a[1] * bw[1] + a[2] * bw[2] + a[3] * bw[3] + a[4] * bw[4] + a[5] * bw[5];
}

// Levi-Civita bookkeeping of the Codazzi block: B_kij (antisymmetric in ij) is stored through
// its dual bb[k][m] = B_{k,(m+1)%3,(m+2)%3}; B_kij = +-bb[k][3-i-j] for i != j.
__host__ __device__ constexpr int third(int i, int j) { return 3 - i - j; }
__host__ __device__ constexpr bool cyclic(int i, int j) { return (j - i + 3) % 3 == 1; }

// Q_ij(X) = P_ikjl X^kl-type contraction: the Gauss-Bonnet S_ij is -4 [... + Q_ij(C)] with
//   Q_ij(X) = gamma_ij (X.Phi) - Phi_i^k X_kj - Phi_j^k X_ik + tr(Phi) X_ij - tr(X)(gamma_ij tr(Phi) - Phi_ij)
template <typename T>
GRF_HD void q_of(const T X[6], const T gd[6], const T gw[6], const T Phd[6], const T Phuw[6], const T Phm[3][3], T trP,
                 T out[6]) {
    const T XP = sdotw(X, Phuw);
    const T trX = sdotw(X, gw);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            T pu = Phm[i][0] * X[sidx(0, j)];
            pu = fma(Phm[i][1], X[sidx(1, j)], pu);
            pu = fma(Phm[i][2], X[sidx(2, j)], pu);
            pu = fma(Phm[j][0], X[sidx(i, 0)], pu);
            pu = fma(Phm[j][1], X[sidx(i, 1)], pu);
            pu = fma(Phm[j][2], X[sidx(i, 2)], pu);
            out[sidx(i, j)] = gd[sidx(i, j)] * (XP - trX * trP) - pu + trP * X[sidx(i, j)] + trX * Phd[sidx(i, j)];
        }
}

// DEC: the decoupled mode as a compile-time constant (0: full theory, 1: no backreaction), or -1
// to read c.decoupled at run time.
// LOP = 1: every advection term beta^k d_k u of an evolved field (the CCZ4 advection terms and
// the shift-contracted derivatives of K_ij and Pi inside the coupled system) is taken from
// adv[27], the lopsided differences; all other derivatives stay centred. adv is not read when
// LOP = 0. COUP = 0 compiles the linear and quadratic couplings only (the exponential one is then
// routed to another instantiation by the host).
template <typename T, typename P = double, int DEC = -1, int LOP = 0, int COUP = 1>
GRF_HD void point_rhs(const CoeffsT<P>& c, const PointInT<T>& in, T rhs[NFIELDS], PointExtraT<T>* extra, bool& ok,
                      const T* adv = nullptr) {
    GRF_SECTION(0);
    const T* v = in.v;
    const T chi = v[F_CHI], K = v[F_K], Th = v[F_TH], al = v[F_LAPSE], phi = v[F_PHI], Pi = v[F_PI];
    T h[6], A[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) { h[m] = v[F_H + m]; A[m] = v[F_A + m]; }
    T hi[6], ideth;
    sym3_inv(h, hi, ideth);
    const T ichi = 1.0 / chi;
    const T ial = 1.0 / al;
    // weighted inverses (off-diagonals doubled) for symmetric contractions; gamma^ij = chi h^ij
    T hw[6], gu[6], gw[6], gd[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const bool off = (m == 1 || m == 2 || m == 4);
        hw[m] = off ? 2.0 * hi[m] : hi[m];
        gu[m] = chi * hi[m];
        gw[m] = chi * hw[m];
        gd[m] = h[m] * ichi;
    }

    GRF_SECTION(1);
#define D1(f, k) in.d1[d1slot(f)][k]
#define D2(f, m) in.d2[d2slot(f)][m]
    T dh[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 6; ++m) dh[k][m] = D1(F_H + m, k);
    T dchi[3], dal[3], dK[3], dTh[3], dphi[3], dPi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dchi[k] = D1(F_CHI, k); dal[k] = D1(F_LAPSE, k); dK[k] = D1(F_K, k);
        dTh[k] = D1(F_TH, k); dphi[k] = D1(F_PHI, k); dPi[k] = D1(F_PI, k);
    }
    T db[3][3];  // db[j][i] = d_j beta^i
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) db[j][i] = D1(F_SHIFT + i, j);
    const T divb = db[0][0] + db[1][1] + db[2][2];
    const T bx = v[F_SHIFT], by = v[F_SHIFT + 1], bz = v[F_SHIFT + 2];
#define ADV(f) (LOP ? adv[f] : (bx * D1(f, 0) + by * D1(f, 1) + bz * D1(f, 2)))

    // ---- conformal Christoffels: G1[l][ij] = Gt_{l ij}, G2[k][ij] = Gt^k_ij,
    //      Gl_l = h^ij Gt_lij (= h_lk Gt^k), Gtc^k = h^kl Gl_l
    GRF_SECTION(2);
    T G1[3][6], G2[3][6], Gl[3], Gtc[3];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j)
                G1[l][sidx(i, j)] = 0.5 * (dh[i][sidx(l, j)] + dh[j][sidx(l, i)] - dh[l][sidx(i, j)]);
#pragma unroll
    for (int l = 0; l < 3; ++l) Gl[l] = sdotw(G1[l], hw);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Gtc[k] = hi[sidx(k, 0)] * Gl[0] + hi[sidx(k, 1)] * Gl[1] + hi[sidx(k, 2)] * Gl[2];
#pragma unroll
        for (int m = 0; m < 6; ++m)
            G2[k][m] = hi[sidx(k, 0)] * G1[0][m] + hi[sidx(k, 1)] * G1[1][m] + hi[sidx(k, 2)] * G1[2][m];
    }

    // ---- dGl[m][l] = d_m Gl_l = d_m h^ij Gt_lij + h^ij d_m d_i h_lj - h^ij d_m d_l h_ij / 2
    GRF_SECTION(3);
    T dGl[3][3];
    T hdd[6];  // h^pq d_m d_l h_pq, symmetric in (m, l)
#pragma unroll
    for (int ml = 0; ml < 6; ++ml) {
        T b = hw[0] * D2(F_H + 0, ml);
#pragma unroll
        for (int q = 1; q < 6; ++q) b = fma(hw[q], D2(F_H + q, ml), b);
        hdd[ml] = b;
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        T Tm[3][3];  // h^ac d_m h_cd
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d)
                Tm[a][d] = hi[sidx(a, 0)] * dh[m][sidx(0, d)] + hi[sidx(a, 1)] * dh[m][sidx(1, d)]
                           + hi[sidx(a, 2)] * dh[m][sidx(2, d)];
        T dhiw[6];  // -(h^-1 d_m h h^-1), off-diagonals doubled
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) {
                const T x = Tm[a][0] * hi[sidx(0, b)] + Tm[a][1] * hi[sidx(1, b)] + Tm[a][2] * hi[sidx(2, b)];
                dhiw[sidx(a, b)] = (a == b) ? -x : -2.0 * x;
            }
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            T s = sdotw(G1[l], dhiw);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) s = fma(hi[sidx(i, j)], D2(F_H + sidx(l, j), sidx(m, i)), s);
            dGl[m][l] = fma(-0.5, hdd[sidx(m, l)], s);
        }
    }

    // ---- physical Christoffels Gp^k_ij = Gt^k_ij - (delta^k_i d_j chi + delta^k_j d_i chi - h_ij h^kl d_l chi)/(2 chi)
    GRF_SECTION(4);
    T hidchi[3], c1[3], c2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        hidchi[k] = hi[sidx(k, 0)] * dchi[0] + hi[sidx(k, 1)] * dchi[1] + hi[sidx(k, 2)] * dchi[2];
        c1[k] = (0.5 * ichi) * dchi[k];
        c2[k] = (0.5 * ichi) * hidchi[k];
    }
    T Gp[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                T t = fma(h[sidx(i, j)], c2[k], G2[k][sidx(i, j)]);
                if (k == j) t = t - c1[i];
                if (k == i) t = t - c1[j];
                Gp[k][sidx(i, j)] = t;
            }

    // ---- plain Ricci tensor of gamma = h/chi:
    // R_ij = -1/2 h^lm d_l d_m h_ij + d_(i Gl_j) - Gt^k Gt_kij
    //        + h^lm (Gt^k_li Gt_jkm + Gt^k_lj Gt_ikm + Gt^k_im Gt_klj) + chi part
    GRF_SECTION(5);
    T Ric[6];
    {
        T U[3][3][3];  // U[k][m][i] = h^lm Gt^k_li
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    U[k][m][i] = hi[sidx(0, m)] * G2[k][sidx(0, i)] + hi[sidx(1, m)] * G2[k][sidx(1, i)]
                                 + hi[sidx(2, m)] * G2[k][sidx(2, i)];
        T Q1[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T s = 0.0;
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        s = (k == 0 && m == 0) ? U[0][0][i] * G1[j][0] : fma(U[k][m][i], G1[j][sidx(k, m)], s);
                Q1[i][j] = s;
            }
        T DDchi[6];
#pragma unroll
        for (int m = 0; m < 6; ++m)
            DDchi[m] = D2(F_CHI, m) - G2[0][m] * dchi[0] - G2[1][m] * dchi[1] - G2[2][m] * dchi[2];
        const T lapchi = sdotw(DDchi, hw);
        const T dchi2 = dchi[0] * hidchi[0] + dchi[1] * hidchi[1] + dchi[2] * hidchi[2];
        const T hichi = 0.5 * ichi, qichi2 = -0.25 * ichi * ichi;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                T r = Q1[i][j] + Q1[j][i] + 0.5 * (dGl[j][i] + dGl[i][j]);
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int l = 0; l < 3; ++l) r = fma(U[k][l][i], G1[k][sidx(l, j)], r);
#pragma unroll
                for (int k = 0; k < 3; ++k) r = fma(-Gtc[k], G1[k][sidx(i, j)], r);
#pragma unroll
                for (int q = 0; q < 6; ++q) r = fma(-0.5 * hw[q], D2(F_H + sidx(i, j), q), r);
                r = fma(hichi, fma(h[sidx(i, j)], lapchi, DDchi[sidx(i, j)]), r);
                r = fma(qichi2, fma(3.0 * h[sidx(i, j)], dchi2, dchi[i] * dchi[j]), r);
                Ric[sidx(i, j)] = r;
            }
    }
    const T Rs = sdotw(Ric, gw);

    // ---- Z terms: Zl_i = (h_ik Gamma-hat^k - Gl_i)/2, R^Z_ij = R_ij + D_i Z_j + D_j Z_i
    GRF_SECTION(6);
    T dG[3], Zl[3], Zu[3];
    const T Gh[3] = {v[F_GAM], v[F_GAM + 1], v[F_GAM + 2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dG[k] = Gh[k] - Gtc[k];
        Zu[k] = (0.5 * chi) * dG[k];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
        Zl[i] = 0.5 * (h[sidx(i, 0)] * Gh[0] + h[sidx(i, 1)] * Gh[1] + h[sidx(i, 2)] * Gh[2] - Gl[i]);
    T RZ[6];
    {
        T dZ[3][3];  // dZ[j][i] = d_j Zl_i
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T s = -dGl[j][i];
#pragma unroll
                for (int k = 0; k < 3; ++k) s = fma(dh[j][sidx(i, k)], Gh[k], fma(h[sidx(i, k)], D1(F_GAM + k, j), s));
                dZ[j][i] = 0.5 * s;
            }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                const T gz = Gp[0][sidx(i, j)] * Zl[0] + Gp[1][sidx(i, j)] * Zl[1] + Gp[2][sidx(i, j)] * Zl[2];
                RZ[sidx(i, j)] = fma(-2.0, gz, Ric[sidx(i, j)] + (dZ[i][j] + dZ[j][i]));
            }
    }
    const T RZs = sdotw(RZ, gw);

    // ---- D_i D_j lapse, D_i D_j phi (physical)
    GRF_SECTION(7);
    T DDa[6], DDp[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        DDa[m] = D2(F_LAPSE, m) - Gp[0][m] * dal[0] - Gp[1][m] * dal[1] - Gp[2][m] * dal[2];
        DDp[m] = D2(F_PHI, m) - Gp[0][m] * dphi[0] - Gp[1][m] * dphi[1] - Gp[2][m] * dphi[2];
    }
    const T lapal = sdotw(DDa, gw);

    // ---- extrinsic curvature K_ij = (A_ij + h_ij K/3)/chi and friends
    GRF_SECTION(8);
    const T K3 = K * (1.0 / 3.0);
    T Kp[6], Aud[3][3];
#pragma unroll
    for (int m = 0; m < 6; ++m) Kp[m] = fma(h[m], K3, A[m]) * ichi;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Aud[i][j] = hi[sidx(i, 0)] * A[sidx(0, j)] + hi[sidx(i, 1)] * A[sidx(1, j)] + hi[sidx(i, 2)] * A[sidx(2, j)];
    // K^i_j = A^i_j + delta^i_j K/3
    auto Kud = [&](int i, int j) -> T { return i == j ? Aud[i][j] + K3 : Aud[i][j]; };
    const T trK = K + Aud[0][0] + Aud[1][1] + Aud[2][2];
    T Au[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            Au[sidx(i, j)] = Aud[i][0] * hi[sidx(0, j)] + Aud[i][1] * hi[sidx(1, j)] + Aud[i][2] * hi[sidx(2, j)];
    const T AA = A[0] * Au[0] + A[3] * Au[3] + A[5] * Au[5] + 2.0 * (A[1] * Au[1] + A[2] * Au[2] + A[4] * Au[4]);
    T KK[6];  // K_ik K^k_j
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            KK[sidx(i, j)] = Kp[sidx(i, 0)] * Kud(0, j) + Kp[sidx(i, 1)] * Kud(1, j) + Kp[sidx(i, 2)] * Kud(2, j);
    T dKp[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T dK3 = dK[k] * (1.0 / 3.0);
#pragma unroll
        for (int m = 0; m < 6; ++m)
            dKp[k][m] = fma(-Kp[m], dchi[k], fma(dh[k][m], K3, fma(h[m], dK3, D1(F_A + m, k)))) * ichi;
    }
    T LbK[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const int m = sidx(i, j);
            T s = LOP ? fma(-Kp[m], adv[F_CHI], fma(adv[F_H + m], K3, fma(h[m], adv[F_K] * (1.0 / 3.0), adv[F_A + m]))) * ichi
                      : bx * dKp[0][m] + by * dKp[1][m] + bz * dKp[2][m];
#pragma unroll
            for (int k = 0; k < 3; ++k) s = fma(Kp[sidx(k, j)], db[i][k], fma(Kp[sidx(i, k)], db[j][k], s));
            LbK[sidx(i, j)] = s;
        }
    // Codazzi block through its dual: bb[k][m] = B_{k,(m+1),(m+2)} = D_a K_kb - D_b K_ka with
    // (a, b) = (m+1, m+2). The Gp^l_ab K_kl parts of the two covariant derivatives cancel (the
    // connection is symmetric), leaving d_a K_kb - d_b K_ka - Gp^l_ak K_lb + Gp^l_bk K_la.
    T bb[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int a = (m + 1) % 3, b = (m + 2) % 3;
            T s = dKp[a][sidx(k, b)] - dKp[b][sidx(k, a)];
#pragma unroll
            for (int l = 0; l < 3; ++l)
                s = fma(-Gp[l][sidx(a, k)], Kp[sidx(l, b)], fma(Gp[l][sidx(b, k)], Kp[sidx(l, a)], s));
            bb[k][m] = s;
        }
#define BC(k, i, j) (cyclic(i, j) ? bb[k][third(i, j)] : -bb[k][third(i, j)])
    T Bv[3];  // B_j = gamma^ab B_abj
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T s = 0.0;
        bool first = true;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if (b != j) {
                    s = first ? gu[sidx(a, b)] * BC(a, b, j) : fma(gu[sidx(a, b)], BC(a, b, j), s);
                    first = false;
                }
        Bv[j] = s;
    }

    // ---- Gauss block S_ij and its Einstein tensor G_S
    GRF_SECTION(9);
    T S[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) S[m] = fma(trK, Kp[m], Ric[m] - KK[m]);
    const T Ss = sdotw(S, gw);
    T GS[6], GSuw[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) GS[m] = fma(-0.5 * Ss, gd[m], S[m]);
    {
        T M1[3][3];  // gamma^ia G_S ab
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                M1[i][b] = gu[sidx(i, 0)] * GS[sidx(0, b)] + gu[sidx(i, 1)] * GS[sidx(1, b)] + gu[sidx(i, 2)] * GS[sidx(2, b)];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                const T x = M1[i][0] * gu[sidx(0, j)] + M1[i][1] * gu[sidx(1, j)] + M1[i][2] * gu[sidx(2, j)];
                GSuw[sidx(i, j)] = (i == j) ? x : 2.0 * x;  // G_S^ij, off-diagonals doubled
            }
    }

    // ---- scalar: nabla nabla phi blocks, Phi = nabla nabla beta(phi)
    GRF_SECTION(10);
    T b1, b2;
    // beta' and beta'' of the coupling: lam phi, lam phi^2 / 2, or lam / (2 kappa) (1 - e^{-kappa phi^2})
    // (beta' = lam phi e^{-kappa phi^2}, beta'' = lam e^{-kappa phi^2} (1 - 2 kappa phi^2))
    if (c.beta_kind == 1) {
        b1 = c.lam * phi; b2 = c.lam;
    } else if (COUP && c.beta_kind == 2) {
        const T kp2 = c.beta_kappa * (phi * phi);
        const T e = exp(-kp2);
        b1 = c.lam * (phi * e);
        b2 = c.lam * (e * fma(-2.0, kp2, 1.0));
    } else {
        b1 = c.lam; b2 = 0.0;
    }
    T dphiu[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dphiu[i] = gu[sidx(i, 0)] * dphi[0] + gu[sidx(i, 1)] * dphi[1] + gu[sidx(i, 2)] * dphi[2];
    const T dphi2 = dphi[0] * dphiu[0] + dphi[1] * dphiu[1] + dphi[2] * dphiu[2];
    const T X = 0.5 * (Pi * Pi - dphi2);
    const T g2 = c.g2;
    T Hij[6], Hn[3];
#pragma unroll
    for (int m = 0; m < 6; ++m) Hij[m] = fma(Kp[m], Pi, DDp[m]);
#pragma unroll
    for (int i = 0; i < 3; ++i) Hn[i] = dPi[i] + Kud(0, i) * dphi[0] + Kud(1, i) * dphi[1] + Kud(2, i) * dphi[2];
    T Phd[6], Phn[3];
    const T b2Pi = b2 * Pi;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Phn[i] = fma(b1, Hn[i], b2Pi * dphi[i]);
        const T b2d = b2 * dphi[i];
#pragma unroll
        for (int j = i; j < 3; ++j) Phd[sidx(i, j)] = fma(b1, Hij[sidx(i, j)], b2d * dphi[j]);
    }
    T Phm[3][3], Phuw[6], Phnu[3];  // Phi_i^k, Phi^ij (off-diagonals doubled), Phi_n^k
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            Phm[i][k] = Phd[sidx(i, 0)] * gu[sidx(0, k)] + Phd[sidx(i, 1)] * gu[sidx(1, k)] + Phd[sidx(i, 2)] * gu[sidx(2, k)];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const T x = gu[sidx(i, 0)] * Phm[0][j] + gu[sidx(i, 1)] * Phm[1][j] + gu[sidx(i, 2)] * Phm[2][j];
            Phuw[sidx(i, j)] = (i == j) ? x : 2.0 * x;
        }
        Phnu[i] = gu[sidx(i, 0)] * Phn[0] + gu[sidx(i, 1)] * Phn[1] + gu[sidx(i, 2)] * Phn[2];
    }
    const T trP = Phm[0][0] + Phm[1][1] + Phm[2][2];

    // ---- sources that do not depend on the unknowns
    GRF_SECTION(11);
    const T fX = fma(2.0 * g2, X, 1.0);
    const T XX = fma(g2 * X, X, X);  // X + g2 X^2
    // decoupled mode: the scalar's stress-energy is left out of the metric equations (rho, S_i,
    // S_ij and their coupling to d_t K_ij); the scalar equation below is unchanged
    const bool dec = (DEC < 0) ? (c.decoupled != 0) : (DEC == 1);
    T rho8 = dec ? T(0.0) : fma(0.5 * fX, Pi * Pi, fma(-4.0, sdotw(GS, Phuw), -0.5 * XX));
    T S8[3];
    const T BPn = Bv[0] * Phnu[0] + Bv[1] * Phnu[1] + Bv[2] * Phnu[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T s = GS[sidx(i, 0)] * Phnu[0] + GS[sidx(i, 1)] * Phnu[1] + GS[sidx(i, 2)] * Phnu[2];
        s = fma(trP, Bv[i], s - (Phm[i][0] * Bv[0] + Phm[i][1] * Bv[1] + Phm[i][2] * Bv[2]));
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l)
                if (l != i) {
                    const T pkl = (k == l) ? Phuw[sidx(k, l)] : 0.5 * Phuw[sidx(k, l)];
                    s = fma(BC(k, i, l), pkl, s);
                }
        S8[i] = dec ? T(0.0) : fma(-0.5 * fX * Pi, dphi[i], 4.0 * s);
    }
    // cubic term: the n-n and n-i parts of its stress tensor (no unknown in them)
    const bool cub = COUP && c.g3 != 0.0;
    T trH3 = 0.0, Hnd3 = 0.0, Hdd3 = 0.0, Hdv3[3];
    if (cub) {
        trH3 = sdotw(Hij, gw);
        Hnd3 = dphiu[0] * Hn[0] + dphiu[1] * Hn[1] + dphiu[2] * Hn[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            Hdv3[i] = Hij[sidx(i, 0)] * dphiu[0] + Hij[sidx(i, 1)] * dphiu[1] + Hij[sidx(i, 2)] * dphiu[2];
        Hdd3 = dphiu[0] * Hdv3[0] + dphiu[1] * Hdv3[1] + dphiu[2] * Hdv3[2];
        if (!dec) {
            const double g3h = 0.5 * c.g3;
            rho8 = fma(g3h, fma(Pi * Pi, trH3, -Hdd3), rho8);
            const T a3 = fma(Pi, trH3, -Hnd3);
#pragma unroll
            for (int i = 0; i < 3; ++i) S8[i] = fma(-g3h, fma(a3, dphi[i], Pi * fma(Pi, Hn[i], -Hdv3[i])), S8[i]);
        }
    }
    T S1[6], Y[6];
    const T fXh = 0.5 * fX, XXh = 0.5 * XX;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            S1[sidx(i, j)] = dec ? T(0.0) : fma(fXh * dphi[i], dphi[j], XXh * gd[sidx(i, j)]);
            T y = fma(Bv[j], Phn[i], Bv[i] * Phn[j]);
            y = fma(-2.0 * BPn, gd[sidx(i, j)], y);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                if (l != j) y = fma(BC(i, j, l), Phnu[l], y);
                if (l != i) y = fma(BC(j, i, l), Phnu[l], y);
            }
            Y[sidx(i, j)] = dec ? T(0.0) : y;
        }

    // C0 = C at d_t K_ij = 0
    GRF_SECTION(12);
    T C0[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) C0[m] = fma(DDa[m] - LbK[m], ial, KK[m]);
    const T bdPi = LOP ? adv[F_PI] : bx * dPi[0] + by * dPi[1] + bz * dPi[2];
    const T dadp = dal[0] * dphiu[0] + dal[1] * dphiu[1] + dal[2] * dphiu[2];
    const T Phnn0 = fma(b1 * ial, -(bdPi + dadp), b2Pi * Pi);

    // L_GB at d_t K_ij = 0: 8 G_S^ij C_ij - 4 B_kij B^kij + 8 B_i B^i, with
    // B_kij B^kij = 2 chi^3 / det(h) h^kk' h_mm' bb[k][m] bb[k'][m']
    GRF_SECTION(13);
    T L0;
    {
        T N[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q)
                N[k][q] = h[sidx(0, q)] * bb[k][0] + h[sidx(1, q)] * bb[k][1] + h[sidx(2, q)] * bb[k][2];
        T tt[6];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int kk = k; kk < 3; ++kk) tt[sidx(k, kk)] = N[k][0] * bb[kk][0] + N[k][1] * bb[kk][1] + N[k][2] * bb[kk][2];
        const T BB = (2.0 * chi * chi * chi * ideth) * sdotw(tt, hw);
        const T Bvu0 = gu[0] * Bv[0] + gu[1] * Bv[1] + gu[2] * Bv[2];
        const T Bvu1 = gu[1] * Bv[0] + gu[3] * Bv[1] + gu[4] * Bv[2];
        const T Bvu2 = gu[2] * Bv[0] + gu[4] * Bv[1] + gu[5] * Bv[2];
        const T BvBv = Bv[0] * Bvu0 + Bv[1] * Bvu1 + Bv[2] * Bvu2;
        L0 = fma(8.0, sdotw(C0, GSuw), fma(-4.0, BB, 8.0 * BvBv));
    }

    // ---- CCZ4 right-hand sides without S_ij (rho and S_i included)
    GRF_SECTION(14);
    rhs[F_CHI] = fma((2.0 / 3.0) * chi, al * K - divb, ADV(F_CHI));
    const T divb23 = (2.0 / 3.0) * divb;
    const T al2 = 2.0 * al;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            T x = fma(-h[sidx(i, j)], divb23, fma(-al2, A[sidx(i, j)], ADV(F_H + sidx(i, j))));
#pragma unroll
            for (int k = 0; k < 3; ++k) x = fma(h[sidx(i, k)], db[j][k], fma(h[sidx(j, k)], db[i][k], x));
            rhs[F_H + sidx(i, j)] = x;
        }
    const T K2Th = K - 2.0 * Th;
    // b(x) of the modified gauge enters through the auxiliary metric g^ab - b n^a n^b of the Z terms
    // of the covariant equation; its 3+1 projection is carried by Hb = H - 16 pi rho
    // - 2 kappa1 (2 + kappa2) Theta (plain H = R - A_ij A^ij + 2/3 K^2) in d_t K and d_t Theta, and
    // by the momentum-constraint combination in d_t Gamma-hat below.
    const T Hb = fma(-2.0 * c.kappa1 * (2.0 + c.kappa2), Th, Rs - AA + (2.0 / 3.0) * K * K - 2.0 * rho8);
    const T Kdot0 = ADV(F_K) + al * fma(K, K2Th, RZs) - (3.0 * c.kappa1 * (1.0 + c.kappa2)) * al * Th - lapal
                    - 1.5 * al * rho8 - (c.bK * al) * Hb;
    T Adot0[6];
    {
        T Xa[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) Xa[m] = fma(al, RZ[m], -DDa[m]);
        const T trX3 = sdotw(Xa, hw) * (1.0 / 3.0);
        const T alK2Th = al * K2Th;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                T x = fma(chi, fma(-h[sidx(i, j)], trX3, Xa[sidx(i, j)]), ADV(F_A + sidx(i, j)));
                x = fma(alK2Th - divb23, A[sidx(i, j)], x);
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    x = fma(A[sidx(i, k)], fma(-al2, Aud[k][j], db[j][k]), fma(A[sidx(j, k)], db[i][k], x));
                Adot0[sidx(i, j)] = x;
            }
    }
    // d_t Theta = beta.dTheta + alpha (D_i Z^i - Theta K) - Z^i d_i alpha + alpha Hb / (2 (1 + b)),
    // with 2 D_i Z^i = RZs - Rs
    rhs[F_TH] = ADV(F_TH) + al * fma(0.5, RZs - Rs, -Th * K) - (Zu[0] * dal[0] + Zu[1] * dal[1] + Zu[2] * dal[2])
                + (c.bTh * al) * Hb;
    {
        T hZ[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) hZ[i] = hi[sidx(i, 0)] * Zl[0] + hi[sidx(i, 1)] * Zl[1] + hi[sidx(i, 2)] * Zl[2];
        T ddbk[3];  // sum_k d_j d_k beta^k
#pragma unroll
        for (int j = 0; j < 3; ++j) ddbk[j] = D2(F_SHIFT, sidx(j, 0)) + D2(F_SHIFT + 1, sidx(j, 1)) + D2(F_SHIFT + 2, sidx(j, 2));
        T Auw[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) Auw[m] = (m == 1 || m == 2 || m == 4) ? 2.0 * Au[m] : Au[m];
        T tk[3];  // 2 (al d_k Theta - Theta d_k al - 2/3 al K Z_k)
        const T alK23 = (2.0 / 3.0) * al * K;
#pragma unroll
        for (int k = 0; k < 3; ++k) tk[k] = 2.0 * fma(al, dTh[k], fma(-Th, dal[k], -alK23 * Zl[k]));
        const T k3div = (4.0 / 3.0) * c.kappa3 * divb;
        const T ak1 = 2.0 * al * c.kappa1;
        // b(x) part of d_t Z_j: -(b/(1+b)) alpha wb_j, wb_j = M_j + d_j Theta - K^k_j Z_k - kappa1 Z_j with
        // the momentum constraint M_j = B_j - 8 pi S_j; Gamma-hat^i carries 2 h^ij Z_j, so d_t Gamma-hat^i
        // gains -(2b/(1+b)) alpha h^ij wb_j (2b/(1+b) = 2 - 4 bTh)
        T wb[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T s = (Bv[j] - S8[j]) + dTh[j];
            s = fma(-c.kappa1, Zl[j], s);
#pragma unroll
            for (int k = 0; k < 3; ++k) s = fma(-Kud(k, j), Zl[k], s);
            wb[j] = s;
        }
        const T abG = (2.0 - 4.0 * c.bTh) * al;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T t1 = sdotw(G2[i], Auw);
            const T t2 = Au[sidx(i, 0)] * dchi[0] + Au[sidx(i, 1)] * dchi[1] + Au[sidx(i, 2)] * dchi[2];
            const T t3 = hi[sidx(i, 0)] * dK[0] + hi[sidx(i, 1)] * dK[1] + hi[sidx(i, 2)] * dK[2];
            const T t4 = Au[sidx(i, 0)] * dal[0] + Au[sidx(i, 1)] * dal[1] + Au[sidx(i, 2)] * dal[2];
            T t5 = 0.0;
#pragma unroll
            for (int q = 0; q < 6; ++q) t5 = (q == 0) ? hw[0] * D2(F_SHIFT + i, 0) : fma(hw[q], D2(F_SHIFT + i, q), t5);
            const T t6 = hZ[0] * db[0][i] + hZ[1] * db[1][i] + hZ[2] * db[2][i];
            T x = ADV(F_GAM + i) + al2 * (t1 - (1.5 * ichi) * t2 - (2.0 / 3.0) * t3) - 2.0 * t4 + t5;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                x = fma(hi[sidx(k, i)], fma(1.0 / 3.0, ddbk[k], tk[k]), x);
                x = fma(-Gtc[k], db[k][i], x);
            }
            x = fma((2.0 / 3.0) * divb, Gtc[i], x);
            x = fma(k3div - ak1, hZ[i], x);
            x = fma(-2.0 * c.kappa3, t6, x);
            x = fma(-al2, hi[sidx(i, 0)] * S8[0] + hi[sidx(i, 1)] * S8[1] + hi[sidx(i, 2)] * S8[2], x);
            x = fma(-abG, hi[sidx(i, 0)] * wb[0] + hi[sidx(i, 1)] * wb[1] + hi[sidx(i, 2)] * wb[2], x);
            rhs[F_GAM + i] = x;
            rhs[F_B + i] = fma(-c.eta, v[F_B + i], x);
            rhs[F_SHIFT + i] = fma(c.shift_F * c.inv_1pa, v[F_B + i],
                                   -(c.a_1pa * al * chi) * (hi[sidx(i, 0)] * dal[0] + hi[sidx(i, 1)] * dal[1] + hi[sidx(i, 2)] * dal[2]));
        }
    }
    rhs[F_LAPSE] = fma(-2.0 * c.inv_1pa * al, K2Th, ADV(F_LAPSE));
    rhs[F_PHI] = fma(al, Pi, ADV(F_PHI));

    // ---- coupled system for v = (d_t K_ij, d_t Pi):
    //   u - 4 L(Q(u)) - 4 b1 L(G_S) w = r,   w - (8 b1 / D) G_S^ij u_ij = r_w,   L(X) = X - gamma tr(X)/2
    GRF_SECTION(15);
    T Msys[7][8];
    T S3[6], PPc[6], HnnSol0 = 0.0;  // cubic term: 8 pi S3_ij without d_t Pi, Pi^2 gamma^ij - d^i phi d^j phi
    T QC0[6];
    q_of(C0, gd, gw, Phd, Phuw, Phm, trP, QC0);
    {
        const T chid = rhs[F_CHI];
        const T trS1h = 0.5 * sdotw(S1, gw), trYh = 0.5 * sdotw(Y, gw), trQh = 0.5 * sdotw(QC0, gw);
        const T Ss4 = 0.25 * Ss;
        const T al4 = 4.0 * al;
        const T four_b1 = 4.0 * b1;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const T LGS = fma(-Ss4, gd[m], S[m]);
            const T U0 = fma(-Kp[m], chid, fma(rhs[F_H + m], K3, fma(h[m], Kdot0 * (1.0 / 3.0), Adot0[m]))) * ichi;
            const T lin = dec ? T(0.0) : fma(LGS, Phnn0, (Y[m] + QC0[m]) - gd[m] * (trYh + trQh));
            Msys[m][7] = fma(al4, lin, fma(-al, fma(-trS1h, gd[m], S1[m]), U0));
            Msys[m][6] = dec ? T(0.0) : -four_b1 * LGS;
        }
        // 6x6 block, column (a,b): -4 L(Q(E_ab)) with E_ab the unit symmetric matrix
        //   = -2 gamma_ij w_ab (Phi^ab - gamma^ab tr Phi) - 4 w_ab gamma^ab Phi_ij + 4 P_ij,ab - 4 tr(Phi) [ij == ab]
        //   P_ij,ab = Phi_i^k E_kj + Phi_j^k E_ik
        const T one4P = fma(-4.0, trP, 1.0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) {
                const int col = sidx(a, b);
                const T sab = Phuw[col] - gw[col] * trP;   // w_ab (Phi^ab - gamma^ab trP)
                const T tab = -4.0 * gw[col];               // -4 w_ab gamma^ab
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = i; j < 3; ++j) {
                        const int row = sidx(i, j);
                        T p = 0.0;
                        bool any = false;
                        // Phi_i^k E_kj: E_kj = [k==a][j==b] + [k==b][j==a] (single term when a == b)
                        if (j == b) { p = any ? p + Phm[i][a] : Phm[i][a]; any = true; }
                        if (a != b && j == a) { p = any ? p + Phm[i][b] : Phm[i][b]; any = true; }
                        if (i == b) { p = any ? p + Phm[j][a] : Phm[j][a]; any = true; }
                        if (a != b && i == a) { p = any ? p + Phm[j][b] : Phm[j][b]; any = true; }
                        T e = fma(-2.0 * gd[row], sab, tab * Phd[row]);
                        if (any) e = fma(4.0, p, e);
                        if (row == col) e = e + one4P;
                        Msys[row][col] = dec ? T(row == col ? 1.0 : 0.0) : e;
                    }
            }
        T Dphi = fma(2.0 * g2, Pi * Pi, fX);
        T E3 = 0.0;  // the cubic term's share of the scalar equation without H_nn and d_t K_ij
        if (cub) {
            Dphi = fma(2.0 * c.g3, trH3, Dphi);
            const T Hnn0 = -(bdPi + dadp) * ial;
            T Hm[3][3], ppw[6], PPuw[6];  // H_i^k, d^i phi d^j phi and Pi^2 gamma^ij - d^i phi d^j phi (weighted)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    Hm[i][k] = Hij[sidx(i, 0)] * gu[sidx(0, k)] + Hij[sidx(i, 1)] * gu[sidx(1, k)] + Hij[sidx(i, 2)] * gu[sidx(2, k)];
            T HH = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) HH = fma(Hm[i][k], Hm[k][i], HH);
            T HnHn = 0.0, BdP = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T hnu = gu[sidx(i, 0)] * Hn[0] + gu[sidx(i, 1)] * Hn[1] + gu[sidx(i, 2)] * Hn[2];
                HnHn = fma(Hn[i], hnu, HnHn);
                BdP = fma(Bv[i], dphiu[i], BdP);
            }
            const T Pi2 = Pi * Pi;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = i; j < 3; ++j) {
                    const T pp = dphiu[i] * dphiu[j];
                    ppw[sidx(i, j)] = (i == j) ? pp : 2.0 * pp;
                    PPuw[sidx(i, j)] = fma(Pi2, gw[sidx(i, j)], -ppw[sidx(i, j)]);
                }
            T e3 = fma(trH3, trH3, fma(2.0, HnHn, -HH));
            e3 = fma(-2.0 * Pi, BdP, e3);
            e3 = e3 - sdotw(S, ppw) - sdotw(C0, PPuw);
            E3 = c.g3 * e3;
            if (!dec) {
                // 8 pi S3_ij without its d_t Pi part, and that part's coefficient in the metric rows:
                // S3_ij = S3_0 + g3 w / (2 alpha) (Pi^2 gamma_ij - d_i phi d_j phi)
                const T pcoef = 0.5 * (trH3 - Hnn0);                               // of d_i phi d_j phi
                const T gcoef = fma(0.5 * Hnn0, Pi2, fma(0.5, Hdd3, -Pi * Hnd3));  // of gamma_ij
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = i; j < 3; ++j) {
                        T x = fma(gcoef, gd[sidx(i, j)], pcoef * (dphi[i] * dphi[j]));
                        x = fma(0.5 * Pi, fma(Hn[i], dphi[j], Hn[j] * dphi[i]), x);
                        x = fma(-0.5, fma(Hdv3[i], dphi[j], Hdv3[j] * dphi[i]), x);
                        S3[sidx(i, j)] = c.g3 * x;
                    }
                const T trS3h = 0.5 * sdotw(S3, gw);
                const T wc = 0.5 * (dphi2 - Pi2);
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const int i = (m < 3) ? 0 : (m < 5 ? 1 : 2);
                    const int j = (m < 3) ? m : (m < 5 ? m - 2 : 2);
                    Msys[m][7] = fma(-al, fma(-trS3h, gd[m], S3[m]), Msys[m][7]);
                    Msys[m][6] = fma(0.5 * c.g3, fma(wc, gd[m], -dphi[i] * dphi[j]), Msys[m][6]);
                }
            }
#pragma unroll
            for (int col = 0; col < 6; ++col) PPc[col] = PPuw[col];
            HnnSol0 = Hnn0;
        }
        const T iD = 1.0 / Dphi;
        const T c8 = -8.0 * b1 * iD;
#pragma unroll
        for (int col = 0; col < 6; ++col) Msys[6][col] = c8 * GSuw[col];
        if (cub) {
#pragma unroll
            for (int col = 0; col < 6; ++col) Msys[6][col] = fma(c.g3 * iD, PPc[col], Msys[6][col]);
        }
        Msys[6][6] = 1.0;
        const T trH = sdotw(Hij, gw);
        const T Hnd = dphiu[0] * Hn[0] + dphiu[1] * Hn[1] + dphiu[2] * Hn[2];
        T Hdd = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T t = Hij[sidx(i, 0)] * dphiu[0] + Hij[sidx(i, 1)] * dphiu[1] + Hij[sidx(i, 2)] * dphiu[2];
            Hdd = (i == 0) ? dphiu[0] * t : fma(dphiu[i], t, Hdd);
        }
        T src = fma(fX, trH, fma(4.0 * g2 * Pi, Hnd, fma(-2.0 * g2, Hdd, b1 * L0)));
        if (cub) src = src + E3;
        Msys[6][7] = fma(al * iD, src, bdPi + dadp);
        if constexpr (std::is_same<T, double>::value) {
            if (extra && extra->want_hyp) {
                extra->hyp[0] = det7(Msys, &extra->hyp[3]);
                extra->hyp[1] = fX * fX * fX * fma(6.0 * g2, X, 1.0);  // g3 = 0; the cubic case below
                extra->hyp[2] = Dphi;
            }
        }
    }
    GRF_SECTION(16);
    ok = solve7(Msys);
    T u[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) u[m] = Msys[m][7];
    const T w = Msys[6][7];
    if constexpr (std::is_same<T, double>::value) {
        if (cub && extra && extra->want_hyp) {
            // g_eff in the basis (n, e_i) at the solution: g_eff^nn = -D (stored above),
            // g_eff^ni = 2 g2 Pi d^i phi + 2 g3 H_n^i, g_eff^ij = (1 + 2 g2 X) gamma^ij
            // - 2 g2 d^i phi d^j phi + 2 g3 (box(phi) gamma^ij - H^ij); by the Schur complement on the
            // n-n entry, det g_eff / det g = D det(g_eff^ij + g_eff^ni g_eff^nj / D) det(gamma_ij)
            const double D = extra->hyp[2];
            const double box = trH3 - fma(w, ial, HnnSol0);
            double e0[3], Hu[3][3], Sc[6];
            for (int i = 0; i < 3; ++i) {
                const double hnu = gu[sidx(i, 0)] * Hn[0] + gu[sidx(i, 1)] * Hn[1] + gu[sidx(i, 2)] * Hn[2];
                e0[i] = 2.0 * (g2 * Pi * dphiu[i] + c.g3 * hnu);
                for (int k = 0; k < 3; ++k)
                    Hu[i][k] = Hij[sidx(i, 0)] * gu[sidx(0, k)] + Hij[sidx(i, 1)] * gu[sidx(1, k)] + Hij[sidx(i, 2)] * gu[sidx(2, k)];
            }
            for (int i = 0; i < 3; ++i)
                for (int j = i; j < 3; ++j) {
                    const double huij = gu[sidx(i, 0)] * Hu[0][j] + gu[sidx(i, 1)] * Hu[1][j] + gu[sidx(i, 2)] * Hu[2][j];
                    const double eij = fX * gu[sidx(i, j)] - 2.0 * g2 * dphiu[i] * dphiu[j]
                                       + 2.0 * c.g3 * (box * gu[sidx(i, j)] - huij);
                    Sc[sidx(i, j)] = eij + e0[i] * e0[j] / D;
                }
            extra->hyp[1] = D * sym3_det(Sc) * sym3_det(gd);
        }
    }

    // ---- full S_ij at the solution and the final K, A_ij, Pi right-hand sides
    GRF_SECTION(17);
    {
        T Qu[6];
        q_of(u, gd, gw, Phd, Phuw, Phm, trP, Qu);
        const T Phnn = fma(b1 * ial, w, Phnn0);
        T S8ij[6];
#pragma unroll
        for (int m = 0; m < 6; ++m)
            S8ij[m] = dec ? T(0.0) : fma(-4.0, fma(GS[m], Phnn, Y[m] + fma(Qu[m], ial, QC0[m])), S1[m]);
        if (cub && !dec) {
            const T gw2 = (0.5 * c.g3) * (w * ial);
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int i = (m < 3) ? 0 : (m < 5 ? 1 : 2);
                const int j = (m < 3) ? m : (m < 5 ? m - 2 : 2);
                S8ij[m] = S8ij[m] + fma(gw2, fma(Pi * Pi, gd[m], -dphi[i] * dphi[j]), S3[m]);
            }
        }
        const T Ss8 = sdotw(S8ij, gw);
        rhs[F_K] = fma(0.5 * al, Ss8, Kdot0);
        const T trh3 = sdotw(S8ij, hw) * (1.0 / 3.0);
        const T alchi = al * chi;
#pragma unroll
        for (int m = 0; m < 6; ++m) rhs[F_A + m] = fma(-alchi, fma(-h[m], trh3, S8ij[m]), Adot0[m]);
        rhs[F_PI] = w;
    }
    if (extra) {
        extra->ham = fma(-2.0, rho8, Ss);
#pragma unroll
        for (int i = 0; i < 3; ++i) extra->mom[i] = Bv[i] - S8[i];
        const T X2 = X * X;
        extra->rho8[0] = 0.5 * (Pi * Pi - X);
        extra->rho8[1] = g2 * fma(X, Pi * Pi, -0.5 * X2);
        extra->rho8[2] = -4.0 * sdotw(GS, Phuw);
        if constexpr (std::is_same<T, double>::value) {
            if (extra->want_psi4) {
                // Psi_4 = R(n, mbar, n, mbar) with n = (u - e_r)/sqrt2, m = (e_theta + i e_phi)/sqrt2: the
                // Ricci and scalar terms of the Weyl tensor vanish on a null tetrad with g(n, mbar) = 0,
                // so with the Riemann blocks (Ricci equation, Codazzi, Gauss)
                //   Psi_4 = 1/2 R_ninj mbar^i mbar^j - R_nikj mbar^i e_r^k mbar^j + 1/2 R_kilj e_r^k mbar^i e_r^l mbar^j,
                //   R_ninj = (d_t K_ij - L_beta K_ij + D_i D_j alpha)/alpha + K_ik K^k_j,
                //   R_nikj = D_k K_ij - D_j K_ik,  R_kilj e_r e_r = R_ij + K_rr K_ij - K_ri K_rj (3D: Ricci form).
                const double x = extra->xyz[0], y = extra->xyz[1], z = extra->xyz[2];
                double pr = 0.0, pim = 0.0;
                if (x * x + y * y != 0.0) {
                    double e[3][3] = {{x, y, z}, {x * z, y * z, -(x * x + y * y)}, {-y, x, 0.0}};
                    auto dotg = [&](const double* a, const double* b) {
                        double d = 0.0;
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int j = 0; j < 3; ++j) d = fma(gd[sidx(i, j)] * a[i], b[j], d);
                        return d;
                    };
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
#pragma unroll
                        for (int b = 0; b < a; ++b) {
                            const double d = dotg(e[a], e[b]);
#pragma unroll
                            for (int i = 0; i < 3; ++i) e[a][i] -= d * e[b][i];
                        }
                        const double inv = 1.0 / sqrt(dotg(e[a], e[a]));
#pragma unroll
                        for (int i = 0; i < 3; ++i) e[a][i] *= inv;
                    }
                    // symmetric forms on (e_theta, e_phi) give Q(mbar, mbar) = (Q_tt - Q_pp - 2i Q_tp)/2
                    auto form = [&](const double* S6, const double* a, const double* b) {
                        double q = 0.0;
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int j = 0; j < 3; ++j) q = fma(S6[sidx(i, j)] * a[i], b[j], q);
                        return q;
                    };
                    double Rn[6];
#pragma unroll
                    for (int m = 0; m < 6; ++m) Rn[m] = fma(u[m] - LbK[m] + DDa[m], ial, KK[m]);
                    const double E1r = 0.5 * (form(Rn, e[1], e[1]) - form(Rn, e[2], e[2]));
                    const double E1i = -form(Rn, e[1], e[2]);
                    const double Krr = form(Kp, e[0], e[0]), Krt = form(Kp, e[0], e[1]), Krp = form(Kp, e[0], e[2]);
                    const double E3r = 0.5 * (form(Ric, e[1], e[1]) - form(Ric, e[2], e[2]))
                                       + Krr * 0.5 * (form(Kp, e[1], e[1]) - form(Kp, e[2], e[2]))
                                       - 0.5 * (Krt * Krt - Krp * Krp);
                    const double E3i = -form(Ric, e[1], e[2]) - Krr * form(Kp, e[1], e[2]) + Krt * Krp;
                    // E2 = sum_i mbar^i W_i, W_i = sum_{k != j} R_nikj e_r^k mbar^j, mbar = (e_t - i e_p)/sqrt2
                    double E2r = 0.0, E2i = 0.0;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        double wr = 0.0, wi = 0.0;
#pragma unroll
                        for (int k = 0; k < 3; ++k)
#pragma unroll
                            for (int j = 0; j < 3; ++j)
                                if (k != j) {
                                    const double Rnikj = BC(i, k, j);
                                    wr = fma(Rnikj * e[0][k], e[1][j], wr);
                                    wi = fma(-Rnikj * e[0][k], e[2][j], wi);
                                }
                        // mbar^i W_i with both factors carrying 1/sqrt2
                        E2r += 0.5 * (e[1][i] * wr + e[2][i] * wi);
                        E2i += 0.5 * (e[1][i] * wi - e[2][i] * wr);
                    }
                    pr = 0.5 * E1r - E2r + 0.5 * E3r;
                    pim = 0.5 * E1i - E2i + 0.5 * E3i;
                }
                extra->psi4[0] = pr;
                extra->psi4[1] = pim;
            }
        }
    }
#undef BC
#undef D1
#undef D2
#undef ADV
}

}  // namespace grf
