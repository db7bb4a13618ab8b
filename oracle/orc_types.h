// C types of the CPU oracle's interface (test infrastructure; see grf_oracle.cpp).
#pragma once

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
    double g3;              // cubic Horndeski coupling: the action's g3 X box(phi) term
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
