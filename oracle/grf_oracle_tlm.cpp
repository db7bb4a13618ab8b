// Tangent-linear model (TLM) of the CPU oracle's evolution: the derivative of the evolved state
// and of the sphere-averaged scalar signal along a direction (delta state_0, delta lambda,
// delta g2), by two independent forward-mode constructions of the same core (orc_core.inc):
//   * dual numbers x + eps x' with eps^2 = 0, propagated exactly through every arithmetic
//     operation (the tangent-linear model proper);
//   * the complex step: the core run on complex numbers x + i h x' with h = 1e-30; for an
//     analytic function, Im f(x + i h x')/h = f'(x) x' + O(h^2), with no subtraction, so the
//     result is exact to rounding (Squire and Trapp, SIAM Review 40 (1998) 110).
// Non-analytic steps act on the value part in both: pivot choices by magnitude, and the chi /
// lapse floors (the derivative of the branch taken).
//
// TEST INFRASTRUCTURE ONLY (see grf_oracle.cpp): used by tests/ to pin the tangent-linear model
// (dual against complex step) and, through it, the GPU adjoint by a dot-product test.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "orc_types.h"

// ---------------------------------------------------------------------------------------------
// Dual numbers over T (double, or long double in the linear solve).
// ---------------------------------------------------------------------------------------------
template <typename T>
struct Dual {
    T v, d;
    Dual() = default;
    Dual(double x) : v(x), d(0) {}  // NOLINT: constants convert implicitly
    Dual(T x, T y) : v(x), d(y) {}
    Dual& operator+=(const Dual& b) { v += b.v; d += b.d; return *this; }
    Dual& operator-=(const Dual& b) { v -= b.v; d -= b.d; return *this; }
    Dual& operator*=(const Dual& b) { d = d * b.v + v * b.d; v *= b.v; return *this; }
};
template <typename T> Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> Dual<T> operator-(const Dual<T>& a) { return {-a.v, -a.d}; }
template <typename T> Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename T> Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
    const T q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
#define ORC_DUAL_MIXED(OP)                                                                              \
    template <typename T> Dual<T> operator OP(const Dual<T>& a, double b) { return a OP Dual<T>(b); } \
    template <typename T> Dual<T> operator OP(double a, const Dual<T>& b) { return Dual<T>(a) OP b; }
ORC_DUAL_MIXED(+)
ORC_DUAL_MIXED(-)
ORC_DUAL_MIXED(*)
ORC_DUAL_MIXED(/)
#undef ORC_DUAL_MIXED
template <typename T> Dual<T> exp(const Dual<T>& a) {
    const T e = std::exp(a.v);
    return {e, e * a.d};
}

namespace orc_dual {

typedef Dual<double> real;
typedef Dual<long double> real_ld;
inline double vval(const real& x) { return x.v; }
inline double vabs(const real& x) { return std::fabs(x.v); }
inline long double vabsl(const real_ld& x) { return fabsl(x.v); }
inline real vmax(const real& x, double c) { return x.v >= c ? x : real(c); }
inline real_ld to_ld(const real& x) { return real_ld((long double)x.v, (long double)x.d); }
inline real from_ld(const real_ld& x) { return real((double)x.v, (double)x.d); }
#define ORC_PLAIN 0
#include "orc_core.inc"
#undef ORC_PLAIN

}  // namespace orc_dual

namespace orc_cs {

typedef std::complex<double> real;
typedef std::complex<long double> real_ld;
inline double vval(const real& x) { return x.real(); }
inline double vabs(const real& x) { return std::fabs(x.real()); }
inline long double vabsl(const real_ld& x) { return fabsl(x.real()); }
inline real vmax(const real& x, double c) { return x.real() >= c ? x : real(c); }
inline real_ld to_ld(const real& x) { return real_ld(x.real(), x.imag()); }
inline real from_ld(const real_ld& x) { return real((double)x.real(), (double)x.imag()); }
using std::exp;
#define ORC_PLAIN 0
#include "orc_core.inc"
#undef ORC_PLAIN

}  // namespace orc_cs

extern "C" {

// Evolves s (ghosted state, in place) by nsteps RK4 steps and ds (same layout) by the tangent-
// linear model along the direction (ds, dparams[0] = delta lambda, dparams[1] = delta g2).
// mode 0: dual numbers; mode 1: complex step with step h (the tangent is Im(...)/h).
// With a sphere {R, cx, cy, cz}, L[0] receives the signal and L[1] its derivative along the
// direction. Returns the oracle's status (0, -5 singular solve, -4 sphere outside the interior).
int orc_tlm_rk4(const orc_box* b, const orc_params* P, const double* dparams, double* s, double* ds, double dt,
                int nsteps, const double* sphere, double* L, int mode, double h) {
    const long long n = 27LL * (b->nx + 2 * b->ng) * (b->ny + 2 * b->ng) * (b->nz + 2 * b->ng);
    int st;
    if (mode == 0) {
        using orc_dual::real;
        std::vector<real> u(n);
        for (long long q = 0; q < n; ++q) u[q] = real(s[q], ds[q]);
        const orc_dual::Prm pr = orc_dual::prm_of(*P, real(P->lam, dparams[0]), real(P->g2, dparams[1]));
        real sig(0.0);
        orc_dual::Sphere sp = {0, {0, 0, 0}};
        if (sphere) sp = {sphere[0], {sphere[1], sphere[2], sphere[3]}};
        st = orc_dual::rk4_box(*b, pr, u.data(), dt, nsteps, sphere ? &sp : nullptr, &sig);
        for (long long q = 0; q < n; ++q) { s[q] = u[q].v; ds[q] = u[q].d; }
        if (L) { L[0] = sig.v; L[1] = sig.d; }
    } else {
        using orc_cs::real;
        std::vector<real> u(n);
        for (long long q = 0; q < n; ++q) u[q] = real(s[q], h * ds[q]);
        const orc_cs::Prm pr = orc_cs::prm_of(*P, real(P->lam, h * dparams[0]), real(P->g2, h * dparams[1]));
        real sig(0.0);
        orc_cs::Sphere sp = {0, {0, 0, 0}};
        if (sphere) sp = {sphere[0], {sphere[1], sphere[2], sphere[3]}};
        st = orc_cs::rk4_box(*b, pr, u.data(), dt, nsteps, sphere ? &sp : nullptr, &sig);
        for (long long q = 0; q < n; ++q) { s[q] = u[q].real(); ds[q] = u[q].imag() / h; }
        if (L) { L[0] = sig.real(); L[1] = sig.imag() / h; }
    }
    return st;
}

}  // extern "C"
