// Host-side FP64 operation count of the pointwise RHS (libgrf_flops.so).
//
// The same source as the CUDA kernels (grf_point.cuh) is instantiated with a scalar type
// that counts operations instead of only computing them. This gives the algorithmic FLOP
// count per grid point of this formulation (add/sub/mul = 1, fma = 2, div = 1), split by
// section, plus the operations whose operand is a literal 0.0 or 1.0 ("waste": an FP64
// pipe slot the GPU spends although the result is known). A measurement tool, not part of
// the method.
#include <cmath>
#include <cstring>

namespace grfc {
struct Counts {
    long long add, mul, fma, div, cmp, waste;
};
constexpr int kSections = 24;
thread_local Counts g_cnt[kSections];
thread_local int g_sec = 0;

struct CD {
    double v;
    bool k;  // a compile-time constant
    CD() : v(0.0), k(true) {}
    CD(double x) : v(x), k(true) {}
    static CD var(double x) { CD c(x); c.k = false; return c; }
};
inline CD mk(double x, bool k) { CD c(x); c.k = k; return c; }
inline bool is(const CD& a, double x) { return a.k && a.v == x; }
inline Counts& C() { return g_cnt[g_sec]; }

inline CD operator+(const CD& a, const CD& b) {
    if (a.k && b.k) return CD(a.v + b.v);
    if (is(a, 0.0) || is(b, 0.0)) C().waste++; else C().add++;
    return mk(a.v + b.v, false);
}
inline CD operator-(const CD& a, const CD& b) {
    if (a.k && b.k) return CD(a.v - b.v);
    if (is(b, 0.0)) return mk(a.v, false);
    if (is(a, 0.0)) C().waste++; else C().add++;
    return mk(a.v - b.v, false);
}
inline CD operator-(const CD& a) { return mk(-a.v, a.k); }
inline CD operator*(const CD& a, const CD& b) {
    if (a.k && b.k) return CD(a.v * b.v);
    if (is(a, 1.0) || is(b, 1.0) || is(a, -1.0) || is(b, -1.0)) return mk(a.v * b.v, false);
    if (is(a, 0.0) || is(b, 0.0)) C().waste++; else C().mul++;
    return mk(a.v * b.v, false);
}
inline CD operator/(const CD& a, const CD& b) {
    if (a.k && b.k) return CD(a.v / b.v);
    C().div++;
    return mk(a.v / b.v, false);
}
inline CD& operator+=(CD& a, const CD& b) { a = a + b; return a; }
inline CD& operator-=(CD& a, const CD& b) { a = a - b; return a; }
inline CD& operator*=(CD& a, const CD& b) { a = a * b; return a; }
inline bool operator>(const CD& a, const CD& b) { C().cmp++; return a.v > b.v; }
inline bool operator<(const CD& a, const CD& b) { C().cmp++; return a.v < b.v; }
inline CD fma(const CD& a, const CD& b, const CD& c) {
    if (a.k && b.k && c.k) return CD(std::fma(a.v, b.v, c.v));
    if (is(a, 0.0) || is(b, 0.0)) { C().waste++; return mk(c.v, c.k); }
    if (is(c, 0.0)) { return a * b; }
    if (is(a, 1.0) || is(b, 1.0)) { return (is(a, 1.0) ? b : a) + c; }
    C().fma++;
    return mk(std::fma(a.v, b.v, c.v), false);
}
inline CD fabs(const CD& a) { return mk(std::fabs(a.v), a.k); }
inline CD exp(const CD& a) {  // counted as one division-class operation
    if (!a.k) C().div++;
    return mk(std::exp(a.v), a.k);
}
inline CD fmax(const CD& a, const CD& b) {
    if (a.k && b.k) return CD(std::fmax(a.v, b.v));
    C().cmp++;
    return mk(std::fmax(a.v, b.v), false);
}
inline void opaque(CD& x) { x.k = false; }
inline void opaque(double&) {}
}  // namespace grfc

#define GRF_SECTION(id) (grfc::g_sec = (id))
#define GRF_OPAQUE(x) grfc::opaque(x)
#include "grf_point.cuh"
#include "grf.h"

namespace {

// The launch coefficients of grf_params as the library builds them, for the centred-advection
// instance (the counts and the host checks use that one).
grf::Coeffs host_coeffs(const grf_params* p) {
    grf::Coeffs c;
    c.kappa1 = p->kappa1; c.kappa2 = p->kappa2; c.kappa3 = p->kappa3; c.shift_F = p->shift_F; c.eta = p->eta;
    c.lam = p->lambda; c.g2 = p->g2; c.g3 = p->g3;
    c.inv_1pa = 1.0 / (1.0 + p->a0); c.a_1pa = p->a0 / (1.0 + p->a0);
    c.bK = 3.0 * p->b0 / (4.0 * (1.0 + p->b0)); c.bTh = 1.0 / (2.0 * (1.0 + p->b0));
    c.beta_kind = p->beta_kind; c.beta_kappa = p->beta_kappa; c.decoupled = p->decoupled;
    c.advection = 0;
    return c;
}

// Point data in the kernel's slot order (v: 27 values, d1: 24 x 3, d2: 12 x 6).
grf::PointInT<double> host_point(const double* v, const double* d1, const double* d2) {
    grf::PointInT<double> in;
    for (int f = 0; f < grf::NFIELDS; ++f) in.v[f] = v[f];
    for (int a = 0; a < 24; ++a)
        for (int d = 0; d < 3; ++d) in.d1[a][d] = d1[a * 3 + d];
    for (int b = 0; b < 12; ++b)
        for (int m = 0; m < 6; ++m) in.d2[b][m] = d2[b * 6 + m];
    return in;
}

}  // namespace

extern "C" {

// Counts the FP64 operations of one pointwise RHS evaluation on the given point data
// (v: 27 values, d1: 24x3, d2: 12x6 in the kernel's slot order). out: [sections][6] =
// {add, mul, fma, div, cmp, waste}. Returns the number of sections.
int grf_count_point_ops(const grf_params* p, const double* v, const double* d1, const double* d2, long long* out) {
    using grfc::CD;
    std::memset(grfc::g_cnt, 0, sizeof(grfc::g_cnt));
    grfc::g_sec = 0;
    grf::PointInT<CD> in;
    for (int f = 0; f < grf::NFIELDS; ++f) in.v[f] = CD::var(v[f]);
    for (int a = 0; a < 24; ++a)
        for (int d = 0; d < 3; ++d) in.d1[a][d] = CD::var(d1[a * 3 + d]);
    for (int b = 0; b < 12; ++b)
        for (int m = 0; m < 6; ++m) in.d2[b][m] = CD::var(d2[b * 6 + m]);
    const grf::Coeffs c = host_coeffs(p);
    CD rhs[grf::NFIELDS];
    grf::PointExtraT<CD> ex;
    bool ok = true;
    grf::point_rhs(c, in, rhs, &ex, ok);
    for (int s = 0; s < grfc::kSections; ++s) {
        const grfc::Counts& k = grfc::g_cnt[s];
        long long* o = out + 6 * s;
        o[0] = k.add; o[1] = k.mul; o[2] = k.fma; o[3] = k.div; o[4] = k.cmp; o[5] = k.waste;
    }
    return grfc::kSections;
}

// The same pointwise RHS instantiated for the host in double precision (for CPU checks of
// the kernel formulas against the oracle). Slots as above; extra (may be NULL): H, M_1..3.
int grf_host_point_rhs(const grf_params* p, const double* v, const double* d1, const double* d2, double* rhs,
                       double* extra) {
    const grf::PointInT<double> in = host_point(v, d1, d2);
    const grf::Coeffs c = host_coeffs(p);
    grf::PointExtraT<double> ex;
    bool ok = true;
    grf::point_rhs(c, in, rhs, &ex, ok);
    if (extra) {
        extra[0] = ex.ham;
        for (int i = 0; i < 3; ++i) extra[1 + i] = ex.mom[i];
    }
    return ok ? 0 : -5;
}

// The kernel's Psi_4 (from the Riemann blocks) of the same host instance; xyz the point's
// coordinates relative to the triad's origin; out2 = (re, im).
int grf_host_point_psi4(const grf_params* p, const double* v, const double* d1, const double* d2, const double* xyz,
                        double* out2) {
    const grf::PointInT<double> in = host_point(v, d1, d2);
    const grf::Coeffs c = host_coeffs(p);
    grf::PointExtraT<double> ex;
    ex.want_psi4 = 1;
    for (int d = 0; d < 3; ++d) ex.xyz[d] = xyz[d];
    double rhs[grf::NFIELDS];
    bool ok = true;
    grf::point_rhs(c, in, rhs, &ex, ok);
    out2[0] = ex.psi4[0];
    out2[1] = ex.psi4[1];
    return ok ? 0 : -5;
}

// The kernel's hyperbolicity diagnostics (det M, det g_eff / det g, -g_eff^nn, smallest pivot
// ratio) of the same host instance; out4 receives the four.
int grf_host_point_hyp(const grf_params* p, const double* v, const double* d1, const double* d2, double* out4) {
    const grf::PointInT<double> in = host_point(v, d1, d2);
    const grf::Coeffs c = host_coeffs(p);
    grf::PointExtraT<double> ex;
    ex.want_hyp = 1;
    double rhs[grf::NFIELDS];
    bool ok = true;
    grf::point_rhs(c, in, rhs, &ex, ok);
    for (int m = 0; m < 4; ++m) out4[m] = ex.hyp[m];
    return ok ? 0 : -5;
}

}  // extern "C"
