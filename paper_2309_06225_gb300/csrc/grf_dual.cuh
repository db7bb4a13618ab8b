// Forward-mode dual number with three tangent directions: value v and derivatives d[0..2]
// with respect to three parameters. Exact first-order propagation through +, -, *, /, fma;
// fabs/fmax/comparisons act on the value (their derivative is that of the selected branch).
#pragma once

#ifdef __CUDACC__
#define GRF_DHD __host__ __device__ __forceinline__
#else
#include <cmath>
#define GRF_DHD inline
#endif

namespace grf_dual {

struct D3 {
    double v, d0, d1, d2;
    D3() = default;
    GRF_DHD D3(double x) : v(x), d0(0.0), d1(0.0), d2(0.0) {}
    GRF_DHD D3(double x, double a, double b, double c) : v(x), d0(a), d1(b), d2(c) {}
};

GRF_DHD D3 operator+(const D3& a, const D3& b) { return D3(a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2); }
GRF_DHD D3 operator+(const D3& a, double b) { return D3(a.v + b, a.d0, a.d1, a.d2); }
GRF_DHD D3 operator+(double a, const D3& b) { return D3(a + b.v, b.d0, b.d1, b.d2); }
GRF_DHD D3 operator-(const D3& a, const D3& b) { return D3(a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2); }
GRF_DHD D3 operator-(const D3& a, double b) { return D3(a.v - b, a.d0, a.d1, a.d2); }
GRF_DHD D3 operator-(double a, const D3& b) { return D3(a - b.v, -b.d0, -b.d1, -b.d2); }
GRF_DHD D3 operator-(const D3& a) { return D3(-a.v, -a.d0, -a.d1, -a.d2); }
GRF_DHD D3 operator*(const D3& a, const D3& b) {
    return D3(a.v * b.v, fma(a.v, b.d0, a.d0 * b.v), fma(a.v, b.d1, a.d1 * b.v), fma(a.v, b.d2, a.d2 * b.v));
}
GRF_DHD D3 operator*(const D3& a, double b) { return D3(a.v * b, a.d0 * b, a.d1 * b, a.d2 * b); }
GRF_DHD D3 operator*(double a, const D3& b) { return D3(a * b.v, a * b.d0, a * b.d1, a * b.d2); }
GRF_DHD D3 operator/(const D3& a, const D3& b) {
    const double ib = 1.0 / b.v;
    const double q = a.v * ib;
    return D3(q, (a.d0 - q * b.d0) * ib, (a.d1 - q * b.d1) * ib, (a.d2 - q * b.d2) * ib);
}
GRF_DHD D3 operator/(const D3& a, double b) { return a * (1.0 / b); }
GRF_DHD D3 exp(const D3& a) {
    const double e = ::exp(a.v);
    return D3(e, e * a.d0, e * a.d1, e * a.d2);
}
GRF_DHD D3 operator/(double a, const D3& b) {
    const double q = a / b.v;
    const double r = -q / b.v;
    return D3(q, r * b.d0, r * b.d1, r * b.d2);
}
GRF_DHD D3& operator+=(D3& a, const D3& b) { a = a + b; return a; }
GRF_DHD D3& operator-=(D3& a, const D3& b) { a = a - b; return a; }
GRF_DHD D3& operator*=(D3& a, const D3& b) { a = a * b; return a; }
GRF_DHD D3& operator*=(D3& a, double b) { a = a * b; return a; }
GRF_DHD bool operator>(const D3& a, const D3& b) { return a.v > b.v; }
GRF_DHD bool operator<(const D3& a, const D3& b) { return a.v < b.v; }

GRF_DHD D3 fma(const D3& a, const D3& b, const D3& c) {
    return D3(::fma(a.v, b.v, c.v), ::fma(a.v, b.d0, ::fma(a.d0, b.v, c.d0)), ::fma(a.v, b.d1, ::fma(a.d1, b.v, c.d1)),
              ::fma(a.v, b.d2, ::fma(a.d2, b.v, c.d2)));
}
GRF_DHD D3 fma(double a, const D3& b, const D3& c) {
    return D3(::fma(a, b.v, c.v), ::fma(a, b.d0, c.d0), ::fma(a, b.d1, c.d1), ::fma(a, b.d2, c.d2));
}
GRF_DHD D3 fma(const D3& a, double b, const D3& c) { return fma(b, a, c); }
GRF_DHD D3 fma(const D3& a, const D3& b, double c) {
    return D3(::fma(a.v, b.v, c), ::fma(a.v, b.d0, a.d0 * b.v), ::fma(a.v, b.d1, a.d1 * b.v), ::fma(a.v, b.d2, a.d2 * b.v));
}
GRF_DHD D3 fma(double a, double b, const D3& c) { return D3(::fma(a, b, c.v), c.d0, c.d1, c.d2); }
GRF_DHD D3 fma(double a, const D3& b, double c) { return D3(::fma(a, b.v, c), a * b.d0, a * b.d1, a * b.d2); }
GRF_DHD D3 fma(const D3& a, double b, double c) { return fma(b, a, c); }
GRF_DHD D3 fabs(const D3& a) { return a.v < 0.0 ? -a : a; }
GRF_DHD D3 fmax(const D3& a, const D3& b) { return a.v >= b.v ? a : b; }
GRF_DHD D3 fmax(const D3& a, double b) { return a.v >= b ? a : D3(b); }

}  // namespace grf_dual
