// Reverse-mode (adjoint) scalar for the pointwise right-hand side: every arithmetic operation on
// two non-constant operands appends one entry to a per-thread tape, holding the operands' node
// indices and the partial derivatives of the result with respect to them; the reverse sweep
// walks the tape backwards and accumulates adjoints (the vector-Jacobian product of the whole
// pointwise function, exact to rounding).
//
//   * a value is {v, i}: its double value and its node index (i < 0: a constant, no derivative);
//   * nodes 0 .. nleaf-1 are the inputs (leaves); tape entry n creates node nleaf + n;
//   * an entry has up to three operands: a (partial pa), b (partial pb) and c (partial 1), so
//     that a*b + c (fma) is one entry;
//   * operations with a constant operand fold: x + c and x - c reuse x's node (partial 1), x * c
//     records one operand, and operations on constants only record nothing;
//   * fabs / fmax / comparisons act on values; a selected operand keeps its node (the derivative
//     of the branch taken), which makes the pivoted 7x7 LU differentiable entry by entry.
//
// Storage: entry n of the thread in column `col` lives at [n * stride + col] (so that a warp's
// entries are contiguous): partials as double2, operand indices as ushort4 (0xffff = none);
// adjoints at adj[node * stride + col].
#pragma once

#ifdef __CUDACC__
#include <cuda_runtime.h>
#define GRF_RHD __device__ __forceinline__
#else
#include <cmath>
#define GRF_RHD inline
#endif

namespace grf_rev {

constexpr unsigned short kNone = 0xffffu;

#ifdef __CUDACC__
struct Tape {
    double2* w;         // partials of operands a, b
    ushort4* ix;        // operand nodes a, b, c (c with partial 1); kNone where absent
    double* adj;        // adjoint of every node
    long long stride;   // columns (threads holding a tape)
    int cap;            // entries per column
    int nleaf;          // leaf nodes
    int* status;        // bit 8 set on tape overflow
};

// The tape of the current launch, and each thread's entry count (blocks of up to 256 threads).
__constant__ Tape c_tape;
__shared__ int s_count[256];

__device__ __forceinline__ long long rev_col() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

__device__ __noinline__ int rev_record(int a, double pa, int b, double pb, int c) {
    const int t = threadIdx.x;
    int n = s_count[t];
    s_count[t] = n + 1;
    if (n >= c_tape.cap) {  // keep the write in bounds; the call reports the overflow
        atomicOr(c_tape.status, 8);
        n = c_tape.cap - 1;
    }
    const long long off = (long long)n * c_tape.stride + rev_col();
    // streaming (evict-first) stores: a wave's tapes are far larger than L2 and are read back only
    // by the sweep, so they should not push the taping kernel's own spilled registers out of L2
    __stcs(&c_tape.w[off], make_double2(pa, pb));
    __stcs(&c_tape.ix[off], make_ushort4(a < 0 ? kNone : (unsigned short)a, b < 0 ? kNone : (unsigned short)b,
                                         c < 0 ? kNone : (unsigned short)c, 0));
    return c_tape.nleaf + n;
}
#define GRF_REV_RECORD(a, pa, b, pb, c) rev_record(a, pa, b, pb, c)
#else
// Host build: entries are only counted (to size the tape); node indices stay consistent.
extern int g_host_entries;
extern int g_host_nleaf;
inline int host_record(int, double, int, double, int) { return g_host_nleaf + g_host_entries++; }
#define GRF_REV_RECORD(a, pa, b, pb, c) host_record(a, pa, b, pb, c)
#endif

struct Rev {
    double v;
    int i;
    Rev() = default;
    GRF_RHD Rev(double x) : v(x), i(-1) {}  // NOLINT: constants convert implicitly
    GRF_RHD Rev(double x, int node) : v(x), i(node) {}
};

GRF_RHD Rev operator+(const Rev& a, const Rev& b) {
    const double v = a.v + b.v;
    if (a.i < 0) return Rev(v, b.i);
    if (b.i < 0) return Rev(v, a.i);
    return Rev(v, GRF_REV_RECORD(a.i, 1.0, b.i, 1.0, -1));
}
GRF_RHD Rev operator-(const Rev& a) {
    if (a.i < 0) return Rev(-a.v);
    return Rev(-a.v, GRF_REV_RECORD(a.i, -1.0, -1, 0.0, -1));
}
GRF_RHD Rev operator-(const Rev& a, const Rev& b) {
    const double v = a.v - b.v;
    if (b.i < 0) return Rev(v, a.i);
    if (a.i < 0) return Rev(v, GRF_REV_RECORD(b.i, -1.0, -1, 0.0, -1));
    return Rev(v, GRF_REV_RECORD(a.i, 1.0, b.i, -1.0, -1));
}
GRF_RHD Rev operator*(const Rev& a, const Rev& b) {
    const double v = a.v * b.v;
    if (a.i < 0 && b.i < 0) return Rev(v);
    if (a.i < 0) return Rev(v, GRF_REV_RECORD(b.i, a.v, -1, 0.0, -1));
    if (b.i < 0) return Rev(v, GRF_REV_RECORD(a.i, b.v, -1, 0.0, -1));
    return Rev(v, GRF_REV_RECORD(a.i, b.v, b.i, a.v, -1));
}
GRF_RHD Rev operator/(const Rev& a, const Rev& b) {
    const double ib = 1.0 / b.v;
    const double q = a.v * ib;
    if (a.i < 0 && b.i < 0) return Rev(a.v / b.v);
    if (b.i < 0) return Rev(q, GRF_REV_RECORD(a.i, ib, -1, 0.0, -1));
    if (a.i < 0) return Rev(q, GRF_REV_RECORD(b.i, -q * ib, -1, 0.0, -1));
    return Rev(q, GRF_REV_RECORD(a.i, ib, b.i, -q * ib, -1));
}
// a * b + c as one entry
GRF_RHD Rev fma(const Rev& a, const Rev& b, const Rev& c) {
    const double v = ::fma(a.v, b.v, c.v);
    const int ia = b.v == 0.0 ? -1 : a.i, ib = a.v == 0.0 ? -1 : b.i;  // zero partials record nothing
    if (ia < 0 && ib < 0) return Rev(v, c.i);
    return Rev(v, GRF_REV_RECORD(ia, b.v, ib, a.v, c.i));
}
GRF_RHD Rev exp(const Rev& a) {
    const double e = ::exp(a.v);
    if (a.i < 0) return Rev(e);
    return Rev(e, GRF_REV_RECORD(a.i, e, -1, 0.0, -1));
}
GRF_RHD Rev& operator+=(Rev& a, const Rev& b) { a = a + b; return a; }
GRF_RHD Rev& operator-=(Rev& a, const Rev& b) { a = a - b; return a; }
GRF_RHD Rev& operator*=(Rev& a, const Rev& b) { a = a * b; return a; }
GRF_RHD bool operator>(const Rev& a, const Rev& b) { return a.v > b.v; }
GRF_RHD bool operator<(const Rev& a, const Rev& b) { return a.v < b.v; }
GRF_RHD Rev fabs(const Rev& a) { return a.v < 0.0 ? -a : a; }
GRF_RHD Rev fmax(const Rev& a, const Rev& b) { return a.v >= b.v ? a : b; }
// pivot tests of the 7x7 LU: magnitudes of values only, nothing recorded
GRF_RHD bool abs_gt(const Rev& a, const Rev& b) { return ::fabs(a.v) > ::fabs(b.v); }
GRF_RHD Rev abs_max7(const Rev M[7][8]) {
    double m = 0.0;
    for (int i = 0; i < 7; ++i)
        for (int j = 0; j < 7; ++j) m = ::fmax(m, ::fabs(M[i][j].v));
    return Rev(m);
}

}  // namespace grf_rev
