// Enumeration of the ghost shell of a box (the Sommerfeld ghost update, the halo exchange of
// split boxes): one index per point, consecutive indices along x rows where the shell has them.
#pragma once

#include "grf_kernels.cuh"

namespace grf {

// Point number t (0 <= t < shell_count) of the shell [L, N)^3 minus the interior, in ghosted
// indices: L = 0 gives every ghost point, L = ng the ghosts beyond a high face with no coordinate
// below the box. Order: the full planes below and above the interior planes, then, plane by plane
// through the interior planes, the full rows below and above the interior rows, then the points
// before and after every interior row.
__device__ __forceinline__ void shell_point(const Geom& g, int L, long long t, int& i, int& j, int& k) {
    const int ex = g.NX - L, ey = g.NY - L, ez = g.NZ - L, a = g.ng - L;
    const long long plane = (long long)ex * ey;
    const long long full = (long long)(ez - g.nz) * plane;
    if (t < full) {
        const int q = (int)(t / plane);
        const long long r = t - q * plane;
        k = q < a ? q : q + g.nz;
        j = (int)(r / ex);
        i = (int)(r - (long long)j * ex);
    } else {
        t -= full;
        const long long rows = (long long)(ey - g.ny) * ex, ring = rows + (long long)g.ny * (ex - g.nx);
        const int q = (int)(t / ring);
        long long r = t - q * ring;
        k = a + q;
        if (r < rows) {
            const int jr = (int)(r / ex);
            j = jr < a ? jr : jr + g.ny;
            i = (int)(r - (long long)jr * ex);
        } else {
            r -= rows;
            const int w = ex - g.nx;
            j = a + (int)(r / w);
            const int e = (int)(r - (long long)(j - a) * w);
            i = e < a ? e : e + g.nx;
        }
    }
    i += L;
    j += L;
    k += L;
}

__host__ __device__ __forceinline__ long long shell_count(const Geom& g, int L) {
    const long long ex = g.NX - L, ey = g.NY - L, ez = g.NZ - L;
    return (ez - g.nz) * ex * ey + (long long)g.nz * ((ey - g.ny) * ex + (long long)g.ny * (ex - g.nx));
}

}  // namespace grf
