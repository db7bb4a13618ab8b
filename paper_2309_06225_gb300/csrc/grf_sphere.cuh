// The 26-point quadrature rule on the unit sphere used by the sphere-averaged scalar signal
// (tangent-linear and adjoint kernels).
#pragma once

namespace grf {

// 26-point rule of degree 7 on the unit sphere: 6 axis points (w 1/21), 12 edge midpoints
// (+-1,+-1,0)/sqrt2 (w 4/105), 8 corners (+-1,+-1,+-1)/sqrt3 (w 9/280); the weights sum to 1.
__device__ __forceinline__ void sphere_point(int q, double& x, double& y, double& z, double& w) {
    const double s2 = 0.70710678118654752440, s3 = 0.57735026918962576451;
    if (q < 6) {
        x = y = z = 0.0;
        const double sgn = (q & 1) ? -1.0 : 1.0;
        if (q < 2) x = sgn; else if (q < 4) y = sgn; else z = sgn;
        w = 1.0 / 21.0;
    } else if (q < 18) {
        const int e = q - 6, pair = e / 4;
        const double a = (e & 1) ? -s2 : s2, b = (e & 2) ? -s2 : s2;
        if (pair == 0) { x = a; y = b; z = 0.0; } else if (pair == 1) { x = a; y = 0.0; z = b; } else { x = 0.0; y = a; z = b; }
        w = 4.0 / 105.0;
    } else {
        const int e = q - 18;
        x = (e & 1) ? -s3 : s3;
        y = (e & 2) ? -s3 : s3;
        z = (e & 4) ? -s3 : s3;
        w = 9.0 / 280.0;
    }
}

}  // namespace grf
