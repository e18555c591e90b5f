// Camera: static observer at (r_cam, theta_o, phi = 0) and the pinhole sky directions.
#pragma once
#include "kerr.cuh"

namespace prt {

// Static-observer tetrad at the camera (t-leg along d_t; spatial legs by Gram-Schmidt of
// d_phi, d_theta, d_r so the radial leg is the Boyer-Lindquist radial direction).
__device__ __forceinline__ void camera_tetrad(double a, double r, double th, double e[4][4]) {
    KS<double> m;
    m.eval(a, r, th);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) e[i][j] = 0.0;
    e[0][0] = 1.0 / sqrt(-m.tt);
    for (int i = 3; i >= 1; i--) {
        double v[4] = {0.0, 0.0, 0.0, 0.0}, w[4];
        v[i] = 1.0;
        double p0 = m.dot(v, e[0]);
        for (int k = 0; k < 4; k++) w[k] = v[k] + p0 * e[0][k];
        for (int j = 3; j > i; j--) {
            double pj = m.dot(v, e[j]);
            for (int k = 0; k < 4; k++) w[k] -= pj * e[j][k];
        }
        double n = 1.0 / sqrt(m.dot(w, w));
        for (int k = 0; k < 4; k++) e[i][k] = w[k] * n;
    }
}

// Sky direction s ~ (-1, -y/r_cam, x/r_cam) on (e_r, e_theta, e_phi) for image-plane (x, y).
__device__ __forceinline__ void sky_direction(const Camera &c, int ix, int iy, double s[3]) {
    double px = ((ix + 0.5) / c.nx - 0.5) * c.fov;
    double py = ((iy + 0.5) / c.ny - 0.5) * c.fov * ((double)c.ny / c.nx);
    double al = px / c.r_cam, be = py / c.r_cam;
    double n = 1.0 / sqrt(1.0 + al * al + be * be);
    s[0] = -n;
    s[1] = -be * n;
    s[2] = al * n;
}

}  // namespace prt
