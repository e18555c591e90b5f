// Camera: static observer at (r_cam, theta_o, phi = 0) and the pinhole sky directions.
#pragma once
#include "kerr.cuh"

namespace prt {

// The static-observer frame at the camera (t-leg along d_t; spatial legs by Gram-Schmidt of
// d_phi, d_theta, d_r so the radial leg is the Boyer-Lindquist radial direction) is computed
// once per camera on the host (host_camera_frame) and carried in Camera::e.

// Sky direction s ~ (-1, -y/r_cam, x/r_cam) on (e_r, e_theta, e_phi) for image-plane (x, y):
// the pixel centre x = (ix + 1/2 - nx/2) fov / nx (square pixels), with the camera's
// precomputed pixel side and 1 / r_cam (no division on the FP64 pipe).
__device__ __forceinline__ void sky_direction(const Camera &c, int ix, int iy, double s[3]) {
    double px = ((double)ix + (0.5 - 0.5 * c.nx)) * c.pix;
    double py = ((double)iy + (0.5 - 0.5 * c.ny)) * c.pix;
    double al = px * c.inv_r_cam, be = py * c.inv_r_cam;
    double n = rsqrt(1.0 + al * al + be * be);
    s[0] = -n;
    s[1] = -be * n;
    s[2] = al * n;
}

}  // namespace prt
