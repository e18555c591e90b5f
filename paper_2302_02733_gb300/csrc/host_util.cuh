// Host-side helpers shared by the entry points: pointer classification, parameter checks, and
// the kernel form of the camera and of the plasma model (constants of the parameters only).
#pragma once
#include <cmath>

#include "rt_ctx.cuh"

namespace prt {

inline bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Prograde ISCO radius (Bardeen, Press & Teukolsky 1972).
inline double r_isco(double a) {
    double z1 = 1.0 + std::cbrt(1.0 - a * a) * (std::cbrt(1.0 + a) + std::cbrt(1.0 - a));
    double z2 = std::sqrt(3.0 * a * a + z1 * z1);
    return 3.0 + z2 - std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

// RT_OK, RT_ERR_INVALID or RT_ERR_SIZE for a camera description.
inline int check_camera(const rt_camera &cam) {
    if (!(std::fabs(cam.a) < 1.0) || !(cam.incl_deg > 0.0 && cam.incl_deg < 180.0) || cam.nx < 1 || cam.ny < 1 ||
        !(cam.freq_hz > 0.0) || !(cam.fov_M > 0.0) || !(cam.M_bh_g > 0.0) || !(cam.dist_cm > 0.0))
        return RT_ERR_INVALID;
    double rh = 1.0 + std::sqrt(1.0 - cam.a * cam.a);
    if (!(cam.r_cam > 2.0 * rh)) return RT_ERR_INVALID;
    if ((long long)cam.nx * cam.ny > (1ll << 31)) return RT_ERR_SIZE;
    return RT_OK;
}

inline Camera make_camera(const rt_camera &rc, double eps, int nmax) {
    Camera cam{};
    cam.a = rc.a;
    cam.r_cam = rc.r_cam;
    cam.theta_o = rc.incl_deg * kPi / 180.0;
    cam.nu_obs = rc.freq_hz;
    cam.fov = rc.fov_M;
    cam.L_unit = kG * rc.M_bh_g / (kC * kC);
    cam.nx = rc.nx;
    cam.ny = rc.ny;
    cam.eps = eps;
    cam.nmax = nmax;
    cam.rh = 1.0 + std::sqrt(1.0 - rc.a * rc.a);
    return cam;
}

// Kernel form of the loaded model for a camera. For a grid, M_unit and R_high replace the
// loaded values when positive.
inline Model make_model(const rt_ctx *c, const Camera &cam, double M_unit = 0.0, double R_high = 0.0) {
    Model mod{};
    mod.kind = c->model.kind;
    mod.edf = c->model.edf;
    mod.kappa = c->model.kappa;
    if (mod.kind == RT_MODEL_ADAF) {
        const rt_adaf_params &a = c->model.adaf;
        mod.adaf = AdafModel{a.n0, a.T0, a.beta, a.f_kep, a.Ti_over_Te, a.r_out, r_isco(cam.a)};
    } else {
        const rt_grid_params &g = c->model.grid;
        GridModel &gm = mod.grid;
        gm.n1 = g.n1;
        gm.n2 = g.n2;
        gm.n3 = g.n3;
        gm.r_in = g.r_in;
        gm.r_out = g.r_out;
        gm.x1in = std::log(g.r_in);
        gm.dx1 = (std::log(g.r_out) - gm.x1in) / g.n1;
        gm.dx2 = 1.0 / g.n2;
        gm.dx3 = 2.0 * kPi / g.n3;
        gm.hslope = g.hslope;
        gm.poly_xt = g.poly_xt;
        gm.poly_alpha = g.poly_alpha;
        gm.mks_smooth = g.mks_smooth;
        gm.poly_norm = 0.5 * kPi / (1.0 + 1.0 / ((g.poly_alpha + 1.0) * std::pow(g.poly_xt, g.poly_alpha)));
        gm.prims = reinterpret_cast<const float4 *>(c->d_prims);
        gm.x2_table = c->d_x2;
        double L = cam.L_unit;
        gm.rho_unit = (M_unit > 0.0 ? M_unit : g.M_unit) / (L * L * L);
        gm.b_unit = kC * std::sqrt(4.0 * kPi * gm.rho_unit);
        gm.ne_unit = gm.rho_unit / (kMp + kMe);
        gm.R_high = R_high > 0.0 ? R_high : g.R_high;
        gm.R_low = g.R_low;
        gm.sigma_cut = g.sigma_cut;
        gm.gamma_ad = g.gamma_ad;
    }
    return mod;
}

}  // namespace prt

namespace prt {
// Release the batched form's buffers, graph and stream (rt_destroy).
void free_batch(rt_ctx *c);
}  // namespace prt
