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
    if ((long long)cam.nx * cam.ny > 2147483647ll) return RT_ERR_SIZE;  // pixels are indexed by int
    return RT_OK;
}

// The static camera's frame on the host (the kernels' camera_tetrad): t-leg along d_t, spatial
// legs by Gram-Schmidt of d_phi, d_theta, d_r in the Kerr-Schild metric at (r, th).
inline void host_camera_frame(double a, double r, double th, double e[4][4]) {
    double s = std::sin(th), c = std::cos(th), s2 = s * s;
    double sig = r * r + a * a * c * c, q = 2.0 * r / sig;
    double g[4][4] = {};
    g[0][0] = -(1.0 - q);
    g[0][1] = g[1][0] = q;
    g[0][3] = g[3][0] = -a * q * s2;
    g[1][1] = 1.0 + q;
    g[1][3] = g[3][1] = -a * s2 * (1.0 + q);
    g[2][2] = sig;
    g[3][3] = s2 * (sig + a * a * s2 * (1.0 + q));
    auto dot = [&](const double *u, const double *v) {
        double d = 0.0;
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) d += g[i][j] * u[i] * v[j];
        return d;
    };
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) e[i][j] = 0.0;
    e[0][0] = 1.0 / std::sqrt(-g[0][0]);
    for (int i = 3; i >= 1; i--) {
        double v[4] = {0.0, 0.0, 0.0, 0.0}, w[4];
        v[i] = 1.0;
        double p0 = dot(v, e[0]);
        for (int k = 0; k < 4; k++) w[k] = v[k] + p0 * e[0][k];
        for (int j = 3; j > i; j--) {
            double pj = dot(v, e[j]);
            for (int k = 0; k < 4; k++) w[k] -= pj * e[j][k];
        }
        double n = 1.0 / std::sqrt(dot(w, w));
        for (int k = 0; k < 4; k++) e[i][k] = w[k] * n;
    }
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
    cam.r_stop = 1.05 * cam.rh;
    cam.f_a = (float)cam.a;
    cam.f_nu_obs = (float)cam.nu_obs;
    cam.f_L_unit = (float)cam.L_unit;
    host_camera_frame(cam.a, cam.r_cam, cam.theta_o, cam.e);
    cam.pix = cam.fov / cam.nx;
    cam.inv_r_cam = 1.0 / cam.r_cam;
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 4; k++) cam.f_e[i][k] = (float)cam.e[i + 1][k];
    cam.f_pix = (float)(cam.fov / cam.nx);
    cam.f_r_cam = (float)cam.r_cam;
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
        AdafModel &m = mod.adaf;
        m.n0 = a.n0;
        m.T0 = a.T0;
        m.beta = a.beta;
        m.f_kep = a.f_kep;
        m.ti_te = a.Ti_over_Te;
        m.r_out = a.r_out;
        m.r_isco = r_isco(cam.a);
        m.te0 = a.T0 * kKb / (kMe * kC * kC);
        m.b0 = std::sqrt(8.0 * kPi * a.n0 * kKb * a.T0 * (1.0 + a.Ti_over_Te) / a.beta);
        m.f_n0 = (float)m.n0;
        m.f_te0 = (float)m.te0;
        m.f_b0 = (float)m.b0;
        m.f_f_kep = (float)m.f_kep;
        m.f_r_out = (float)m.r_out;
        m.f_r_isco = (float)m.r_isco;
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
        gm.x1_irc = c->d_x1c;
        gm.x1_irc_f2 = reinterpret_cast<const float2 *>(c->d_x1c + g.n1);
        gm.idx3 = g.n3 / (2.0 * kPi);
        gm.f_idx3_hi = (float)gm.idx3;
        gm.f_idx3_lo = (float)(gm.idx3 - (double)gm.f_idx3_hi);
        double L = cam.L_unit;
        gm.rho_unit = (M_unit > 0.0 ? M_unit : g.M_unit) / (L * L * L);
        gm.b_unit = kC * std::sqrt(4.0 * kPi * gm.rho_unit);
        gm.ne_unit = gm.rho_unit / (kMp + kMe);
        gm.R_high = R_high > 0.0 ? R_high : g.R_high;
        gm.R_low = g.R_low;
        gm.sigma_cut = g.sigma_cut;
        gm.gamma_ad = g.gamma_ad;
        gm.x2_table_f = c->d_x2f;
        gm.f_r_in = (float)gm.r_in;
        gm.f_r_out = (float)gm.r_out;
        gm.f_x1in = (float)gm.x1in;
        gm.f_dx1 = (float)gm.dx1;
        gm.f_dx2 = (float)gm.dx2;
        gm.f_dx3 = (float)gm.dx3;
        gm.f_hslope = (float)gm.hslope;
        gm.f_poly_xt = (float)gm.poly_xt;
        gm.f_poly_alpha = (float)gm.poly_alpha;
        gm.f_poly_alpha1 = (float)(gm.poly_alpha + 1.0);
        gm.f_poly_norm = (float)gm.poly_norm;
        gm.f_mks_smooth = (float)gm.mks_smooth;
        gm.f_b_unit = (float)gm.b_unit;
        gm.f_ne_unit = (float)gm.ne_unit;
        gm.f_R_high = (float)gm.R_high;
        gm.f_R_low = (float)gm.R_low;
        gm.f_sigma_cut = (float)gm.sigma_cut;
        gm.f_gamma_ad = (float)gm.gamma_ad;
    }
    return mod;
}

}  // namespace prt

namespace prt {
// Release the batched form's buffers, graph and stream (rt_destroy).
void free_batch(rt_ctx *c);
}  // namespace prt

// capi.cu: the batched form through the overlapped two-kernel shape
int render_jobs_overlap(rt_ctx *c, int form, const prt::JobDev *d_jobs, const prt::JobDev *h_jobs, int njobs,
                        long long nrays);
