/*
 * Plain FP64 CPU oracle: test infrastructure only (see oracle.h for who may call it).
 *
 * Everything here is written as directly as the definitions allow. It has no blocking, no
 * fusion and no reordering beyond what each definition states, so a reader can check every
 * function against the formula cited in its comment. Units are G = c = M = 1 for geometry,
 * and cgs for radiation. The paper (Sections 2.1-2.2) describes the method in prose only.
 * Where it is silent, the reading used is stated in the function's comment.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

/* CODATA 2018 cgs constants */
#define O_G 6.67430e-8
#define O_C 2.99792458e10
#define O_ME 9.1093837015e-28
#define O_MP 1.67262192369e-24
#define O_QE 4.80320471257e-10
#define O_KB 1.380649e-16
#define O_H 6.62607015e-27
#define O_PI 3.14159265358979323846

static double dot4(const double g[16], const double u[4], const double v[4]) {
    double s = 0.0;
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) s += g[m * 4 + n] * u[m] * v[n];
    return s;
}

static void lower4(const double g[16], const double u[4], double ul[4]) {
    for (int m = 0; m < 4; m++) {
        ul[m] = 0.0;
        for (int n = 0; n < 4; n++) ul[m] += g[m * 4 + n] * u[n];
    }
}

/* ============================ geometry ==================================================
 * Reading: rays are integrated in spherical Kerr-Schild coordinates (t, r, theta, phi);
 * the paper names only "the" geodesic equation (Section 2.1). With Sigma = r^2 + a^2 cos^2:
 *   g_tt = -(1 - 2r/Sigma), g_tr = 2r/Sigma, g_tphi = -2 a r sin^2/Sigma,
 *   g_rr = 1 + 2r/Sigma, g_rphi = -a sin^2 (1 + 2r/Sigma), g_thth = Sigma,
 *   g_phiphi = sin^2 (Sigma + a^2 sin^2 (1 + 2r/Sigma)).
 */
void ora_metric_ks(double a, double r, double th, double g[16]) {
    double s = sin(th), c = cos(th), s2 = s * s;
    double sig = r * r + a * a * c * c;
    double q = 2.0 * r / sig;
    memset(g, 0, 16 * sizeof(double));
    g[0] = -1.0 + q;
    g[1] = g[4] = q;
    g[3] = g[12] = -a * s2 * q;
    g[5] = 1.0 + q;
    g[7] = g[13] = -a * s2 * (1.0 + q);
    g[10] = sig;
    g[15] = s2 * (sig + a * a * s2 * (1.0 + q));
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success, and the determinant via
 * ora_det4 below uses the same elimination. */
static int gj_invert(const double g[16], double inv[16], double *det) {
    double A[4][8];
    double d = 1.0;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 8; j++) A[i][j] = (j < 4) ? g[i * 4 + j] : (j - 4 == i ? 1.0 : 0.0);
    for (int c = 0; c < 4; c++) {
        int p = c;
        for (int i = c + 1; i < 4; i++)
            if (fabs(A[i][c]) > fabs(A[p][c])) p = i;
        if (A[p][c] == 0.0) return -1;
        if (p != c) {
            for (int j = 0; j < 8; j++) {
                double t = A[p][j];
                A[p][j] = A[c][j];
                A[c][j] = t;
            }
            d = -d;
        }
        double piv = A[c][c];
        d *= piv;
        for (int j = 0; j < 8; j++) A[c][j] /= piv;
        for (int i = 0; i < 4; i++) {
            if (i == c) continue;
            double f = A[i][c];
            for (int j = 0; j < 8; j++) A[i][j] -= f * A[c][j];
        }
    }
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) inv[i * 4 + j] = A[i][j + 4];
    if (det) *det = d;
    return 0;
}

int ora_invert4(const double g[16], double ginv[16]) { return gj_invert(g, ginv, NULL); }

/* Partial derivatives d/dr and d/dtheta of the Kerr-Schild metric above, by hand.
 * With q = 2r/Sigma: dq/dr = 2(a^2 cos^2 - r^2)/Sigma^2, dq/dth = 4 a^2 r sin cos/Sigma^2,
 * dSigma/dth = -2 a^2 sin cos. */
void ora_metric_derivs(double a, double r, double th, double dr[16], double dt[16]) {
    double s = sin(th), c = cos(th), s2 = s * s, sc = s * c;
    double sig = r * r + a * a * c * c;
    double q = 2.0 * r / sig;
    double dq_r = 2.0 * (a * a * c * c - r * r) / (sig * sig);
    double dq_t = 4.0 * a * a * r * sc / (sig * sig);
    double dsig_t = -2.0 * a * a * sc;
    memset(dr, 0, 16 * sizeof(double));
    memset(dt, 0, 16 * sizeof(double));
    dr[0] = dq_r;
    dt[0] = dq_t;
    dr[1] = dr[4] = dq_r;
    dt[1] = dt[4] = dq_t;
    dr[3] = dr[12] = -a * s2 * dq_r;
    dt[3] = dt[12] = -a * (2.0 * sc * q + s2 * dq_t);
    dr[5] = dq_r;
    dt[5] = dq_t;
    dr[7] = dr[13] = -a * s2 * dq_r;
    dt[7] = dt[13] = -a * (2.0 * sc * (1.0 + q) + s2 * dq_t);
    dr[10] = 2.0 * r;
    dt[10] = dsig_t;
    dr[15] = s2 * (2.0 * r + a * a * s2 * dq_r);
    dt[15] = 2.0 * sc * (sig + a * a * s2 * (1.0 + q)) +
             s2 * (dsig_t + a * a * (2.0 * sc * (1.0 + q) + s2 * dq_t));
}

/* Christoffel symbols of the second kind, by their definition
 *   Gamma^mu_{al be} = 1/2 g^{mu nu} (d_al g_{nu be} + d_be g_{nu al} - d_nu g_{al be}),
 * with d_t = d_phi = 0 (stationary, axisymmetric metric). */
void ora_connection(double a, double r, double th, double G[64]) {
    double g[16], gi[16], dg[4][16];
    ora_metric_ks(a, r, th, g);
    gj_invert(g, gi, NULL);
    memset(dg, 0, sizeof(dg));
    ora_metric_derivs(a, r, th, dg[1], dg[2]);
    for (int mu = 0; mu < 4; mu++)
        for (int al = 0; al < 4; al++)
            for (int be = 0; be < 4; be++) {
                double s = 0.0;
                for (int nu = 0; nu < 4; nu++)
                    s += gi[mu * 4 + nu] *
                         (dg[al][nu * 4 + be] + dg[be][nu * 4 + al] - dg[nu][al * 4 + be]);
                G[mu * 16 + al * 4 + be] = 0.5 * s;
            }
}

/* ============================ camera ====================================================
 * Section 2.1: one photon is launched per pixel from the camera. Reading:
 *   a static observer at (r_cam, theta = inclination, phi = 0), with e_(0) along d_t;
 *   spatial legs by metric Gram-Schmidt of d_phi, d_theta, d_r in that order, so the
 *   radial leg is the Boyer-Lindquist radial direction (in Kerr-Schild coordinates d_r
 *   leans along d_phi by a sin^2/r, which would tilt the line of sight);
 *   a pinhole image plane with pixel centres
 *     x = ((i + 1/2)/nx - 1/2) FOV,  y = ((j + 1/2)/ny - 1/2) FOV ny/nx;
 *   sky direction s ~ (-1, -y/r_cam, x/r_cam) on (e_r, e_theta, e_phi), so "up" is -theta;
 *   the backward (past-directed) tangent K^(a) = (-1, s_hat). The photon energy is 1 in
 *   units of the observing frequency: k = -K has -k.u_cam = 1.
 */
static void camera_frame(const ora_camera *cam, double e[4][4]) {
    double th = cam->incl_deg * O_PI / 180.0;
    double g[16];
    ora_metric_ks(cam->a, cam->r_cam, th, g);
    memset(e, 0, 16 * sizeof(double));
    e[0][0] = 1.0 / sqrt(-g[0]);
    /* Gram-Schmidt order d_phi, d_theta, d_r: legs e[3], e[2], e[1] */
    for (int i = 3; i >= 1; i--) {
        double v[4] = {0, 0, 0, 0}, w[4];
        v[i] = 1.0;
        double p0 = dot4(g, v, e[0]);
        for (int m = 0; m < 4; m++) w[m] = v[m] + p0 * e[0][m];
        for (int j = 3; j > i; j--) {
            double pj = dot4(g, v, e[j]);
            for (int m = 0; m < 4; m++) w[m] -= pj * e[j][m];
        }
        double n = sqrt(dot4(g, w, w));
        for (int m = 0; m < 4; m++) e[i][m] = w[m] / n;
    }
}

static void sky_dir(const ora_camera *cam, double px, double py, double s[3]) {
    double al = px / cam->r_cam, be = py / cam->r_cam;
    double n = sqrt(1.0 + al * al + be * be);
    s[0] = -1.0 / n;
    s[1] = -be / n;
    s[2] = al / n;
}

void ora_camera_ray(const ora_camera *cam, double px, double py, double x[4], double K[4]) {
    double e[4][4], s[3];
    camera_frame(cam, e);
    sky_dir(cam, px, py, s);
    for (int m = 0; m < 4; m++) K[m] = -e[0][m] + s[0] * e[1][m] + s[1] * e[2][m] + s[2] * e[3][m];
    x[0] = 0.0;
    x[1] = cam->r_cam;
    x[2] = cam->incl_deg * O_PI / 180.0;
    x[3] = 0.0;
}

static void pixel_xy(const ora_camera *cam, int ix, int iy, int pert, double *px, double *py) {
    *px = ((ix + 0.5) / cam->nx - 0.5) * cam->fov_M;
    *py = ((iy + 0.5) / cam->ny - 0.5) * cam->fov_M * ((double)cam->ny / cam->nx);
    if (pert == 1) *px = nextafter(*px, INFINITY);
    if (pert == 2) *py = nextafter(*py, INFINITY);
}

/* ============================ geodesic ==================================================
 * Null geodesic dx/dl = K, dK^mu/dl = -Gamma^mu_{al be} K^al K^be, integrated backward from
 * the camera and saved (Section 2.1; Section 2.2: the CPU code saves the path). Reading of
 * "adaptive and parameterized" step: classic RK4 with
 *   h = eps / (|K^r|/r + |K^th|/max(min(th, pi - th), 0.01) + |K^ph| + 1e-40),
 * i.e. at most a fraction eps of r, of the polar distance to the axis (down to 0.01 rad)
 * and eps radians of azimuth per step. The floor lets rays that pass through the axis cross
 * it in a few steps instead of approaching it geometrically.
 * Stops, checked in this order after each step: r < 1.05 r_h (HORIZON); r > r_cam with
 * K^r > 0 (ESCAPE); steps >= nmax (NMAX). A step that leaves 0 < theta < pi is reflected
 * through the pole (theta -> -theta or 2 pi - theta, phi += pi, K^th -> -K^th), and h is
 * stored negative to mark it.
 */
static void geo_rhs(double a, const double y[8], double dy[8]) {
    double G[64];
    ora_connection(a, y[1], y[2], G);
    for (int m = 0; m < 4; m++) dy[m] = y[4 + m];
    for (int m = 0; m < 4; m++) {
        double acc = 0.0;
        for (int al = 0; al < 4; al++)
            for (int be = 0; be < 4; be++) acc -= G[m * 16 + al * 4 + be] * y[4 + al] * y[4 + be];
        dy[4 + m] = acc;
    }
}

static double geo_step(double eps, const double y[8]) {
    double tt = fmax(fmin(y[2], O_PI - y[2]), 1e-2);
    return eps / (fabs(y[5]) / y[1] + fabs(y[6]) / tt + fabs(y[7]) + 1e-40);
}

static void rk4(double a, double h, const double y[8], double out[8]) {
    double k1[8], k2[8], k3[8], k4[8], t[8];
    geo_rhs(a, y, k1);
    for (int i = 0; i < 8; i++) t[i] = y[i] + 0.5 * h * k1[i];
    geo_rhs(a, t, k2);
    for (int i = 0; i < 8; i++) t[i] = y[i] + 0.5 * h * k2[i];
    geo_rhs(a, t, k3);
    for (int i = 0; i < 8; i++) t[i] = y[i] + h * k3[i];
    geo_rhs(a, t, k4);
    for (int i = 0; i < 8; i++) out[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

static int trace(const ora_camera *cam, double px, double py, int maxstates, double *st, int *status) {
    double y[8], yn[8];
    double rh = 1.0 + sqrt(1.0 - cam->a * cam->a);
    ora_camera_ray(cam, px, py, y, y + 4);
    for (int i = 0; i < 8; i++) st[i] = y[i];
    st[8] = 0.0;
    int n = 0;
    *status = 0;
    for (;;) {
        double h = geo_step(cam->eps, y);
        rk4(cam->a, h, y, yn);
        int refl = 0;
        if (yn[2] < 0.0) {
            yn[2] = -yn[2];
            yn[3] += O_PI;
            yn[6] = -yn[6];
            refl = 1;
        } else if (yn[2] > O_PI) {
            yn[2] = 2.0 * O_PI - yn[2];
            yn[3] += O_PI;
            yn[6] = -yn[6];
            refl = 1;
        }
        st[n * 9 + 8] = refl ? -h : h;
        n++;
        for (int i = 0; i < 8; i++) {
            y[i] = yn[i];
            st[n * 9 + i] = yn[i];
        }
        st[n * 9 + 8] = 0.0;
        int bad = 0;
        for (int i = 1; i < 8; i++)
            if (!isfinite(y[i])) bad = 1;
        if (bad) {
            *status = ORA_NAN;
            break;
        }
        if (y[1] < 1.05 * rh) {
            *status = ORA_HORIZON;
            break;
        }
        if (y[1] > cam->r_cam && y[5] > 0.0) {
            *status = ORA_ESCAPE;
            break;
        }
        if (n >= cam->nmax || n + 1 >= maxstates) {
            *status = ORA_NMAX;
            break;
        }
    }
    return n;
}

int ora_trace_geodesic(const ora_camera *cam, double px, double py, int maxstates, double *states,
                       int *status) {
    return trace(cam, px, py, maxstates, states, status);
}

/* ============================ plasma ====================================================
 * Section 2.1: plasma quantities are interpolated (GRMHD) or computed (semi-analytic) at
 * every point of the geodesic. */

/* Prograde marginally stable orbit (Bardeen, Press & Teukolsky 1972). */
static double r_isco(double a) {
    double z1 = 1.0 + cbrt(1.0 - a * a) * (cbrt(1.0 + a) + cbrt(1.0 - a));
    double z2 = sqrt(3.0 * a * a + z1 * z1);
    return 3.0 + z2 - sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

/* Semi-analytic ADAF. Reading (the model paper is not available):
 *   n_e = n0 r^-3/2, T_e = T0 / r, Theta_e = k T_e / (m_e c^2);
 *   B^2 / 8 pi = n_e k T_e (1 + T_i/T_e) / beta;
 *   Boyer-Lindquist u_mu = (-1, u_r, 0, l) with l = f l_K(max(r, r_isco)) sin^2 theta and
 *   u_r < 0 from the normalisation, raised, moved to KS (u^t += 2r/Delta u^r,
 *   u^phi += a/Delta u^r) and renormalised;
 *   field direction from KS components B^i ~ (1, 0, 1/r) through b^t = B^i u_i,
 *   b^i = (B^i + b^t u^i)/u^t; emission only for r <= r_out. */
static void adaf_plasma(const ora_camera *cam, const ora_model *m, const double x[4], double out[12]) {
    double a = cam->a, r = x[1], th = x[2];
    memset(out, 0, 12 * sizeof(double));
    if (r > m->r_out_emit) return;
    double ne = m->n0 * pow(r, -1.5);
    double Te = m->T0 / r;
    double thetae = O_KB * Te / (O_ME * O_C * O_C);
    double B = sqrt(8.0 * O_PI * ne * O_KB * Te * (1.0 + m->Ti_over_Te) / m->beta);
    double s = sin(th), c = cos(th), s2 = s * s;
    double sig = r * r + a * a * c * c;
    double del = r * r - 2.0 * r + a * a;
    double A = (r * r + a * a) * (r * r + a * a) - a * a * del * s2;
    double gtt = -A / (sig * del), gtp = -2.0 * a * r / (sig * del);
    double gpp = (del - a * a * s2) / (sig * del * s2), grr = del / sig;
    double rk = fmax(r, r_isco(a));
    double sq = sqrt(rk);
    double lK = (rk * rk - 2.0 * a * sq + a * a) / (rk * sq - 2.0 * sq + a);
    double l = m->f_kep * lK * s2;
    double rhs = -1.0 - gtt + 2.0 * gtp * l - gpp * l * l;
    double ur_low = -sqrt(fmax(rhs, 0.0) / grr);
    double u[4];
    u[0] = -gtt + gtp * l;
    u[1] = grr * ur_low;
    u[2] = 0.0;
    u[3] = -gtp + gpp * l;
    u[0] += 2.0 * r / del * u[1];
    u[3] += a / del * u[1];
    double g[16];
    ora_metric_ks(a, r, th, g);
    double nrm = sqrt(-dot4(g, u, u));
    for (int i = 0; i < 4; i++) u[i] /= nrm;
    double ul[4];
    lower4(g, u, ul);
    double Bi[4] = {0.0, 1.0, 0.0, 1.0 / r};
    double bt = Bi[1] * ul[1] + Bi[2] * ul[2] + Bi[3] * ul[3];
    double b[4] = {bt, 0, 0, 0};
    for (int i = 1; i < 4; i++) b[i] = (Bi[i] + bt * u[i]) / u[0];
    out[0] = ne;
    out[1] = thetae;
    out[2] = B;
    out[3] = 1.0;
    for (int i = 0; i < 4; i++) {
        out[4 + i] = u[i];
        out[8 + i] = b[i];
    }
}

/* FMKS polar angle: theta = theta_G + exp(s (X1_in - X1)) (theta_J - theta_G), with
 *   theta_G = pi X2 + (1 - h)/2 sin(2 pi X2),
 *   theta_J = N y (1 + (y/x_t)^alpha/(alpha + 1)) + pi/2, y = 2 X2 - 1,
 *   N = (pi/2) / (1 + x_t^-alpha/(alpha + 1)); X1 = ln r, X3 = phi. */
double ora_fmks_theta(const ora_model *m, double X1, double X2, double *dth1, double *dth2) {
    double h = m->hslope, al = m->poly_alpha, xt = m->poly_xt;
    double thg = O_PI * X2 + 0.5 * (1.0 - h) * sin(2.0 * O_PI * X2);
    double dthg = O_PI * (1.0 + (1.0 - h) * cos(2.0 * O_PI * X2));
    double y = 2.0 * X2 - 1.0;
    double N = 0.5 * O_PI / (1.0 + 1.0 / ((al + 1.0) * pow(xt, al)));
    double thj = N * y * (1.0 + pow(y / xt, al) / (al + 1.0)) + 0.5 * O_PI;
    double dthj = 2.0 * N * (1.0 + pow(y / xt, al));
    double w = exp(m->mks_smooth * (log(m->r_in) - X1));
    if (dth1) *dth1 = -m->mks_smooth * w * (thj - thg);
    if (dth2) *dth2 = dthg + w * (dthj - dthg);
    return thg + w * (thj - thg);
}

/* Inverse of theta(X1, X2) in X2 by bisection on [0, 1] to the last bit. */
double ora_fmks_x2(const ora_model *m, double X1, double th) {
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (ora_fmks_theta(m, X1, mid, NULL, NULL) < th)
            lo = mid;
        else
            hi = mid;
    }
    double flo = fabs(ora_fmks_theta(m, X1, lo, NULL, NULL) - th);
    double fhi = fabs(ora_fmks_theta(m, X1, hi, NULL, NULL) - th);
    return flo <= fhi ? lo : hi;
}

/* Trilinear interpolation on cell centres; clamped in X1 and X2, periodic in X3. */
void ora_grid_interp(const ora_model *m, double X1, double X2, double X3, double out[8]) {
    double x1in = log(m->r_in), dx1 = (log(m->r_out) - x1in) / m->n1;
    double dx2 = 1.0 / m->n2, dx3 = 2.0 * O_PI / m->n3;
    double fi = (X1 - x1in) / dx1 - 0.5;
    double fj = X2 / dx2 - 0.5;
    double fk = X3 / dx3 - 0.5;
    fi = fmin(fmax(fi, 0.0), m->n1 - 1.0);
    fj = fmin(fmax(fj, 0.0), m->n2 - 1.0);
    int i0 = (int)floor(fi), j0 = (int)floor(fj);
    if (i0 > m->n1 - 2) i0 = m->n1 - 2;
    if (j0 > m->n2 - 2) j0 = m->n2 - 2;
    double w1 = fi - i0, w2 = fj - j0;
    double kf = floor(fk);
    double w3 = fk - kf;
    long k0 = ((long)kf % m->n3 + m->n3) % m->n3, k1 = (k0 + 1) % m->n3;
    for (int v = 0; v < 8; v++) out[v] = 0.0;
    for (int di = 0; di < 2; di++)
        for (int dj = 0; dj < 2; dj++)
            for (int dk = 0; dk < 2; dk++) {
                double w = (di ? w1 : 1.0 - w1) * (dj ? w2 : 1.0 - w2) * (dk ? w3 : 1.0 - w3);
                long k = dk ? k1 : k0;
                const float *p = m->prims + (((long)(i0 + di) * m->n2 + (j0 + dj)) * m->n3 + k) * 8;
                for (int v = 0; v < 8; v++) out[v] += w * (double)p[v];
            }
}

/* GRMHD-shaped grid. Reading (HARM primitive conventions):
 *   U^i is the velocity relative to the normal observer and B^i the field; both are
 *   moved from FMKS to KS components with the spatial Jacobian d(r, th, ph)/d(X1, X2, X3);
 *   lapse alpha = (-g^tt)^-1/2, shift beta^i = alpha^2 g^ti, gamma = sqrt(1 + g_ij U^i U^j);
 *   u^t = gamma/alpha, u^i = U^i - gamma beta^i/alpha; b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t.
 *   Units: L = GM/c^2, rho_unit = M_unit/L^3, B_unit = c sqrt(4 pi rho_unit),
 *   n_e = rho rho_unit/(m_p + m_e).
 *   beta_p = 2(gamma_ad - 1) u / b^2, R = R_high beta_p^2/(1 + beta_p^2) + R_low/(1 + beta_p^2)
 *   (taken as R_low once (1/beta_p)^2 exceeds 1e30),
 *   Theta_e = (m_p/m_e)(gamma_ad - 1) u / (rho (1 + R)).
 *   No emission where sigma = b^2/rho > sigma_cut or outside r_in <= r <= r_out. */
static void grid_plasma(const ora_camera *cam, const ora_model *m, const double x[4], double out[12]) {
    double a = cam->a, r = x[1], th = x[2];
    memset(out, 0, 12 * sizeof(double));
    if (r < m->r_in || r > m->r_out) return;
    double X1 = log(r);
    double X2 = ora_fmks_x2(m, X1, th);
    double X3 = fmod(x[3], 2.0 * O_PI);
    if (X3 < 0.0) X3 += 2.0 * O_PI;
    double P[8];
    ora_grid_interp(m, X1, X2, X3, P);
    double rho = P[0], uu = P[1];
    if (!(rho > 0.0) || !(uu > 0.0)) return;
    double dth1, dth2;
    ora_fmks_theta(m, X1, X2, &dth1, &dth2);
    double Ut[4] = {0.0, r * P[2], dth1 * P[2] + dth2 * P[3], P[4]};
    double Bi[4] = {0.0, r * P[5], dth1 * P[5] + dth2 * P[6], P[7]};
    double g[16], gi[16];
    ora_metric_ks(a, r, th, g);
    gj_invert(g, gi, NULL);
    double alpha = 1.0 / sqrt(-gi[0]);
    double beta[4] = {0.0, gi[1] * alpha * alpha, gi[2] * alpha * alpha, gi[3] * alpha * alpha};
    double qsp = 0.0;
    for (int i = 1; i < 4; i++)
        for (int j = 1; j < 4; j++) qsp += g[i * 4 + j] * Ut[i] * Ut[j];
    double gam = sqrt(1.0 + qsp);
    double u[4];
    u[0] = gam / alpha;
    for (int i = 1; i < 4; i++) u[i] = Ut[i] - gam * beta[i] / alpha;
    double ul[4];
    lower4(g, u, ul);
    double bt = Bi[1] * ul[1] + Bi[2] * ul[2] + Bi[3] * ul[3];
    double b[4] = {bt, 0, 0, 0};
    for (int i = 1; i < 4; i++) b[i] = (Bi[i] + bt * u[i]) / u[0];
    double bsq = dot4(g, b, b);
    if (bsq / rho > m->sigma_cut) return;
    double L = O_G * cam->M_bh_g / (O_C * O_C);
    double rho_unit = m->M_unit / (L * L * L);
    double B_unit = O_C * sqrt(4.0 * O_PI * rho_unit);
    double ga = m->gamma_ad;
    /* R = (R_high b^2 + R_low)/(1 + b^2) in terms of 1/b, b = beta_p, so nothing overflows */
    double ib = bsq / (2.0 * (ga - 1.0) * uu);
    double ib2 = ib * ib;
    double R = ib2 < 1e30 ? (m->R_high + m->R_low * ib2) / (1.0 + ib2) : m->R_low;
    out[0] = rho * rho_unit / (O_MP + O_ME);
    out[1] = (O_MP / O_ME) * (ga - 1.0) * uu / (rho * (1.0 + R));
    out[2] = sqrt(fmax(bsq, 0.0)) * B_unit;
    out[3] = 1.0;
    for (int i = 0; i < 4; i++) {
        out[4 + i] = u[i];
        out[8 + i] = b[i];
    }
}

/* Static sphere, for the pins of the camera-to-flux chain and of the depth maps: a model whose
 * image has a closed form (it is not one of the paper's models). Inside r < R the temperature
 * and field strength are constant and the density is constant or, with sph_smooth, falls as
 * (1 - r^2/R^2)^2 to zero at the surface (so that sums along a ray converge without an edge
 * term); the fluid is at rest, u = d_t / |d_t| (outside the ergoregion), and the field
 * direction is d_phi made normal to u. */
static void sphere_plasma(const ora_camera *cam, const ora_model *m, const double x[4], double out[12]) {
    memset(out, 0, 12 * sizeof(double));
    if (!(x[1] < m->sph_R)) return;
    double g[16];
    ora_metric_ks(cam->a, x[1], x[2], g);
    if (!(g[0] < 0.0)) return;
    double u[4] = {1.0 / sqrt(-g[0]), 0.0, 0.0, 0.0};
    double ph[4] = {0.0, 0.0, 0.0, 1.0};
    double pu = dot4(g, ph, u);
    double b[4];
    for (int i = 0; i < 4; i++) b[i] = ph[i] + pu * u[i];
    double nb = sqrt(dot4(g, b, b));
    double q = 1.0 - x[1] * x[1] / (m->sph_R * m->sph_R);
    out[0] = m->sph_smooth ? m->sph_ne * q * q : m->sph_ne;
    out[1] = m->sph_Te;
    out[2] = m->sph_B;
    out[3] = 1.0;
    for (int i = 0; i < 4; i++) {
        out[4 + i] = u[i];
        out[8 + i] = b[i] / nb;
    }
}

void ora_plasma(const ora_camera *cam, const ora_model *m, const double x[4], double out[12]) {
    if (m->kind == ORA_MODEL_ADAF)
        adaf_plasma(cam, m, x, out);
    else if (m->kind == ORA_MODEL_SPHERE)
        sphere_plasma(cam, m, x, out);
    else
        grid_plasma(cam, m, x, out);
}

/* ============================ coefficients ==============================================
 * Section 2.1: synchrotron emission, self-absorption, Faraday rotation and conversion for a
 * thermal (Maxwell-Juttner) distribution. Reading: the fits of Dexter (2016) for emission,
 * Kirchhoff's law for absorption, and the Shcherbakov (2008) rotativity fits in the form
 * collected by Dexter (2016). Polarization basis: Stokes Q is positive along the fluid-frame
 * leg e_(1), perpendicular to the projected field, so j_U = a_U = r_U = 0. The circular
 * terms carry the sign of cos(theta_B). */

/* e^z K_n(z) from the integral representation K_n(z) = int_0^inf exp(-z cosh t) cosh(n t) dt,
 * by the trapezoid rule (exponentially convergent for this analytic integrand). */
double ora_bessel_k_scaled(int n, double z) {
    double h = 0.05 * fmin(1.0, 1.0 / sqrt(z));
    double sum = 0.5;
    for (int k = 1; k < 2000000; k++) {
        double t = k * h;
        double sh = sinh(0.5 * t);
        double e = z * 2.0 * sh * sh;
        double f = exp(-e) * cosh(n * t);
        sum += f;
        if (e > n * t + 50.0 && f < 1e-20 * sum) break;
    }
    return h * sum;
}

void ora_thermal_coeffs(double ne, double Te, double B, double nu, double thB, double out[8]) {
    for (int i = 0; i < 8; i++) out[i] = 0.0;
    if (!(ne > 0.0) || !(Te > 0.0) || !(B > 0.0)) return;
    double s = sin(thB), c = cos(thB);
    double nuB = O_QE * B / (2.0 * O_PI * O_ME * O_C);
    /* rotativities (Shcherbakov 2008 fits as in Dexter 2016) */
    double X = Te * sqrt(sqrt(2.0) * fabs(s) * 1.0e3 * nuB / nu);
    double z = 1.0 / Te;
    double k0 = ora_bessel_k_scaled(0, z), k1 = ora_bessel_k_scaled(1, z), k2 = ora_bessel_k_scaled(2, z);
    double f = 2.011 * exp(-pow(X, 1.035) / 4.7) - cos(0.5 * X) * exp(-pow(X, 1.2) / 2.73) -
               0.011 * exp(-X / 47.2);
    if (X > 1.0)
        f += (0.011 * exp(-X / 47.2) - pow(2.0, -1.0 / 3.0) / pow(3.0, 23.0 / 6.0) * 1.0e4 * O_PI *
                                           pow(X, -8.0 / 3.0)) *
             0.5 * (1.0 + tanh(10.0 * log(X / 120.0)));
    double gX = 1.0 - 0.11 * log(1.0 + 0.035 * X);
    out[6] = ne * O_QE * O_QE * nuB * nuB * s * s / (O_ME * O_C * nu * nu * nu) * f * (k1 / k2 + 6.0 * Te);
    out[7] = 2.0 * ne * O_QE * O_QE * nuB * c / (O_ME * O_C * nu * nu) * (k0 / k2) * gX;
    /* emission and absorption (Dexter 2016 fits; Kirchhoff) */
    if (fabs(s) < 1e-12) return;
    double nuc = 1.5 * nuB * fabs(s) * Te * Te;
    double x = nu / nuc;
    double x13 = cbrt(x), x23 = x13 * x13;
    double ex = exp(-1.8899 * x13);
    double pre = ne * O_QE * O_QE * nu / (2.0 * sqrt(3.0) * O_C * Te * Te);
    double jI = pre * 2.5651 * (1.0 + 1.92 / x13 + 0.9977 / x23) * ex;
    double jQ = pre * 2.5651 * (1.0 + 0.93193 / x13 + 0.499873 / x23) * ex;
    double jV = 2.0 * ne * O_QE * O_QE * nu * (c / s) / (3.0 * sqrt(3.0) * O_C * Te * Te * Te) *
                (1.81348 / x + 3.42319 / x23 + 0.0292545 / sqrt(x) + 2.03773 / x13) * ex;
    /* emissivities this small carry no relative precision (they border the subnormal range)
     * and cannot reach any image: flush them, with their absorption, to zero */
    if (!(jI > 1e-250)) return;
    /* the fits are used outside their range (small theta_B, cold plasma); keep the emission
     * vector inside the light cone, |j_P| <= j_I, which the exact formulae always satisfy */
    if (jI > 0.0) {
        double rq = jQ / jI, rv = jV / jI;
        double p = sqrt(rq * rq + rv * rv);
        if (p > 1.0) {
            jQ /= p;
            jV /= p;
        }
    }
    double Bnu = 2.0 * O_H * nu * nu * nu / (O_C * O_C) / expm1(O_H * nu / (O_ME * O_C * O_C * Te));
    out[0] = jI;
    out[1] = jQ;
    out[2] = jV;
    out[3] = jI / Bnu;
    out[4] = jQ / Bnu;
    out[5] = jV / Bnu;
}

/* ============================ analytic substep ==========================================
 * dS/ds = J - M S with M = [[aI aQ aU aV],[aQ aI rV -rU],[aU -rV aI rQ],[aV rU -rQ aI]].
 * For constant coefficients the exact solution over ds is the exponential of the augmented
 * 5x5 system [[-M ds, J ds],[0, 0]] applied to (S0, 1). It is computed by scaling and
 * squaring a Taylor series to full double precision. */
static void mat5mul(const double A[5][5], const double B[5][5], double C[5][5]) {
    double T[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            double s = 0.0;
            for (int k = 0; k < 5; k++) s += A[i][k] * B[k][j];
            T[i][j] = s;
        }
    memcpy(C, T, sizeof(T));
}

static double norm1_5(const double A[5][5]) {
    double m = 0.0;
    for (int j = 0; j < 5; j++) {
        double s = 0.0;
        for (int i = 0; i < 5; i++) s += fabs(A[i][j]);
        if (s > m) m = s;
    }
    return m;
}

void ora_substep(const double cf[11], double ds, const double S0[4], double S1[4]) {
    double jI = cf[0], jQ = cf[1], jU = cf[2], jV = cf[3];
    double aI = cf[4], aQ = cf[5], aU = cf[6], aV = cf[7];
    double rQ = cf[8], rU = cf[9], rV = cf[10];
    double M[4][4] = {{aI, aQ, aU, aV}, {aQ, aI, rV, -rU}, {aU, -rV, aI, rQ}, {aV, rU, -rQ, aI}};
    /* the solution is linear in (S0, J): scale both by a power of two (exact) so that the
     * products formed below stay far from the subnormal range */
    double big = 0.0;
    double J[4] = {jI, jQ, jU, jV};
    for (int i = 0; i < 4; i++) big = fmax(big, fmax(fabs(J[i] * ds), fabs(S0[i])));
    int ex = 0;
    if (big > 0.0 && isfinite(big)) frexp(big, &ex);
    double S0s[4];
    for (int i = 0; i < 4; i++) {
        J[i] = ldexp(J[i], -ex);
        S0s[i] = ldexp(S0[i], -ex);
    }
    double G[5][5];
    memset(G, 0, sizeof(G));
    for (int i = 0; i < 4; i++) {
        for (int j = 0; j < 4; j++) G[i][j] = -M[i][j] * ds;
        G[i][4] = J[i] * ds;
    }
    double nrm = norm1_5(G);
    int sq = 0;
    while (nrm > 0.5 && sq < 2000) {
        nrm *= 0.5;
        sq++;
    }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) G[i][j] = ldexp(G[i][j], -sq);
    double E[5][5], T[5][5];
    memset(E, 0, sizeof(E));
    memset(T, 0, sizeof(T));
    for (int i = 0; i < 5; i++) E[i][i] = T[i][i] = 1.0;
    for (int k = 1; k <= 40; k++) {
        mat5mul(T, G, T);
        for (int i = 0; i < 5; i++)
            for (int j = 0; j < 5; j++) T[i][j] /= k;
        for (int i = 0; i < 5; i++)
            for (int j = 0; j < 5; j++) E[i][j] += T[i][j];
        if (norm1_5(T) < 1e-22 * norm1_5(E)) break;
    }
    for (int k = 0; k < sq; k++) mat5mul(E, E, E);
    for (int i = 0; i < 4; i++) {
        double s = E[i][4];
        for (int j = 0; j < 4; j++) s += E[i][j] * S0s[j];
        S1[i] = ldexp(s, ex);
    }
}

/* ============================ polarized transfer ========================================
 * Section 2.1: the polarization is the complex coherency matrix N^{mu nu} in the coordinate
 * frame, and the transfer runs along the saved geodesic toward the observer. Reading:
 *   - N is parallel transported between saved points, each index as a vector with the
 *     Heun propagator P of dv/dl' = T v, T^mu_be = Gamma^mu_{al be} K^al at both ends
 *     (l' is the forward parameter, K the saved past-directed tangent): N <- P N P^T,
 *     which keeps N positive semi-definite;
 *   - at each point the fluid tetrad is e_(0) = u, e_(3) along the photon direction,
 *     e_(2) along the projected field, and e_(1) from the Levi-Civita tensor so that
 *     (e1, e2, e3) is right handed; Stokes in that frame are I = N11 + N22,
 *     Q = N11 - N22, U = 2 Re N12, V = -2 Im N12;
 *   - the analytic constant-coefficient step uses the coefficients of the arrival point,
 *     with path length ds = (-k.u) dl L; N holds the invariant I/nu^3 in units of the
 *     observing frequency (I nu_obs^3/nu^3), so the fluid-frame Stokes vector is
 *     S = (nu/nu_obs)^3 (N-Stokes) and the camera reads I_nu directly;
 *   - N starts at zero at the far end of the path (no background light). */
typedef double complex cplx;

static void tmat(double a, double r, double th, const double K[4], double T[4][4]) {
    double G[64];
    ora_connection(a, r, th, G);
    for (int mu = 0; mu < 4; mu++)
        for (int be = 0; be < 4; be++) {
            double s = 0.0;
            for (int al = 0; al < 4; al++) s += G[mu * 16 + al * 4 + be] * K[al];
            T[mu][be] = s;
        }
}

/* Heun's method for the vector transport dv/dl' = T v from point n+1 (T1) to point n (T0):
 * v* = v + h T1 v, v_n = v + h/2 (T1 v + T0 v*), i.e. v_n = P v with
 * P = 1 + h/2 (T1 + T0) + h^2/2 T0 T1. */
static void heun_propagator(double h, double T1[4][4], double T0[4][4], double P[4][4]) {
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            double t01 = 0.0;
            for (int k = 0; k < 4; k++) t01 += T0[m][k] * T1[k][n];
            P[m][n] = (m == n ? 1.0 : 0.0) + 0.5 * h * (T1[m][n] + T0[m][n]) + 0.5 * h * h * t01;
        }
}

/* The propagator of the vector transport over the segment from saved point n+1 (s1) to point
 * n (sn). A segment that crossed the polar axis saved point n+1 reflected (theta -> -theta or
 * 2 pi - theta, phi + pi, K^theta -> -K^theta); it is taken back to the chart of point n, and
 * *flip tells the caller to change the sign of the theta components of what it transports. */
static void segment_propagator(double a, const double *sn, const double *s1, double P[4][4], int *flip) {
    double h = fabs(sn[8]);
    double th1 = s1[2], K1[4] = {s1[4], s1[5], s1[6], s1[7]};
    *flip = sn[8] < 0.0;
    if (*flip) {
        th1 = (sn[2] < 0.5 * O_PI) ? -th1 : 2.0 * O_PI - th1;
        K1[2] = -K1[2];
    }
    double T1[4][4], T0[4][4];
    tmat(a, s1[1], th1, K1, T1);
    tmat(a, sn[1], sn[2], sn + 4, T0);
    heun_propagator(h, T1, T0, P);
}

/* A real vector f given at the far end of a saved path (point M), transported to every saved
 * point in turn exactly as the transfer transports each index of N. out holds M + 1 rows of
 * 4 components, row n at point n (row M = f). For the pins of the transport. */
void ora_transport_vector(double a, const double *states, int M, const double f[4], double *out) {
    for (int i = 0; i < 4; i++) out[M * 4 + i] = f[i];
    for (int n = M - 1; n >= 0; n--) {
        const double *sn = states + n * 9, *s1 = states + (n + 1) * 9;
        double P[4][4], v[4];
        int flip;
        segment_propagator(a, sn, s1, P, &flip);
        for (int i = 0; i < 4; i++) v[i] = out[(n + 1) * 4 + i];
        if (flip) v[2] = -v[2];
        for (int i = 0; i < 4; i++) {
            double acc = 0.0;
            for (int k = 0; k < 4; k++) acc += P[i][k] * v[k];
            out[n * 4 + i] = acc;
        }
    }
}

/* Each index of N^{mu nu} is transported as a vector: N <- P N P^T. */
static void congruence(double P[4][4], cplx N[4][4]) {
    cplx X[4][4];
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            cplx s = 0.0;
            for (int k = 0; k < 4; k++) s += P[m][k] * N[k][n];
            X[m][n] = s;
        }
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            cplx s = 0.0;
            for (int k = 0; k < 4; k++) s += X[m][k] * P[n][k];
            N[m][n] = s;
        }
}

static void levi_e1(const double g[16], const double e0[4], const double e2[4], const double e3[4],
                    double e1[4]) {
    double gi[16], det;
    gj_invert(g, gi, &det);
    double sg = sqrt(-det);
    double low[4];
    static const int perm[24][4] = {
        {0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 1, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}, {0, 3, 2, 1},
        {1, 0, 2, 3}, {1, 0, 3, 2}, {1, 2, 0, 3}, {1, 2, 3, 0}, {1, 3, 0, 2}, {1, 3, 2, 0},
        {2, 0, 1, 3}, {2, 0, 3, 1}, {2, 1, 0, 3}, {2, 1, 3, 0}, {2, 3, 0, 1}, {2, 3, 1, 0},
        {3, 0, 1, 2}, {3, 0, 2, 1}, {3, 1, 0, 2}, {3, 1, 2, 0}, {3, 2, 0, 1}, {3, 2, 1, 0}};
    for (int i = 0; i < 4; i++) low[i] = 0.0;
    for (int p = 0; p < 24; p++) {
        const int *q = perm[p];
        int inv = 0;
        for (int i = 0; i < 4; i++)
            for (int j = i + 1; j < 4; j++)
                if (q[i] > q[j]) inv++;
        double sgn = (inv & 1) ? -1.0 : 1.0;
        low[q[0]] += -sgn * sg * e0[q[1]] * e2[q[2]] * e3[q[3]];
    }
    for (int m = 0; m < 4; m++) {
        e1[m] = 0.0;
        for (int n = 0; n < 4; n++) e1[m] += gi[m * 4 + n] * low[n];
    }
}

/* Fluid tetrad: e0 = u, e3 the unit projection of k normal to u (k = w (u + e3) for an
 * exactly null k, w = -k.u),
 * e2 along the part of b normal to (u, e3) (d_theta projected if b is along k), e1 from the
 * Levi-Civita tensor. Returns the angle between b and e3 in the fluid frame. */
static double fluid_tetrad(const double g[16], const double K[4], const double u[4], const double b[4],
                           double e0[4], double e1[4], double e2[4], double e3[4]) {
    double k[4] = {-K[0], -K[1], -K[2], -K[3]};
    double w = dot4(g, K, u);
    for (int i = 0; i < 4; i++) {
        e0[i] = u[i];
        e3[i] = k[i] - w * u[i];
    }
    double n3 = sqrt(dot4(g, e3, e3));
    for (int i = 0; i < 4; i++) e3[i] /= n3;
    double bb = dot4(g, b, b), be3 = dot4(g, b, e3);
    for (int i = 0; i < 4; i++) e2[i] = b[i] - be3 * e3[i];
    double n2 = sqrt(fmax(dot4(g, e2, e2), 0.0));
    /* the angle between b and e3: atan2 of the normal and parallel parts of b, which stays
     * accurate when b is nearly along the ray (acos of the cosine would not) */
    double thB = atan2(n2, be3);
    if (!(n2 > 1e-10 * sqrt(bb))) {
        double v[4] = {0, 0, 1, 0};
        double vu = dot4(g, v, u), ve = dot4(g, v, e3);
        for (int i = 0; i < 4; i++) e2[i] = v[i] + vu * u[i] - ve * e3[i];
        n2 = sqrt(dot4(g, e2, e2));
    }
    for (int i = 0; i < 4; i++) e2[i] /= n2;
    levi_e1(g, e0, e2, e3, e1);
    return thB;
}

double ora_fluid_tetrad(double a, const double x[4], const double K[4], const double u[4], const double b[4],
                        double e[16]) {
    double g[16];
    ora_metric_ks(a, x[1], x[2], g);
    return fluid_tetrad(g, K, u, b, e, e + 4, e + 8, e + 12);
}

static void stokes_from_N(const double g[16], const double e1[4], const double e2[4], cplx N[4][4],
                          double S[4]) {
    double l1[4], l2[4];
    lower4(g, e1, l1);
    lower4(g, e2, l2);
    cplx n11 = 0, n22 = 0, n12 = 0;
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            n11 += l1[m] * l1[n] * N[m][n];
            n22 += l2[m] * l2[n] * N[m][n];
            n12 += l1[m] * l2[n] * N[m][n];
        }
    S[0] = creal(n11 + n22);
    S[1] = creal(n11 - n22);
    S[2] = 2.0 * creal(n12);
    S[3] = -2.0 * cimag(n12);
}

static void N_from_stokes(const double e1[4], const double e2[4], const double S[4], cplx N[4][4]) {
    cplx n11 = 0.5 * (S[0] + S[1]), n22 = 0.5 * (S[0] - S[1]);
    cplx n12 = 0.5 * (S[2] - I * S[3]), n21 = 0.5 * (S[2] + I * S[3]);
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++)
            N[m][n] = n11 * e1[m] * e1[n] + n22 * e2[m] * e2[n] + n12 * e1[m] * e2[n] + n21 * e2[m] * e1[n];
}

/* The camera's reading of N for the pixel at image coordinates (px, py): Stokes on the image
 * basis x ~ e_phi, y ~ -e_theta of the camera frame, each projected normal to the ray. */
static void camera_stokes(const ora_camera *cam, double px, double py, cplx N[4][4], double S[4]) {
    double e[4][4], s[3];
    camera_frame(cam, e);
    sky_dir(cam, px, py, s);
    double xh[3] = {0.0 - s[2] * s[0], 0.0 - s[2] * s[1], 1.0 - s[2] * s[2]};
    double nx = sqrt(xh[0] * xh[0] + xh[1] * xh[1] + xh[2] * xh[2]);
    for (int i = 0; i < 3; i++) xh[i] /= nx;
    double yh[3] = {0.0 + s[1] * s[0], -1.0 + s[1] * s[1], 0.0 + s[1] * s[2]};
    double yx = yh[0] * xh[0] + yh[1] * xh[1] + yh[2] * xh[2];
    for (int i = 0; i < 3; i++) yh[i] -= yx * xh[i];
    double ny = sqrt(yh[0] * yh[0] + yh[1] * yh[1] + yh[2] * yh[2]);
    for (int i = 0; i < 3; i++) yh[i] /= ny;
    double X[4], Y[4];
    for (int mm = 0; mm < 4; mm++) {
        X[mm] = xh[0] * e[1][mm] + xh[1] * e[2][mm] + xh[2] * e[3][mm];
        Y[mm] = yh[0] * e[1][mm] + yh[1] * e[2][mm] + yh[2] * e[3][mm];
    }
    double g[16];
    ora_metric_ks(cam->a, cam->r_cam, cam->incl_deg * O_PI / 180.0, g);
    stokes_from_N(g, X, Y, N, S);
}

/* camera_stokes for a caller's N^{mu nu} (real and imaginary parts, row-major 4 x 4). For the
 * pins of the camera's Stokes basis. */
void ora_camera_stokes(const ora_camera *cam, double px, double py, const double Nre[16], const double Nim[16],
                       double S[4]) {
    cplx N[4][4];
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) N[m][n] = Nre[m * 4 + n] + I * Nim[m * 4 + n];
    camera_stokes(cam, px, py, N, S);
}

typedef struct {
    double st[4], minpol;
    double tau, phi; /* optical depth sum alpha_I ds and Faraday depth sum rho_V ds */
} pix_out;

static pix_out transfer(const ora_camera *cam, const ora_model *m, const double *st, int M, double px,
                        double py) {
    double a = cam->a;
    double nu_obs = cam->freq_hz;
    double L = O_G * cam->M_bh_g / (O_C * O_C);
    cplx N[4][4];
    memset(N, 0, sizeof(N));
    double minpol = 1.0, tau = 0.0, phi = 0.0;
    for (int n = M - 1; n >= 0; n--) {
        const double *sn = st + n * 9, *s1 = st + (n + 1) * 9;
        double h = fabs(sn[8]);
        /* transport N from point n+1 to point n */
        double P[4][4];
        int flip;
        segment_propagator(a, sn, s1, P, &flip);
        if (flip)
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++)
                    if ((i == 2) != (j == 2)) N[i][j] = -N[i][j];
        congruence(P, N);
        /* radiative step at point n */
        double pl[12];
        ora_plasma(cam, m, sn, pl);
        if (pl[3] == 0.0) continue;
        double g[16];
        ora_metric_ks(a, sn[1], sn[2], g);
        const double *K = sn + 4, *u = pl + 4, *b = pl + 8;
        double w = dot4(g, K, u); /* = -k.u = nu_fluid / nu_obs */
        double e0[4], e1[4], e2[4], e3[4];
        double thB = fluid_tetrad(g, K, u, b, e0, e1, e2, e3);
        double S[4];
        stokes_from_N(g, e1, e2, N, S);
        double nu = w * nu_obs;
        double c8[8];
        if (m->edf == ORA_EDF_KAPPA)
            ora_kappa_coeffs(pl[0], pl[1], pl[2], nu, thB, m->kappa, c8);
        else
            ora_thermal_coeffs(pl[0], pl[1], pl[2], nu, thB, c8);
        if (m->unpol_test)
            c8[1] = c8[2] = c8[4] = c8[5] = c8[6] = c8[7] = 0.0;
        double cf[11] = {c8[0], c8[1], 0.0, c8[2], c8[3], c8[4], 0.0, c8[5], c8[6], 0.0, c8[7]};
        double ds = w * h * L;
        /* depths: the exponents of the isotropic absorption and the Faraday rotation that
         * this segment's constant-coefficient step applies, summed along the ray */
        tau += c8[3] * ds;
        phi += c8[7] * ds;
        double w3 = w * w * w;
        double Sf[4], Sf1[4];
        for (int i = 0; i < 4; i++) Sf[i] = S[i] * w3;
        ora_substep(cf, ds, Sf, Sf1);
        for (int i = 0; i < 4; i++) S[i] = Sf1[i] / w3;
        if (Sf1[0] > 0.0) {
            double q = Sf1[1] / Sf1[0], uu = Sf1[2] / Sf1[0], v = Sf1[3] / Sf1[0];
            double mp = 1.0 - sqrt(q * q + uu * uu + v * v);
            if (mp < minpol) minpol = mp;
        }
        N_from_stokes(e1, e2, S, N);
    }
    double S[4];
    camera_stokes(cam, px, py, N, S);
    pix_out o = {{S[0], S[1], S[2], S[3]}, minpol, tau, phi};
    return o;
}

/* Unpolarized transfer (Stokes I only, emissivity j_I and absorptivity a_I): I/nu^3 is
 * invariant along the ray, so each segment multiplies it by e^-tau and adds the segment's
 * emission (j_I ds / w^3) (1 - e^-tau) / tau, at the arrival point, as in the polarized case. */
static double transfer_unpol(const ora_camera *cam, const ora_model *m, const double *st, int M) {
    double a = cam->a, nu_obs = cam->freq_hz, L = O_G * cam->M_bh_g / (O_C * O_C);
    double Iv = 0.0;
    for (int n = M - 1; n >= 0; n--) {
        const double *sn = st + n * 9;
        double h = fabs(sn[8]);
        double pl[12];
        ora_plasma(cam, m, sn, pl);
        if (pl[3] == 0.0) continue;
        double g[16];
        ora_metric_ks(a, sn[1], sn[2], g);
        const double *K = sn + 4, *u = pl + 4, *b = pl + 8;
        double w = dot4(g, K, u);
        double e0[4], e1[4], e2[4], e3[4];
        double thB = fluid_tetrad(g, K, u, b, e0, e1, e2, e3);
        double c8[8];
        ora_thermal_coeffs(pl[0], pl[1], pl[2], w * nu_obs, thB, c8);
        double ds = w * h * L, tau = c8[3] * ds;
        double f = tau > 1e-8 ? -expm1(-tau) / tau : 1.0 - 0.5 * tau;
        Iv = Iv * exp(-tau) + c8[0] * ds / (w * w * w) * f;
    }
    return Iv;
}

int ora_render_unpol(const ora_camera *cam, const ora_model *m, int npix, const int *ix, const int *iy,
                     double *Iout, int nthreads) {
    int err = 0;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
    {
        int maxst = cam->nmax + 2;
        double *st = (double *)malloc((size_t)maxst * 9 * sizeof(double));
        if (!st) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = -1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 2)
#endif
            for (int p = 0; p < npix; p++) {
                double px, py;
                int stat;
                pixel_xy(cam, ix[p], iy[p], 0, &px, &py);
                int M = trace(cam, px, py, maxst, st, &stat);
                Iout[p] = transfer_unpol(cam, m, st, M);
            }
            free(st);
        }
    }
    return err;
}

int ora_render_pixels(const ora_camera *cam, const ora_model *m, int npix, const int *ix, const int *iy,
                      int pert, double *iquv, int *nsteps, int *status, double *minpol, double *depth,
                      int nthreads) {
    int err = 0;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
    {
        int maxst = cam->nmax + 2;
        double *st = (double *)malloc((size_t)maxst * 9 * sizeof(double));
        if (!st) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = -1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 2)
#endif
            for (int p = 0; p < npix; p++) {
                double px, py;
                int stat;
                pixel_xy(cam, ix[p], iy[p], pert, &px, &py);
                int M = trace(cam, px, py, maxst, st, &stat);
                pix_out o = transfer(cam, m, st, M, px, py);
                for (int k = 0; k < 4; k++) iquv[4 * p + k] = o.st[k];
                if (nsteps) nsteps[p] = M;
                if (status) status[p] = stat;
                if (minpol) minpol[p] = o.minpol;
                if (depth) {
                    depth[2 * p] = o.tau;
                    depth[2 * p + 1] = o.phi;
                }
            }
            free(st);
        }
    }
    return err;
}

/* Total flux F = sum I dOmega x 1e23 Jy with dOmega = (FOV L / (nx D))^2; net linear and
 * circular polarization fractions from the Stokes sums. */
void ora_image_stats(const ora_camera *cam, const double *iquv, long npix, double *flux_jy, double *lp,
                     double *cp) {
    long double sI = 0, sQ = 0, sU = 0, sV = 0;
    for (long p = 0; p < npix; p++) {
        sI += iquv[4 * p];
        sQ += iquv[4 * p + 1];
        sU += iquv[4 * p + 2];
        sV += iquv[4 * p + 3];
    }
    double L = O_G * cam->M_bh_g / (O_C * O_C);
    double pix = cam->fov_M * L / (cam->nx * cam->dist_cm);
    *flux_jy = (double)sI * pix * pix * 1e23;
    *lp = sqrt((double)(sQ * sQ + sU * sU)) / (double)sI;
    *cp = (double)sV / (double)sI;
}
