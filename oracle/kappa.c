/*
 * Synchrotron coefficients of an isotropic electron distribution by direct quadrature: the
 * kappa distribution of the paper's nonthermal models (Section 2.1 names the thermal and the
 * nonthermal electron distribution functions; its outlook in Section 4 proposes numerical
 * integration over the distribution), and the Maxwell-Juttner distribution for the pins.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Plain FP64, slow, no tables.
 *
 * Readings (the paper gives no formulas; each is listed in the design notes):
 *  - kappa distribution: N(g) = n C g sqrt(g^2-1) (1 + (g-1)/(kappa w))^-(kappa+1) with
 *    w = (kappa-3) Theta_e / kappa, C by quadrature.
 *  - emission in the ultrarelativistic synchrotron approximation: with X = nu / nu_s,
 *    nu_s = (3/2) nu_B sin(theta), x = X / g^2 and A = sqrt(3) e^3 B sin(theta) / (4 pi m c^2):
 *      j_I = A int N F(x) dg,  j_Q = A int N G(x) dg,  j_V = A (4/3) cot(theta) int N H(x) / g dg,
 *      F(x) = x int_x^inf K_5/3,  G(x) = x K_2/3(x),  H(x) = x K_1/3(x) + int_x^inf K_1/3.
 *    F and G are the single-electron synchrotron functions (Rybicki & Lightman 6.31-6.32); the
 *    circular kernel H and its factor 4/3 are fixed by the thermal limit: with the
 *    Maxwell-Juttner distribution these integrals are exactly those that the thermal fits
 *    approximate. All three are the leading order in 1/gamma of the exact sum over cyclotron
 *    harmonics (the Schott series), which the tests evaluate for both distributions.
 *  - absorption for every Stokes component from the emission kernel k_S (j_S = int N k_S):
 *      a_S = -(1 / (2 nu^2 m)) int k_S g^2 d/dg (N / g^2) dg     (Rybicki & Lightman 6.50),
 *    which reduces to Kirchhoff's law (Rayleigh-Jeans) for Maxwell-Juttner electrons.
 *  - rotativities: the thermal form (Shcherbakov's corrections f(X), g(X) at the same X as
 *    the thermal fits) with the Bessel-function ratios replaced by distribution averages whose
 *    kernels reproduce them exactly for Maxwell-Juttner electrons:
 *      r_V = (2 e^2 nu_B cos / (m c nu^2)) g(X) int N asinh(p) / (g p) dg        (n K0/K2),
 *      r_Q = (e^2 nu_B^2 sin^2 / (m c nu^3)) f(X) int N (2 g - 1/g) dg           (n (K1/K2 + 6 Theta)),
 *    p = sqrt(g^2 - 1), so that kappa -> infinity gives the thermal rotativities.
 *  - as for the thermal fits, (j_Q, j_V) and (a_Q, a_V) are kept inside the light cone.
 *
 * Quadrature: every distribution integral is taken over s = ln p by composite Gauss-Legendre
 * (8 nodes per panel of width 1/8); the kernels F, G, H by the trapezoid rule in t of their
 * representations int_0^inf exp(-x cosh t) cosh(a t) [/cosh t] dt, step min(1, x^-1/2) / 10.
 */
#include <math.h>
#include <string.h>

#define K_C 2.99792458e10
#define K_ME 9.1093837015e-28
#define K_QE 4.80320471257e-10
#define K_PI 3.14159265358979323846

double ora_bessel_k_scaled(int n, double z);

/* F, G, H at x > 0 */
void ora_synch_kernels(double x, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    if (!(x > 0.0) || x > 740.0) return;
    /* the integrand peaks at t = 0 with width x^-1/2: the step follows it (geometric convergence
     * of the trapezoid rule for these analytic integrands, below 1e-15 relative) */
    const double h = 0.1 * fmin(1.0, 1.0 / sqrt(x));
    double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
    for (int k = 0; k < 100000; k++) {
        double t = k * h, wgt = k == 0 ? 0.5 : 1.0;
        double ch = cosh(t);
        double arg = x * ch;
        if (arg > 745.0) break;
        double e = exp(-arg) * wgt;
        double c53 = cosh(5.0 * t / 3.0), c23 = cosh(2.0 * t / 3.0), c13 = cosh(t / 3.0);
        s1 += e * c53 / ch;
        s2 += e * c23;
        s3 += e * c13;
        s4 += e * c13 / ch;
        if (k > 10 && e * c53 < 1e-19 * s1) break;
    }
    out[0] = x * h * s1;
    out[1] = x * h * s2;
    out[2] = x * h * s3 + h * s4;
}

/* Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the Chebyshev guess) */
static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; i++) {
        double z = cos(K_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; j++) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            pp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

typedef struct {
    int thermal;
    double theta, kappa, w, norm; /* norm: C (kappa) or 1/(Theta e^{1/Theta} K2(1/Theta)) */
} edf_t;

/* N/n and g^2 d/dg (N/g^2) / n at momentum p (g = sqrt(1 + p^2)) */
static void edf_eval(const edf_t *d, double p, double *N, double *D) {
    double g = sqrt(1.0 + p * p);
    if (d->thermal) {
        double e = exp(-(g - 1.0) / d->theta) * d->norm;
        *N = g * p * e;
        *D = e * (1.0 / p - g * p / d->theta);
    } else {
        double kw = d->kappa * d->w;
        double q = pow(1.0 + (g - 1.0) / kw, -(d->kappa + 1.0)) * d->norm;
        *N = g * p * q;
        *D = q * (1.0 / p - g * p * (d->kappa + 1.0) / (kw + g - 1.0));
    }
}

#define NGL 8

/* int over s = ln p in [s0, s1] of f(p) dp = f(p) p ds, composite Gauss-Legendre */
typedef void (*integrand_t)(double p, void *ctx, double *acc, double wgt);

static void integrate_s(double s0, double s1, integrand_t f, void *ctx, double *acc) {
    double glx[NGL], glw[NGL];
    gauss_legendre(NGL, glx, glw);
    int panels = (int)ceil((s1 - s0) * 8.0);
    if (panels < 1) panels = 1;
    double hw = 0.5 * (s1 - s0) / panels;
    for (int k = 0; k < panels; k++) {
        double c = s0 + (2 * k + 1) * hw;
        for (int i = 0; i < NGL; i++) {
            double s = c + hw * glx[i];
            double p = exp(s);
            f(p, ctx, acc, hw * glw[i] * p);
        }
    }
}

static void norm_integrand(double p, void *ctx, double *acc, double wgt) {
    edf_t *d = (edf_t *)ctx;
    double N, D;
    edf_eval(d, p, &N, &D);
    /* N dg = N p / g dp */
    acc[0] += wgt * N * p / sqrt(1.0 + p * p);
}

typedef struct {
    const edf_t *d;
    double X; /* nu / nu_s */
} coef_ctx;

static double conv_corr(double X) {
    double f = 2.011 * exp(-pow(X, 1.035) / 4.7) - cos(0.5 * X) * exp(-pow(X, 1.2) / 2.73) -
               0.011 * exp(-X / 47.2);
    if (X > 1.0)
        f += (0.011 * exp(-X / 47.2) -
              pow(2.0, -1.0 / 3.0) / pow(3.0, 23.0 / 6.0) * 1.0e4 * K_PI * pow(X, -8.0 / 3.0)) *
             0.5 * (1.0 + tanh(10.0 * log(X / 120.0)));
    return f;
}

/* acc: int N F, N G, N H/g, D F, D G, D H/g (emission and absorption integrals, per dg) */
static void emis_integrand(double p, void *ctx, double *acc, double wgt) {
    coef_ctx *c = (coef_ctx *)ctx;
    double g = sqrt(1.0 + p * p);
    double N, D, k[3];
    edf_eval(c->d, p, &N, &D);
    ora_synch_kernels(c->X / (g * g), k);
    double dg = wgt * p / g;
    acc[0] += dg * N * k[0];
    acc[1] += dg * N * k[1];
    acc[2] += dg * N * k[2] / g;
    acc[3] += dg * D * k[0];
    acc[4] += dg * D * k[1];
    acc[5] += dg * D * k[2] / g;
}

/* acc: int N asinh(p)/(g p), int N (2g - 1/g) */
static void rot_integrand(double p, void *ctx, double *acc, double wgt) {
    coef_ctx *c = (coef_ctx *)ctx;
    double g = sqrt(1.0 + p * p);
    double N, D;
    edf_eval(c->d, p, &N, &D);
    double dg = wgt * p / g;
    acc[0] += dg * N * asinh(p) / (g * p);
    acc[1] += dg * N * (2.0 * g - 1.0 / g);
}

/* kappa > 0: kappa distribution (kappa > 3); kappa <= 0: Maxwell-Juttner. out as the thermal
 * coefficients: jI jQ jV aI aQ aV rQ rV. */
void ora_kappa_coeffs(double ne, double Te, double B, double nu, double thB, double kappa, double out[8]) {
    for (int i = 0; i < 8; i++) out[i] = 0.0;
    if (!(ne > 0.0) || !(Te > 0.0) || !(B > 0.0) || !(nu > 0.0)) return;
    if (kappa > 0.0 && !(kappa > 3.0)) return;
    edf_t d;
    memset(&d, 0, sizeof(d));
    double s_lo_all = log(1e-4), s_hi;
    if (kappa <= 0.0) {
        d.thermal = 1;
        d.theta = Te;
        d.norm = 1.0 / (Te * ora_bessel_k_scaled(2, 1.0 / Te));
        double ghi = 1.0 + 800.0 * Te;
        s_hi = log(sqrt(ghi * ghi - 1.0));
    } else {
        d.kappa = kappa;
        d.w = (kappa - 3.0) * Te / kappa;
        d.norm = 1.0;
        /* the slowest tail (emission) falls like g^(7/3 - kappa) per unit ln g */
        double knee = 1.0 + kappa * d.w;
        s_hi = log(knee * 10.0) + fmin(45.0 / (kappa - 2.34), 600.0);
        double acc[1] = {0.0};
        integrate_s(s_lo_all, s_hi, norm_integrand, &d, acc);
        d.norm = 1.0 / acc[0];
    }
    double s = sin(thB), c = cos(thB);
    double nuB = K_QE * B / (2.0 * K_PI * K_ME * K_C);
    coef_ctx cx = {&d, 0.0};
    /* rotativities */
    double racc[2] = {0.0, 0.0};
    integrate_s(s_lo_all, s_hi, rot_integrand, &cx, racc);
    double Xr = Te * sqrt(sqrt(2.0) * fabs(s) * 1.0e3 * nuB / nu);
    double gX = 1.0 - 0.11 * log(1.0 + 0.035 * Xr);
    out[6] = ne * K_QE * K_QE * nuB * nuB * s * s / (K_ME * K_C * nu * nu * nu) * conv_corr(Xr) * racc[1];
    out[7] = 2.0 * ne * K_QE * K_QE * nuB * c / (K_ME * K_C * nu * nu) * gX * racc[0];
    if (fabs(s) < 1e-12) return;
    /* emission and absorption: x = X/g^2 above 740 contributes nothing, so start at g^2 = X/740 */
    cx.X = nu / (1.5 * nuB * fabs(s));
    double g0 = sqrt(fmax(cx.X / 740.0, 1.0));
    double s_lo = g0 > 1.0 + 1e-8 ? log(sqrt(g0 * g0 - 1.0)) : s_lo_all;
    if (s_lo >= s_hi) return;
    double eacc[6] = {0, 0, 0, 0, 0, 0};
    integrate_s(s_lo, s_hi, emis_integrand, &cx, eacc);
    double A = sqrt(3.0) * K_QE * K_QE * K_QE * B * fabs(s) / (4.0 * K_PI * K_ME * K_C * K_C);
    double cot = c / s;
    double jI = ne * A * eacc[0], jQ = ne * A * eacc[1], jV = ne * A * (4.0 / 3.0) * cot * eacc[2];
    double ab = -ne * A / (2.0 * nu * nu * K_ME);
    double aI = ab * eacc[3], aQ = ab * eacc[4], aV = ab * (4.0 / 3.0) * cot * eacc[5];
    if (!(jI > 1e-250)) return;
    double p = sqrt((jQ / jI) * (jQ / jI) + (jV / jI) * (jV / jI));
    if (p > 1.0) {
        jQ /= p;
        jV /= p;
    }
    if (aI > 0.0) {
        double pa = sqrt((aQ / aI) * (aQ / aI) + (aV / aI) * (aV / aI));
        if (pa > 1.0) {
            aQ /= pa;
            aV /= pa;
        }
    }
    out[0] = jI;
    out[1] = jQ;
    out[2] = jV;
    out[3] = aI;
    out[4] = aQ;
    out[5] = aV;
}
