// Synchrotron coefficients of kappa-distributed (or Maxwell-Juttner) electrons by quadrature
// over the distribution: the nonthermal models of the paper's Section 2.1, integrated
// numerically as its outlook (Section 4) proposes. This is the accurate path: it makes the
// surrogate's training set, is the reference the surrogate is checked against, and stands in
// for it outside its box.
//
// Definitions, in an isotropic distribution N(g) (g the Lorentz factor, p = sqrt(g^2 - 1)):
//   kappa:  N = n C g p (1 + (g - 1)/(kappa w))^-(kappa+1), w = (kappa - 3) Theta / kappa;
//   j_I, j_Q, j_V = A int N [F, G, (4/3) cot(theta) H / g](X / g^2) dg,
//     A = sqrt(3) e^3 B sin(theta) / (4 pi m c^2), X = nu / ((3/2) nu_B sin(theta)),
//     F = x int_x K_5/3, G = x K_2/3, H = x K_1/3 + int_x K_1/3 (ultrarelativistic kernels);
//   a_S = -(1 / (2 nu^2 m)) int k_S g^2 d/dg (N / g^2) dg for each kernel k_S;
//   r_V = (2 e^2 nu_B cos / (m c nu^2)) g(X_T) int N asinh(p) / (g p) dg,
//   r_Q = (e^2 nu_B^2 sin^2 / (m c nu^3)) f(X_T) int N (2 g - 1/g) dg,
// with the Shcherbakov corrections f, g at X_T as for the thermal fits, and (j_Q, j_V),
// (a_Q, a_V) kept inside the light cone. For Maxwell-Juttner electrons the rotativity averages
// are exactly K0/K2 and K1/K2 + 6 Theta.
//
// Numerics (device), two grades:
//  - tabulated (kExact false; the FP32 render, the surrogate's training set and fallback,
//    rt_kappa_coeffs): F, G, H from tables of their logarithms on 4096 nodes in ln x
//    (x in [1e-12, 740]) with cubic interpolation, built once per context by the trapezoid
//    rule on their cosh-integral representations; the distribution integrals over s = ln p
//    by Gauss-Legendre, 8 nodes per panel of width 1/2 (1/8 for Maxwell-Juttner electrons);
//    about 1e-8 relative;
//  - exact (kExact true; the FP64 render): F, G, H evaluated at every node by the trapezoid
//    rule (synch_kernels_exact, about 1e-14 relative) and 8 nodes per panel of width 1/8 for
//    every distribution, so that the quadrature error is far below the FP64 form's 1e-9.
#pragma once
#include "rt_common.cuh"

namespace prt {

constexpr int kSynTab = 4096;
constexpr double kSynLo = -27.631021115928547;  // ln 1e-12
constexpr double kSynHi = 6.606650186198215;    // ln 740

// KappaTables (rt_common.cuh): lnk [3][kSynTab] = ln F, ln G, ln H at ln x = kSynLo + i h, and
// the 8-point Gauss-Legendre nodes and weights.

// F, G, H at x (0 beyond the table's upper end).
__device__ __forceinline__ void synch_kernels_tab(const KappaTables &T, double x, double k[3]) {
    if (!(x > 0.0) || x >= 740.0) {
        k[0] = k[1] = k[2] = 0.0;
        return;
    }
    const double h = (kSynHi - kSynLo) / (kSynTab - 1);
    double u = (log(x) - kSynLo) / h;
    if (u < 1.0) {  // below the table the kernels follow their small-x power laws: extrapolate ln k linearly
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const double *L = T.lnk + j * kSynTab;
            k[j] = exp(L[0] + u * (L[1] - L[0]));
        }
        return;
    }
    int i = (int)u;
    if (i > kSynTab - 3) i = kSynTab - 3;
    double t = u - i;
    // Catmull-Rom cubic through nodes i-1 .. i+2
    double c0 = t * ((2.0 - t) * t - 1.0) * 0.5, c1 = (t * t * (3.0 * t - 5.0) + 2.0) * 0.5;
    double c2 = t * ((4.0 - 3.0 * t) * t + 1.0) * 0.5, c3 = (t - 1.0) * t * t * 0.5;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const double *L = T.lnk + j * kSynTab + i - 1;
        k[j] = exp(c0 * L[0] + c1 * L[1] + c2 * L[2] + c3 * L[3]);
    }
}

// F, G, H at x by the trapezoid rule on int_0^inf e^{-x cosh t} c(t) dt with
// c = cosh(5t/3)/cosh t, cosh(2t/3), cosh(t/3) and cosh(t/3)/cosh t, at step 0.25 min(1, x^-1/2)
// (the integrand's peak at t = 0 is x^-1/2 wide; the rule converges geometrically for these
// analytic integrands, to about 1e-14 relative here), every cosh from u = e^{t/3}.
__device__ __forceinline__ void synch_kernels_exact(double x, double k[3]) {
    k[0] = k[1] = k[2] = 0.0;
    if (!(x > 0.0) || x >= 740.0) return;
    const double h = 0.25 * fmin(1.0, rsqrt(x));
    double e0 = 0.5 * exp(-x);  // t = 0, half weight: every c(0) = 1
    double a = e0, b = e0, c = e0, d = e0;
    for (int i = 1; i < 4096; i++) {
        double u = exp(i * h * (1.0 / 3.0)), iu = 1.0 / u;
        double u2 = u * u, iu2 = iu * iu, u3 = u2 * u, iu3 = iu2 * iu;
        double ch = 0.5 * (u3 + iu3);
        double arg = x * ch;
        if (arg > 745.0) break;
        double e = exp(-arg), ich = 1.0 / ch;
        double c13 = 0.5 * (u + iu);
        double ta = e * 0.5 * (u3 * u2 + iu3 * iu2) * ich;
        a += ta;
        b += e * 0.5 * (u2 + iu2);
        c += e * c13;
        d += e * c13 * ich;
        if (i > 4 && ta < 1e-19 * a) break;
    }
    k[0] = x * h * a;
    k[1] = x * h * b;
    k[2] = x * h * c + h * d;
}

struct Edf {
    bool thermal;
    double theta, kappa, kw, norm;
    // N/n and g^2 d/dg (N/g^2)/n at momentum p
    __device__ __forceinline__ void eval(double p, double g, double &N, double &D) const {
        if (thermal) {
            double e = exp(-(g - 1.0) / theta) * norm;
            N = g * p * e;
            D = e * (1.0 / p - g * p / theta);
        } else {
            double q = exp(-(kappa + 1.0) * log1p((g - 1.0) / kw)) * norm;
            N = g * p * q;
            D = q * (1.0 / p - g * p * (kappa + 1.0) / (kw + g - 1.0));
        }
    }
};

__device__ __forceinline__ double shcherbakov_f(double X) {
    double f = 2.011 * exp(-pow(X, 1.035) / 4.7) - cos(0.5 * X) * exp(-pow(X, 1.2) / 2.73) - 0.011 * exp(-X / 47.2);
    if (X > 1.0)
        f += (0.011 * exp(-X / 47.2) - 369.6934286909082 * pow(X, -8.0 / 3.0))  // 2^-1/3 3^-23/6 1e4 pi
             * 0.5 *
             (1.0 + tanh(10.0 * log(X / 120.0)));
    return f;
}

// e^z K_2(z) by the trapezoid rule on int_0^inf exp(-z (cosh t - 1)) cosh(2t) dt.
__device__ __forceinline__ double bessel_k2_scaled(double z) {
    double h = 0.05 * fmin(1.0, 1.0 / sqrt(z)), sum = 0.5;
    for (int k = 1; k < 200000; k++) {
        double t = k * h, sh = sinh(0.5 * t), e = 2.0 * z * sh * sh;
        double f = exp(-e) * cosh(2.0 * t);
        sum += f;
        if (e > 2.0 * t + 50.0 && f < 1e-20 * sum) break;
    }
    return h * sum;
}

// out: jI jQ jV aI aQ aV rQ rV (cgs). kappa <= 0 selects Maxwell-Juttner electrons. kExact:
// the exact grade (kernels at every node, 8 panels per unit of s), else the tabulated one.
template <bool kExact = false>
__device__ __forceinline__ void kappa_coeffs_quad(const KappaTables &T, double ne, double Te, double B, double nu,
                                                  double thB, double kappa, double out[8]) {
#pragma unroll
    for (int i = 0; i < 8; i++) out[i] = 0.0;
    if (!(ne > 0.0) || !(Te > 0.0) || !(B > 0.0) || !(nu > 0.0)) return;
    if (kappa > 0.0 && !(kappa > 3.0)) return;
    Edf d;
    double s_lo = log(1e-4), s_hi;
    if (kappa <= 0.0) {
        d.thermal = true;
        d.theta = Te;
        d.kappa = 0.0;
        d.kw = 1.0;
        d.norm = 1.0 / (Te * bessel_k2_scaled(1.0 / Te));
        double ghi = 1.0 + 800.0 * Te;
        s_hi = 0.5 * log(ghi * ghi - 1.0);
    } else {
        d.thermal = false;
        d.theta = Te;
        d.kappa = kappa;
        d.kw = (kappa - 3.0) * Te;
        d.norm = 1.0;
        s_hi = log((1.0 + d.kw) * 10.0) + fmin(45.0 / (kappa - 2.34), 600.0);
    }
    // panels per unit of s: the kappa integrands are smooth power laws; far above nu_c the
    // Maxwell-Juttner integrand is a peak about 0.1 wide in s and needs four times more
    const int kPanels = (kExact || d.thermal) ? 8 : 2;
    // normalisation (kappa) and rotativity averages over the whole momentum range
    double nacc = 0.0, rv = 0.0, rq = 0.0;
    {
        int np = (int)ceil((s_hi - s_lo) * kPanels);
        double hw = 0.5 * (s_hi - s_lo) / np;
        for (int k = 0; k < np; k++) {
            double c = s_lo + (2 * k + 1) * hw;
            for (int i = 0; i < 8; i++) {
                double p = exp(c + hw * T.glx[i]);
                double g = sqrt(1.0 + p * p);
                double N, D;
                d.eval(p, g, N, D);
                double dg = hw * T.glw[i] * p * p / g;
                nacc += dg * N;
                rv += dg * N * asinh(p) / (g * p);
                rq += dg * N * (2.0 * g - 1.0 / g);
            }
        }
    }
    if (!d.thermal) {  // the kappa normalisation C = 1 / int N dg
        d.norm = 1.0 / nacc;
        rv *= d.norm;
        rq *= d.norm;
    }
    double s = sin(thB), c = cos(thB);
    double nuB = kQe * B / (2.0 * kPi * kMe * kC);
    double Xr = Te * sqrt(1.4142135623730951 * fabs(s) * 1.0e3 * nuB / nu);
    out[6] = ne * kQe * kQe * nuB * nuB * s * s / (kMe * kC * nu * nu * nu) * shcherbakov_f(Xr) * rq;
    out[7] = 2.0 * ne * kQe * kQe * nuB * c / (kMe * kC * nu * nu) * (1.0 - 0.11 * log1p(0.035 * Xr)) * rv;
    if (fabs(s) < 1e-12) return;
    double X = nu / (1.5 * nuB * fabs(s));
    double g0 = sqrt(fmax(X / 740.0, 1.0));
    double se = g0 > 1.0 + 1e-8 ? 0.5 * log(g0 * g0 - 1.0) : s_lo;
    if (se >= s_hi) return;
    double e[6] = {0, 0, 0, 0, 0, 0};
    int np = (int)ceil((s_hi - se) * kPanels);
    double hw = 0.5 * (s_hi - se) / np;
    for (int k = 0; k < np; k++) {
        double cc = se + (2 * k + 1) * hw;
        for (int i = 0; i < 8; i++) {
            double p = exp(cc + hw * T.glx[i]);
            double g = sqrt(1.0 + p * p);
            double N, D, kk[3];
            d.eval(p, g, N, D);
            if (kExact)
                synch_kernels_exact(X / (g * g), kk);
            else
                synch_kernels_tab(T, X / (g * g), kk);
            double dg = hw * T.glw[i] * p * p / g;
            double ig = 1.0 / g;
            e[0] += dg * N * kk[0];
            e[1] += dg * N * kk[1];
            e[2] += dg * N * kk[2] * ig;
            e[3] += dg * D * kk[0];
            e[4] += dg * D * kk[1];
            e[5] += dg * D * kk[2] * ig;
        }
    }
    double A = 1.7320508075688772 * kQe * kQe * kQe * B * fabs(s) / (4.0 * kPi * kMe * kC * kC);
    double cot = c / s;
    double jI = ne * A * e[0], jQ = ne * A * e[1], jV = ne * A * (4.0 / 3.0) * cot * e[2];
    double ab = -ne * A / (2.0 * nu * nu * kMe);
    double aI = ab * e[3], aQ = ab * e[4], aV = ab * (4.0 / 3.0) * cot * e[5];
    if (!(jI > 1e-250)) return;
    double pj = sqrt((jQ / jI) * (jQ / jI) + (jV / jI) * (jV / jI));
    if (pj > 1.0) {
        jQ /= pj;
        jV /= pj;
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

}  // namespace prt
