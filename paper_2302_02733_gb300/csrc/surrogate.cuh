// The surrogate's variables. Inputs (per plasma point): f = (ln(nu / nu_c), theta_B,
// ln Theta_e, kappa) with nu_c = (3/2) nu_B sin(theta_B) Theta_e^2, theta_B folded into
// (0, pi/2] (the circular terms change sign with cos theta_B, the rest are even). Outputs: the
// logarithms of the 8 coefficients over their prefactors,
//   j_I, j_Q = P_j e^y0, e^y1,               P_j = n e^2 nu / (2 sqrt3 c Theta^2),
//   j_V = P_j (4 / (3 Theta)) |cot| e^y2,     (the thermal fits' circular prefactor),
//   a_I, a_Q = P_a e^y3, e^y4,               P_a = n e^2 / (4 sqrt3 m c nu Theta^3),
//   a_V = P_a |cot| e^y5,
//   r_Q = P_rQ f(X) e^y6,                    P_rQ = n e^2 nu_B^2 sin^2 / (m c nu^3),
//   r_V = P_rV g(X) e^y7,                    P_rV = 2 n e^2 nu_B |cos| / (m c nu^2),
// with f, g Shcherbakov's corrections at X as for the thermal fits, and the circular terms
// carrying the sign of cos theta_B. In these variables every target is a smooth function of f
// only (the prefactors absorb n_e, B and nu), which the network learns in standardised form.
#pragma once
#include "kappa.cuh"

namespace prt {

// Cubic polynomial basis in the normalised inputs (all monomials of degree <= 3 in 4
// variables, 35 terms): the baseline that carries the targets' large trends, so the network
// learns a residual of small range.
constexpr int kSurBasis = 35;
__device__ __forceinline__ void sur_basis(const float x[4], float phi[kSurBasis]) {
    int m = 0;
    phi[m++] = 1.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) phi[m++] = x[i];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = i; j < 4; j++) phi[m++] = x[i] * x[j];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = i; j < 4; j++)
#pragma unroll
            for (int k = j; k < 4; k++) phi[m++] = x[i] * x[j] * x[k];
}

struct SurPref {
    double Pj, PjV, Pa, PaV, PrQ, PrV, sgn;
};

__device__ __forceinline__ SurPref sur_prefactors(double ne, double Te, double B, double nu, double th) {
    SurPref p;
    double s = sin(th), c = cos(th), as = fabs(s), ac = fabs(c);
    double nuB = kQe * B / (2.0 * kPi * kMe * kC);
    double e2 = kQe * kQe;
    double cot = as > 0.0 ? ac / as : 0.0;
    p.Pj = ne * e2 * nu / (2.0 * 1.7320508075688772 * kC * Te * Te);
    p.PjV = p.Pj * (4.0 / (3.0 * Te)) * cot;
    p.Pa = ne * e2 / (4.0 * 1.7320508075688772 * kMe * kC * nu * Te * Te * Te);
    p.PaV = p.Pa * cot;
    double X = Te * sqrt(1.4142135623730951 * as * 1.0e3 * nuB / nu);
    p.PrQ = ne * e2 * nuB * nuB * s * s / (kMe * kC * nu * nu * nu) * shcherbakov_f(X);
    p.PrV = 2.0 * ne * e2 * nuB * ac / (kMe * kC * nu * nu) * (1.0 - 0.11 * log1p(0.035 * X));
    p.sgn = c < 0.0 ? -1.0 : 1.0;
    return p;
}

// surrogate input features of a plasma point
__device__ __forceinline__ void sur_features(double Te, double B, double nu, double th, double kappa, float f[4]) {
    double tf = th > 0.5 * kPi ? kPi - th : th;
    double nuB = kQe * B / (2.0 * kPi * kMe * kC);
    double nuc = 1.5 * nuB * sin(tf) * Te * Te;
    f[0] = (float)log(nu / nuc);
    f[1] = (float)tf;
    f[2] = (float)log(Te);
    f[3] = (float)kappa;
}

// coefficients (quadrature order jI jQ jV aI aQ aV rQ rV) -> targets y; false if not all finite
__device__ __forceinline__ bool sur_reduce(const SurPref &p, const double c[8], float y[8]) {
    double q[8] = {c[0] / p.Pj, c[1] / p.Pj, p.sgn * c[2] / p.PjV, c[3] / p.Pa,
                   c[4] / p.Pa, p.sgn * c[5] / p.PaV, c[6] / p.PrQ, p.sgn * c[7] / p.PrV};
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        double l = log(q[k]);
        ok &= isfinite(l);
        y[k] = (float)l;
    }
    return ok;
}

// targets -> coefficients, with the light-cone clamps of the quadrature
__device__ __forceinline__ void sur_expand(const SurPref &p, const float y[8], double c[8]) {
    c[0] = p.Pj * exp((double)y[0]);
    c[1] = p.Pj * exp((double)y[1]);
    c[2] = p.sgn * p.PjV * exp((double)y[2]);
    c[3] = p.Pa * exp((double)y[3]);
    c[4] = p.Pa * exp((double)y[4]);
    c[5] = p.sgn * p.PaV * exp((double)y[5]);
    c[6] = p.PrQ * exp((double)y[6]);
    c[7] = p.sgn * p.PrV * exp((double)y[7]);
    double pj = sqrt(c[1] * c[1] + c[2] * c[2]);
    if (pj > c[0] && pj > 0.0) {
        c[1] *= c[0] / pj;
        c[2] *= c[0] / pj;
    }
    double pa = sqrt(c[4] * c[4] + c[5] * c[5]);
    if (pa > c[3] && pa > 0.0) {
        c[4] *= c[3] / pa;
        c[5] *= c[3] / pa;
    }
}

}  // namespace prt
