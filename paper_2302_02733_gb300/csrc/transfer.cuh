// Forward polarized transfer along the saved geodesic (the paper's Section 2.1: the covariant,
// fully polarized transfer equations are integrated toward the observer; plasma quantities are
// interpolated or computed at every point; the coherency matrix lives in the coordinate frame).
//
// Representation. The coherency tensor after each radiative step is rank two in the screen
// of the fluid frame: N^{mu nu} = sum_ab n^{ab} E_a^mu E_b^nu with the 2x2 coherency n built
// from the Stokes vector S and the screen legs (E_1, E_2). Parallel transport of N by the
// Heun propagator P (each index as a vector) therefore equals transporting E_1 and E_2 by
// Heun and keeping S. Projecting onto the next fluid screen (e_1', e_2') is the 2x2 congruence
// n' = C n C^T with C_{a'a} = e_a' . E_a, which keeps n positive semi-definite (I >= |P|).
//
// Templated on the transfer precision R: double for the FP64 form, float for the mixed form
// (the path itself is always the FP64 geodesic).
#pragma once
#include "camera.cuh"
#include "ffloat.cuh"
#include "rt_kernels.cuh"

namespace prt {

// ------------------------------------------------------------------------------------------
// precision-dispatched math
template <typename R>
struct Mth;
template <>
struct Mth<double> {
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double expm1_(double x) { return expm1(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
    static __device__ __forceinline__ double log2_(double x) { return log2(x); }
    static __device__ __forceinline__ double exp2_(double x) { return exp2(x); }
    static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
    static __device__ __forceinline__ double cbrt_(double x) { return cbrt(x); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double tanh_(double x) { return tanh(x); }
    static __device__ __forceinline__ void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
    static __device__ __forceinline__ double sin_(double x) { return sin(x); }
    static __device__ __forceinline__ double cos_(double x) { return cos(x); }
    static __device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
    static __device__ __forceinline__ double sinh_(double x) { return sinh(x); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
    static __device__ __forceinline__ double fmod_(double x, double y) { return fmod(x, y); }
    static constexpr double jflush = 1e-250;  // emissivity below this carries no precision
    static constexpr int taylor_max = 24;
    static constexpr double taylor_tol = 1e-17;
    static constexpr double degen_D = 1e-9, degen_tp = 1e-3;
};
template <>
struct Mth<float> {
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
    static __device__ __forceinline__ float log2_(float x) { return log2f(x); }
    static __device__ __forceinline__ float exp2_(float x) { return exp2f(x); }
    static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
    static __device__ __forceinline__ float cbrt_(float x) { return cbrtf(x); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float tanh_(float x) { return tanhf(x); }
    static __device__ __forceinline__ void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
    static __device__ __forceinline__ float sin_(float x) { return sinf(x); }
    static __device__ __forceinline__ float cos_(float x) { return cosf(x); }
    static __device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
    static __device__ __forceinline__ float sinh_(float x) { return sinhf(x); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
    static __device__ __forceinline__ float fmod_(float x, float y) { return fmodf(x, y); }
    static constexpr float jflush = 1e-35f;
    static constexpr int taylor_max = 14;
    static constexpr float taylor_tol = 3e-8f;
    static constexpr float degen_D = 1e-4f, degen_tp = 1e-2f;
};

// ------------------------------------------------------------------------------------------
// e^z K_n(z), n = 0, 1, 2.
//   z < 2: ascending series (Abramowitz & Stegun 9.6.11, 9.6.13),
//     K0 = -(ln(z/2) + gamma) I0 + sum H_k t^k/(k!)^2,
//     K1 = 1/z + (ln(z/2) + gamma) I1 - (z/4) sum (H_k + H_{k+1}) t^k/(k!(k+1)!),  t = z^2/4;
//   z >= 2: with u = sqrt(2z) sinh(s/2) in K_n = int_0^inf e^{-z cosh s} cosh(ns) ds,
//     e^z K_n(z) = sqrt(2/z) int_0^inf e^{-u^2} c_n(u) / sqrt(1 + u^2/(2z)) du,
//     c_0 = 1, c_1 = 1 + u^2/z, c_2 = 2 c_1^2 - 1, by the trapezoid rule on fixed nodes u_k = k h
//     (the integrand is analytic in |Im u| < sqrt(2z), so the rule converges geometrically).
//   K2 = K0 + (2/z) K1 for the series branch.
template <typename R>
struct BesselCfg;
template <>
struct BesselCfg<double> {
    static constexpr int nser = 14, nq = 27;
    static constexpr double h = 0.25;
};
template <>
struct BesselCfg<float> {
    static constexpr int nser = 8, nq = 10;
    static constexpr float h = 0.5f;
};

// gw[k] = exp(-(k h)^2), halved at k = 0 (trapezoid end weight); kept in shared memory.
template <typename R>
__device__ __forceinline__ void bessel_k012_scaled(R z, const R *gw, R &k0, R &k1, R &k2) {
    typedef Mth<R> F;
    typedef BesselCfg<R> B;
    R iz = R(1) / z;
    if (z < R(2)) {
        R hz = R(0.5) * z, t = hz * hz;
        R lg = F::log_(hz) + R(0.57721566490153286061);
        R i0 = 0, s0 = 0, i1s = 0, s1 = 0, term0 = 1, term1 = 1, H = 0;
#pragma unroll
        for (int k = 0; k < B::nser; k++) {
            R ik1 = R(1) / R(k + 1);
            i0 += term0;
            s0 += H * term0;
            i1s += term1;
            s1 += (R(2) * H + ik1) * term1;
            H += ik1;
            term0 *= t * ik1 * ik1;
            term1 *= t * ik1 / R(k + 2);
        }
        R e = F::exp_(z);
        R K0 = -lg * i0 + s0;
        R K1 = iz + lg * (hz * i1s) - R(0.25) * z * s1;
        k0 = K0 * e;
        k1 = K1 * e;
        k2 = k0 + R(2) * iz * k1;
    } else {
        R i2z = R(0.5) * iz;
        R a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int k = 0; k < B::nq; k++) {
            R u = R(k) * B::h, u2 = u * u;
            R w = gw[k];
            R rr = w * F::rsqrt_(R(1) + u2 * i2z);
            R c1 = R(1) + u2 * iz;
            a0 += rr;
            a1 += rr * c1;
            a2 += rr * (R(2) * c1 * c1 - R(1));
        }
        R sc = F::sqrt_(R(2) * iz) * B::h;
        k0 = sc * a0;
        k1 = sc * a1;
        k2 = sc * a2;
    }
}

// ------------------------------------------------------------------------------------------
// Shcherbakov's (2008) correction of rho_Q,
//   f(X) = 2.011 e^{-X^1.035/4.7} - cos(X/2) e^{-X^1.2/2.73} - 0.011 e^{-X/47.2}
//          + [X > 1] (0.011 e^{-X/47.2} - 2^{-1/3} 3^{-23/6} 1e4 pi X^{-8/3}) (1 + tanh(10 ln(X/120)))/2,
// with the three powers from one log2 X, and (1 + tanh y)/2 = 1 - 1/(e^{2y} + 1) where
// e^{2y} = (X/120)^20 (which may overflow to infinity: the form stays exact there).
template <typename R>
__device__ __forceinline__ R shcherbakov_fX(R X) {
    typedef Mth<R> F;
    const R lX = F::log2_(X);  // -inf at X = 0, where the powers are 0
    const R eX = F::exp_(-X / R(47.2));
    R f = R(2.011) * F::exp_(-F::exp2_(R(1.035) * lX) / R(4.7)) -
          F::cos_(R(0.5) * X) * F::exp_(-F::exp2_(R(1.2) * lX) / R(2.73)) - R(0.011) * eX;
    if (X > R(1)) {
        const R t = F::exp2_(R(20) * (lX - R(6.9068905956085187)));  // (X/120)^20; log2 120
        f += (R(0.011) * eX - R(369.6934286909082) * F::exp2_(R(-8.0 / 3.0) * lX)) * (R(1) - R(1) / (t + R(1)));
    }
    return f;
}

// ------------------------------------------------------------------------------------------
// Thermal synchrotron coefficients in the fluid frame (cgs).
// Emission: the Dexter (2016) fits with nu_c = (3/2) nu_B sin(th) Theta^2, x = nu/nu_c:
//   j_I = n e^2 nu/(2 sqrt3 c Theta^2) 2.5651 (1 + 1.92 x^-1/3 + 0.9977 x^-2/3) e^{-1.8899 x^1/3},
//   j_Q = same with (1 + 0.93193 x^-1/3 + 0.499873 x^-2/3),
//   j_V = 2 n e^2 nu cot(th)/(3 sqrt3 c Theta^3) (1.81348/x + 3.42319 x^-2/3 + 0.0292545 x^-1/2
//         + 2.03773 x^-1/3) e^{-1.8899 x^1/3};
// absorption from Kirchhoff's law a_S = j_S / B_nu(T_e); rotativities from the Shcherbakov
// (2008) fits with X = Theta sqrt(sqrt2 sin(th) 1e3 nu_B/nu):
//   rho_V = 2 n e^2 nu_B cos(th)/(m c nu^2) K0/K2 (1 - 0.11 ln(1 + 0.035 X)),
//   rho_Q = n e^2 nu_B^2 sin^2(th)/(m c nu^3) f_m(X) (K1/K2 + 6 Theta).
// Stokes Q is positive across the projected field, so j_U = a_U = rho_U = 0. Emissivities
// below a flush level are zeroed with their absorption, and (j_Q, j_V) are scaled back inside
// the light cone |j_P| <= j_I where the fits are used out of range.
// out: jI jQ jV aI aQ aV rQ rV
template <typename R>
__device__ __forceinline__ void thermal_coeffs(R ne, R Te, R B, R nu, R sth, R cth, const R *gw, R out[8]) {
    typedef Mth<R> F;
#pragma unroll
    for (int i = 0; i < 8; i++) out[i] = R(0);
    if (!(ne > R(0)) || !(Te > R(0)) || !(B > R(0))) return;
    const R cB = R(kQe / (2.0 * kPi * kMe * kC));        // nu_B / B
    const R cQ2 = R(kQe * kQe / (kMe * kC));             // e^2 / (m c)
    const R cJ = R(kQe * kQe / (2.0 * 1.7320508075688772 * kC));
    const R cJV = R(2.0 * kQe * kQe / (3.0 * 1.7320508075688772 * kC));
    const R cT = R(kH / (kMe * kC * kC));                // h nu / (m c^2 Theta) = cT nu / Theta
    const R c2h = R(2.0 * kH);
    const R ic = R(1.0 / kC);
    R nuB = cB * B;
    R rb = nuB / nu;
    R X = Te * F::sqrt_(R(1.4142135623730951) * sth * R(1e3) * rb);
    R k0, k1, k2;
    if (Te > R(1e-12)) {
        bessel_k012_scaled<R>(R(1) / Te, gw, k0, k1, k2);
    } else {  // K_n(z)/K_2(z) -> 1 as z -> infinity
        k0 = k1 = k2 = R(1);
    }
    R f = shcherbakov_fX(X);
    R gX = R(1) - R(0.11) * F::log1p_(R(0.035) * X);
    out[6] = cQ2 * ne * rb * rb / nu * sth * sth * f * (k1 / k2 + R(6) * Te);
    out[7] = R(2) * cQ2 * ne * rb / nu * cth * (k0 / k2) * gX;
    if (sth < R(1e-12)) return;
    R nuc = R(1.5) * nuB * sth * Te * Te;
    R x = nu / nuc;
    R x13 = F::cbrt_(x), ix13 = R(1) / x13, ix23 = ix13 * ix13;
    R ex = F::exp_(R(-1.8899) * x13);
    R pre = cJ * ne * nu / (Te * Te);
    R jI = pre * R(2.5651) * (R(1) + R(1.92) * ix13 + R(0.9977) * ix23) * ex;
    if (!(jI > F::jflush)) return;
    R jQ = pre * R(2.5651) * (R(1) + R(0.93193) * ix13 + R(0.499873) * ix23) * ex;
    R jV = cJV * ne * nu * (cth / sth) / (Te * Te * Te) *
           (R(1.81348) / x + R(3.42319) * ix23 + R(0.0292545) * F::rsqrt_(x) + R(2.03773) * ix13) * ex;
    R rq = jQ / jI, rv = jV / jI;
    R pj = F::sqrt_(rq * rq + rv * rv);
    if (pj > R(1)) {
        jQ /= pj;
        jV /= pj;
    }
    R nuic = nu * ic;
    R Bnu = c2h * nu * nuic * nuic / F::expm1_(cT * nu / Te);
    R iB = R(1) / Bnu;
    out[0] = jI;
    out[1] = jQ;
    out[2] = jV;
    out[3] = jI * iB;
    out[4] = jQ * iB;
    out[5] = jV * iB;
}

// j_I and a_I alone (the unpolarized transfer): the same fit and Kirchhoff's law as
// thermal_coeffs, without the rotativities (and so without the Bessel functions).
template <typename R>
__device__ __forceinline__ void thermal_jI_aI(R ne, R Te, R B, R nu, R sth, R &jI, R &aI) {
    typedef Mth<R> F;
    jI = aI = R(0);
    if (!(ne > R(0)) || !(Te > R(0)) || !(B > R(0)) || sth < R(1e-12)) return;
    const R cB = R(kQe / (2.0 * kPi * kMe * kC));
    const R cJ = R(kQe * kQe / (2.0 * 1.7320508075688772 * kC));
    const R cT = R(kH / (kMe * kC * kC));
    const R c2h = R(2.0 * kH);
    const R ic = R(1.0 / kC);
    R nuB = cB * B;
    R nuc = R(1.5) * nuB * sth * Te * Te;
    R x = nu / nuc;
    R x13 = F::cbrt_(x), ix13 = R(1) / x13, ix23 = ix13 * ix13;
    R ex = F::exp_(R(-1.8899) * x13);
    R pre = cJ * ne * nu / (Te * Te);
    R j = pre * R(2.5651) * (R(1) + R(1.92) * ix13 + R(0.9977) * ix23) * ex;
    if (!(j > F::jflush)) return;
    R nuic = nu * ic;
    R Bnu = c2h * nu * nuic * nuic / F::expm1_(cT * nu / Te);
    jI = j;
    aI = j * (R(1) / Bnu);
}

// ------------------------------------------------------------------------------------------
// Exact constant-coefficient step of dS/ds = J - M S over ds (M as in the transfer matrix
// with j_U = a_U = r_U = 0): S <- exp(-M ds) S + (int_0^ds exp(-M v) dv) J.
// Small steps (||M ds|| <= 1/2): Taylor series of the augmented system applied to the vector.
// Otherwise M ds = tau 1 + B with B a Lorentz generator whose eigenvalues are +-P, +-iQ:
//   exp(-B) = C0 + C1 B + C2 B^2 + C3 B^3,
//   C0 = (Q^2 cosh P + P^2 cos Q)/D, C2 = (cosh P - cos Q)/D,
//   C1 = -(P^2 sinc Q + Q^2 sinhc P)/D, C3 = (sinc Q - sinhc P)/D,   D = P^2 + Q^2,
// and int_0^1 e^{-(tau + B) v} dv = f0 + f1 B + f2 B^2 + f3 B^3 with the same combinations of
//   Ec = int e^{-tau v} cosh(Pv), Es = int e^{-tau v} sinh(Pv)/P,
//   EC = int e^{-tau v} cos(Qv),  ES = int e^{-tau v} sin(Qv)/Q   (v from 0 to 1),
// each evaluated in a form free of cancellation (exponentials folded with e^{-tau}).
// Error-free transformation of a sum (Knuth's TwoSum): hi + d = s + err exactly; s becomes the
// value and err joins the compensation lo. Six additions, no assumption on |hi| vs |d|.
template <typename R>
__device__ __forceinline__ void two_sum_add(R &hi, R &lo, R d) {
    R s = hi + d;
    R bb = s - hi;
    R err = (hi - (s - bb)) + (d - bb);
    hi = s;
    lo += err;
}

// Kahan's compensated summation: s + (-c) carries the running sum.
template <typename R>
__device__ __forceinline__ void kahan_add(R &s, R &c, R x) {
    R y = x - c;
    R t = s + y;
    c = (t - s) - y;
    s = t;
}

template <typename R>
__device__ __forceinline__ R phi1(R x) {  // (1 - e^-x)/x
    typedef Mth<R> F;
    if (x == R(0)) return R(1);
    return -F::expm1_(-x) / x;
}
template <typename R>
__device__ __forceinline__ R gamma2(R t) {  // 1 - (1 + t) e^-t
    typedef Mth<R> F;
    if (t < R(0.5)) {
        R s = 0, p = t * t, f = R(0.5);
#pragma unroll
        for (int k = 2; k < 18; k++) {
            s += f * p;
            p *= -t;
            f *= R(k) / (R(k - 1) * R(k + 1));  // (k)/((k+1)!) from (k-1)/k!
        }
        return s;
    }
    return R(1) - (R(1) + t) * F::exp_(-t);
}

// E_s(tau, P) = int_0^1 e^{-tau v} sinh(P v)/P dv for tau < 1/2 (then P <= tau < 1/2):
// sum_k P^2k/(2k+1)! m_{2k+1}(tau) with m_n(tau) = int_0^1 v^n e^{-tau v} dv, m_13 from its
// series sum_j (-tau)^j/(j! (14 + j)) and the stable downward recurrence
// m_{n-1} = (tau m_n + e^{-tau})/n.
template <typename R>
__device__ __forceinline__ R es_small(R tau, R P, R e) {
    const int nj = sizeof(R) == 8 ? 18 : 10;
    R term = R(1), m = R(0);
#pragma unroll
    for (int j = 0; j < nj; j++) {
        m += term / R(14 + j);
        term *= -tau / R(j + 1);
    }
    R mm[14];
    mm[13] = m;
#pragma unroll
    for (int n = 13; n >= 1; n--) mm[n - 1] = (tau * mm[n] + e) / R(n);
    R P2 = P * P, c = R(1), acc = R(0);
#pragma unroll
    for (int k = 0; k < 7; k++) {
        acc += c * mm[2 * k + 1];
        c *= P2 / (R(2 * k + 2) * R(2 * k + 3));
    }
    return acc;
}

template <typename R>
__device__ __forceinline__ void bmul(R aQ, R aV, R rQ, R rV, const R v[4], R o[4]) {
    o[0] = aQ * v[1] + aV * v[3];
    o[1] = aQ * v[0] + rV * v[2];
    o[2] = -rV * v[1] + rQ * v[3];
    o[3] = aV * v[0] - rQ * v[2];
}

// Increment of one constant-coefficient step by the Taylor series of the exponential applied
// to the vector: acc = sum_k t_k, t_1 = J - M S, t_k = -M t_{k-1} / k.
template <typename R>
__device__ __forceinline__ void taylor_inc(R tau, R aQ, R aV, R rQ, R rV, const R J[4], const R S[4], R acc[4]) {
    typedef Mth<R> F;
    R t[4], b[4];
    bmul(aQ, aV, rQ, rV, S, b);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        t[i] = J[i] - tau * S[i] - b[i];
        acc[i] = t[i];
    }
    for (int k = 2; k <= F::taylor_max; k++) {
        bmul(aQ, aV, rQ, rV, t, b);
        R ik = R(1) / R(k);
        R m = 0, sz = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            t[i] = -(tau * t[i] + b[i]) * ik;
            acc[i] += t[i];
            m = fmax(m, fabs(t[i]));
            sz = fmax(sz, fabs(acc[i]) + fabs(S[i]));
        }
        if (m <= F::taylor_tol * sz) break;
    }
}

// One exact constant-coefficient step of dS/ds = J js - M S over ds on the compensated value
// S + Slo (js scales the emissivities: 1/w^3 for the invariant form). Thin steps (the common
// case) form the increment by the Taylor series and add it without rounding loss; thick steps
// fold Slo in and apply the closed form.
template <typename R>
__device__ void substep(const R cf[8], R ds, R js, R S[4], R Slo[4]) {
    typedef Mth<R> F;
    R tau = cf[3] * ds, aQ = cf[4] * ds, aV = cf[5] * ds, rQ = cf[6] * ds, rV = cf[7] * ds;
    R jds = js * ds;
    R J[4] = {cf[0] * jds, cf[1] * jds, R(0), cf[2] * jds};
    R nrm = tau + fabs(aQ) + fabs(aV) + fabs(rQ) + fabs(rV);
    if (!(nrm > R(0.5))) {
        R acc[4];
        taylor_inc(tau, aQ, aV, rQ, rV, J, S, acc);
#pragma unroll
        for (int i = 0; i < 4; i++) two_sum_add(S[i], Slo[i], acc[i]);
        return;
    }
    R a2 = aQ * aQ + aV * aV, r2 = rQ * rQ + rV * rV, ar = aQ * rQ + aV * rV;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        S[i] += Slo[i];
        Slo[i] = R(0);
    }
    if (a2 + r2 == R(0)) {  // isotropic absorption and emission only
        R e = F::exp_(-tau), p = phi1(tau);
#pragma unroll
        for (int i = 0; i < 4; i++) S[i] = e * S[i] + p * J[i];
        return;
    }
    // eigenvalue magnitudes: P^2 - Q^2 = a^2 - r^2, P^2 Q^2 = (a.r)^2; the larger root from the
    // sum, the smaller from the product (no cancellation when one of a, r dominates)
    R hd = R(0.5) * (a2 - r2);
    R disc = F::sqrt_(hd * hd + ar * ar);
    R P2r, Q2r;
    if (hd >= R(0)) {
        P2r = disc + hd;
        Q2r = P2r > R(0) ? ar * ar / P2r : R(0);
    } else {
        Q2r = disc - hd;
        P2r = Q2r > R(0) ? ar * ar / Q2r : R(0);
    }
    R P = F::sqrt_(P2r), Q = F::sqrt_(Q2r);
    R D = R(2) * disc;
    if (D < F::degen_D * (a2 + r2) || (tau >= R(0.5) && (tau - P) < F::degen_tp * tau)) {
        // near-degenerate generator or maximal dichroism: sub-stepped Taylor series
        int m = (int)fmin(ceil(nrm / R(0.5)), R(8192));
        R inv = R(1) / R(m);
        R Js[4] = {J[0] * inv, J[1] * inv, J[2] * inv, J[3] * inv};
        for (int k = 0; k < m; k++) {
            R acc[4];
            taylor_inc(tau * inv, aQ * inv, aV * inv, rQ * inv, rV * inv, Js, S, acc);
#pragma unroll
            for (int i = 0; i < 4; i++) two_sum_add(S[i], Slo[i], acc[i]);
        }
        return;
    }
    R iD = R(1) / D, P2 = P * P, Q2 = Q * Q;
    R e = F::exp_(-tau);
    R sQ, cQ;
    F::sincos_(Q, &sQ, &cQ);
    R scQ = (Q < R(1e-4)) ? R(1) - Q2 / R(6) : sQ / Q;
    R omscQ;  // 1 - sinc Q
    if (Q < R(0.1)) {
        R q2 = Q2;
        omscQ = q2 * (R(1) / R(6) - q2 * (R(1) / R(120) - q2 * (R(1) / R(5040) - q2 / R(362880))));
    } else {
        omscQ = R(1) - scQ;
    }
    R sh2 = F::sin_(R(0.5) * Q);
    sh2 = R(2) * sh2 * sh2;  // 1 - cos Q
    R ech, esh, esh_m_e, ech_m_e;  // e^-tau cosh P, e^-tau sinh(P)/P, and minus e^-tau
    if (P < R(1)) {
        R p2 = P2, shcm1;
        if (P < R(0.1))
            shcm1 = p2 * (R(1) / R(6) + p2 * (R(1) / R(120) + p2 * (R(1) / R(5040) + p2 / R(362880))));
        else
            shcm1 = F::sinh_(P) / P - R(1);
        R hs = F::sinh_(R(0.5) * P);
        R chm1 = R(2) * hs * hs;  // cosh P - 1
        ech = e * (R(1) + chm1);
        esh = e * (R(1) + shcm1);
        esh_m_e = e * shcm1;
        ech_m_e = e * chm1;
    } else {
        R em = F::exp_(-(tau - P)), ep = F::exp_(-(tau + P));
        ech = R(0.5) * (em + ep);
        esh = R(0.5) * (em - ep) / P;
        esh_m_e = esh - e;
        ech_m_e = ech - e;
    }
    // homogeneous part
    R eC0 = (Q2 * ech + P2 * e * cQ) * iD;
    R eC2 = (ech - e * cQ) * iD;
    R eC1 = -(P2 * e * scQ + Q2 * esh) * iD;
    R eC3 = (e * scQ - esh) * iD;
    // emission integrals
    R g2 = gamma2(tau);
    R Ec = R(0.5) * (phi1(tau - P) + phi1(tau + P));
    R Es = tau < R(0.5) ? es_small(tau, P, e) : (g2 - tau * esh_m_e - ech_m_e) / ((tau - P) * (tau + P));
    R tq = tau * tau + Q2;
    R Aa = -F::expm1_(-tau) + e * sh2;
    R EC = (Aa * tau + e * sQ * Q) / tq;
    R ES = (g2 + e * sh2 + tau * e * omscQ) / tq;
    R f0 = (Q2 * Ec + P2 * EC) * iD;
    R f2 = (Ec - EC) * iD;
    R f1 = -(P2 * ES + Q2 * Es) * iD;
    R f3 = (ES - Es) * iD;
    R b1[4], b2[4], b3[4], j1[4], j2[4], j3[4];
    bmul(aQ, aV, rQ, rV, S, b1);
    bmul(aQ, aV, rQ, rV, b1, b2);
    bmul(aQ, aV, rQ, rV, b2, b3);
    bmul(aQ, aV, rQ, rV, J, j1);
    bmul(aQ, aV, rQ, rV, j1, j2);
    bmul(aQ, aV, rQ, rV, j2, j3);
#pragma unroll
    for (int i = 0; i < 4; i++)
        S[i] = eC0 * S[i] + eC1 * b1[i] + eC2 * b2[i] + eC3 * b3[i] + f0 * J[i] + f1 * j1[i] + f2 * j2[i] +
               f3 * j3[i];
}

// ------------------------------------------------------------------------------------------
// Plasma models. out: valid flag; ne, Theta_e, B [G]; u^mu, b^mu (direction) in KS.
template <typename R>
struct Plasma {
    bool valid;
    R ne, Te, B;
    R u[4], b[4];
};

template <typename R>
__device__ __forceinline__ void adaf_plasma(const AdafModel &p, R a, const KS<R> &m, R r, Plasma<R> &o) {
    typedef Mth<R> F;
    o.valid = false;
    if (r > pick<R>(p.r_out, p.f_r_out)) return;
    R ir = R(1) / r;
    R r15 = ir * F::rsqrt_(r);
    o.ne = pick<R>(p.n0, p.f_n0) * r15;
    o.Te = pick<R>(p.te0, p.f_te0) * ir;
    o.B = pick<R>(p.b0, p.f_b0) * F::sqrt_(r15 * ir);
    // Boyer-Lindquist inverse metric pieces
    R a2 = a * a, s2 = m.s2;
    R del = r * r - R(2) * r + a2;
    R rr2 = r * r + a2;
    R A = rr2 * rr2 - a2 * del * s2;
    R isd = R(1) / (m.sig * del);
    R gtt = -A * isd, gtp = -R(2) * a * r * isd, gpp = (del - a2 * s2) * isd / s2, grr = del * m.isig;
    // -1 - g^tt = (A - Sigma Delta)/(Sigma Delta) = 2r (r^2 + a^2)/(Sigma Delta): no cancellation
    R m1_gtt = R(2) * r * rr2 * isd;
    R rk = fmax(r, pick<R>(p.r_isco, p.f_r_isco));
    R sq = F::sqrt_(rk);
    R lK = (rk * rk - R(2) * a * sq + a2) / (rk * sq - R(2) * sq + a);
    R l = pick<R>(p.f_kep, p.f_f_kep) * lK * s2;
    R rhs = m1_gtt + R(2) * gtp * l - gpp * l * l;
    R ur_low = -F::sqrt_(fmax(rhs, R(0)) / grr);
    R u[4];
    u[1] = grr * ur_low;
    u[0] = -gtt + gtp * l + R(2) * r / del * u[1];
    u[2] = R(0);
    u[3] = -gtp + gpp * l + a / del * u[1];
    R nrm = R(1) / F::sqrt_(-m.dot(u, u));
#pragma unroll
    for (int i = 0; i < 4; i++) o.u[i] = u[i] * nrm;
    R ul[4];
    m.lower(o.u, ul);
    R bt = ul[1] + ul[3] * ir;
    R iut = R(1) / o.u[0];
    o.b[0] = bt;
    o.b[1] = (R(1) + bt * o.u[1]) * iut;
    o.b[2] = bt * o.u[2] * iut;
    o.b[3] = (ir + bt * o.u[3]) * iut;
    o.valid = true;
}

// FMKS polar angle in offset form: mu = theta - pi/2 as a function of y = X2 - 1/2, at blend
// weight w = exp(s (X1_in - X1)); also d theta / d X2 and theta_j - theta_g. With x2 = 1/2 + y,
// sin(2 pi x2) = -sin(2 pi y) and cos(2 pi x2) = -cos(2 pi y), so every term is small near the
// equator and an FP32 evaluation keeps the relative precision of mu there.
template <typename R>
__device__ __forceinline__ R fmks_mu(const GridModel &g, R w, R y, R *dth2, R *thj_m_thg) {
    typedef Mth<R> F;
    R s2p, c2p;
    F::sincos_(R(2 * kPi) * y, &s2p, &c2p);
    R omh = R(1) - pick<R>(g.hslope, g.f_hslope);
    R mug = R(kPi) * y - R(0.5) * omh * s2p;  // theta_g - pi/2
    R dthg = R(kPi) * (R(1) - omh * c2p);
    R yp = R(2) * y;                          // 2 X2 - 1
    R yx = yp / pick<R>(g.poly_xt, g.f_poly_xt);
    R ya = F::pow_(fabs(yx), pick<R>(g.poly_alpha, g.f_poly_alpha));
    R N = pick<R>(g.poly_norm, g.f_poly_norm);
    R muj = N * yp * (R(1) + ya / pick<R>(g.poly_alpha + 1.0, g.f_poly_alpha1));  // theta_j - pi/2
    R dthj = R(2) * N * (R(1) + ya);
    if (dth2) *dth2 = dthg + w * (dthj - dthg);
    if (thj_m_thg) *thj_m_thg = muj - mug;
    return mug + w * (muj - mug);
}

// FMKS polar angle theta(X2) at blend weight w, and d/dX2.
template <typename R>
__device__ __forceinline__ R fmks_theta_w(const GridModel &g, R w, R x2, R *dth2, R *thj_m_thg) {
    return R(0.5 * kPi) + fmks_mu(g, w, x2 - R(0.5), dth2, thj_m_thg);
}

// y = X2 - 1/2 of the point at polar angle th (mu = th - pi/2, formed before rounding to R):
// a table guess in (w, theta), then Newton on mu.
template <typename R>
__device__ __forceinline__ R fmks_y(const GridModel &g, R w, R th, R mu) {
    R fw = w * R(kX2TabW - 1);
    R ft = th * R((kX2TabT - 1) / kPi);
    int iw, it;
    R tw, tt;
    if constexpr (sizeof(R) == 4) {  // fw in [0, 63], ft in [0, 1023]: no conversion instructions
        iw = min(max(floor_small(fw), 0), kX2TabW - 2);
        it = min(max(floor_small(ft), 0), kX2TabT - 2);
        tw = fw - i2f_small(iw);
        tt = ft - i2f_small(it);
    } else {
        iw = min(max((int)fw, 0), kX2TabW - 2);
        it = min(max((int)ft, 0), kX2TabT - 2);
        tw = fw - R(iw);
        tt = ft - R(it);
    }
    R x00, x01, x10, x11;
    if (sizeof(R) == 8) {
        const double *T = g.x2_table;
        x00 = R(T[iw * kX2TabT + it]), x01 = R(T[iw * kX2TabT + it + 1]);
        x10 = R(T[(iw + 1) * kX2TabT + it]), x11 = R(T[(iw + 1) * kX2TabT + it + 1]);
    } else {
        const float *T = g.x2_table_f;
        x00 = R(T[iw * kX2TabT + it]), x01 = R(T[iw * kX2TabT + it + 1]);
        x10 = R(T[(iw + 1) * kX2TabT + it]), x11 = R(T[(iw + 1) * kX2TabT + it + 1]);
    }
    R y = (R(1) - tw) * ((R(1) - tt) * x00 + tt * x01) + tw * ((R(1) - tt) * x10 + tt * x11) - R(0.5);
    // the bilinear table guess is within 1.3e-5 of the root in y (a cell is 1/n2 = 7.8e-3); one
    // Newton step takes that below 1e-9 and a second to FP64's resolution. FP32 takes two as
    // well: after one the result still depends on how the guess was rounded, which differs
    // between the kernels this is inlined into (the single, batched and staged transfers give
    // bit-identical mixed images only after the second)
    const int iters = 2;
#pragma unroll
    for (int k = 0; k < iters; k++) {
        R d;
        R f = fmks_mu(g, w, y, &d, (R *)nullptr) - mu;
        y -= f / d;
    }
    return fmin(fmax(y, R(-0.5)), R(0.5));
}

// Corner index and fraction of one axis of the trilinear fetch, from an approximate cell
// coordinate (within one cell of the truth) and the exact fraction relative to that corner;
// clamped to the first and last cell centres.
template <typename R>
__device__ __forceinline__ void cell_axis(int n, int &i0, R &f) {
    if (f < R(0) && i0 > 0) {
        i0--;
        f += R(1);
    } else if (f >= R(1) && i0 < n - 2) {
        i0++;
        f -= R(1);
    }
    if (i0 < 0) i0 = 0, f = R(0);
    if (i0 > n - 2) i0 = n - 2, f = R(1);
    f = fmin(fmax(f, R(0)), R(1));
}

// The trilinear fetch of the FMKS grid at (r, theta, phi) in three steps, so that a caller can
// stage the eight cells itself (grid_plasma runs all three):
//  - grid_cell: the corner cell (i0, j0, k0) and the fractions. They are formed from FP64
//    differences to a cell centre (r / r_c - 1, theta - pi/2 of the equator, phi / dx3 minus
//    its floor) before rounding to R: on a grid with structure from cell to cell, a fraction
//    taken from the absolute FP32 coordinates (X1 up to ln r_out, the cell index up to n) is
//    off by 1e-5 of a cell, which the steep thermal emissivity magnifies about twentyfold.
//  - grid_interp (or an interpolation of staged cells in the same order): the primitives;
//  - grid_state: the primitives converted to n_e, Theta_e, B, u and b.
template <typename R>
struct GridCell {
    int i0, j0, k0, k1;
    R r, w, y;      // r in R, the FMKS blend weight and y = X2 - 1/2
    R w1, w2, w3;   // trilinear fractions
};

// false outside r_in <= r <= r_out
template <typename R>
__device__ __forceinline__ bool grid_cell(const GridModel &g, double rd, double thd, double phd, GridCell<R> &c) {
    typedef Mth<R> F;
    R r, th, y, w, w1, w2, w3;
    int i0, j0, k0;
    if constexpr (sizeof(R) == 4) {
        // FP32 form: r, theta, phi as FP32 pairs; the fractions' differences from the pairs by
        // error-free products, with no FP64 instruction and no int/float conversion
        float rl, thl, ph, phl;
        split_ff(rd, r, rl);
        split_ff(thd, th, thl);
        split_ff(phd, ph, phl);
        if (r < g.f_r_in || r > g.f_r_out) return false;
        float X1 = logf(r);
        w = expf(g.f_mks_smooth * (g.f_x1in - X1));
        i0 = min(max(floor_small((X1 - g.f_x1in) / g.f_dx1 - 0.5f), 0), g.n1 - 2);
        // r / r_c - 1 = (p - 1) + (e + r il + rl ih): p = r ih rounded (in [1/2, 2], so p - 1 is
        // exact), e its exact error; one rounding at the end
        const float2 ic = g.x1_irc_f2[i0];
        float pr = r * ic.x;
        float dl = (pr - 1.0f) + (fmaf(r, ic.x, -pr) + fmaf(r, ic.y, rl * ic.x));
        w1 = log1pf(dl) / g.f_dx1;  // ln(r / r_c) / dx1
        cell_axis(g.n1, i0, w1);
        // theta - pi/2 from the pair, pi/2 = 1.57079637f - 4.37113883e-8f
        y = fmks_y(g, w, th, (th - 1.57079637f) + (thl + 4.37113883e-8f));
        float t = y * i2f_small(g.n2), c2 = 0.5f * i2f_small(g.n2 - 1);
        j0 = min(max(floor_small(t + c2), 0), g.n2 - 2);
        w2 = t - (i2f_small(j0) - c2);
        cell_axis(g.n2, j0, w2);
        // azimuthal: phi / dx3 - 1/2 = p + pc - 1/2, p = ph ih rounded, pc its exact error and
        // the remainders' products (|phi / dx3| < 2^22)
        float p = ph * g.f_idx3_hi;
        float pc = fmaf(ph, g.f_idx3_hi, -p) + fmaf(ph, g.f_idx3_lo, phl * g.f_idx3_hi);
        float tk = p - 0.5f;
        int kk = floor_small(tk);
        float fr = (tk - i2f_small(kk)) + pc;
        if (fr < 0.0f) {
            fr += 1.0f;
            kk--;
        } else if (fr >= 1.0f) {
            fr -= 1.0f;
            kk++;
        }
        w3 = fr;
        kk %= g.n3;
        k0 = kk < 0 ? kk + g.n3 : kk;
    } else {
        r = R(rd);
        th = R(thd);
        if (r < pick<R>(g.r_in, g.f_r_in) || r > pick<R>(g.r_out, g.f_r_out)) return false;
        R X1 = F::log_(r);
        w = F::exp_(pick<R>(g.mks_smooth, g.f_mks_smooth) * (pick<R>(g.x1in, g.f_x1in) - X1));
        // radial: corner from the approximate X1, fraction ln(r / r_c) / dx1 about that centre
        i0 = (int)F::floor_((X1 - pick<R>(g.x1in, g.f_x1in)) / pick<R>(g.dx1, g.f_dx1) - R(0.5));
        i0 = min(max(i0, 0), g.n1 - 2);
        w1 = F::log1p_(R(rd * g.x1_irc[i0] - 1.0)) / pick<R>(g.dx1, g.f_dx1);
        cell_axis(g.n1, i0, w1);
        // polar: y = X2 - 1/2; fj = y n2 + (n2 - 1)/2, fraction about the half-integer j0 - (n2 - 1)/2
        y = fmks_y(g, w, th, R(thd - 0.5 * kPi));
        R t = y * R(g.n2), c2 = R(0.5 * (g.n2 - 1));
        j0 = (int)F::floor_(t + c2);
        j0 = min(max(j0, 0), g.n2 - 2);
        w2 = t - (R(j0) - c2);
        cell_axis(g.n2, j0, w2);
        // azimuthal (periodic)
        double fk = phd * g.idx3 - 0.5, kf = floor(fk);
        w3 = R(fk - kf);
        long long kl = (long long)kf % g.n3;
        k0 = (int)(kl < 0 ? kl + g.n3 : kl);
    }
    c.i0 = i0;
    c.j0 = j0;
    c.k0 = k0;
    c.k1 = k0 + 1 == g.n3 ? 0 : k0 + 1;
    c.r = r;
    c.w = w;
    c.y = y;
    c.w1 = w1;
    c.w2 = w2;
    c.w3 = w3;
    return true;
}

template <typename R>
__device__ __forceinline__ void grid_interp(const GridModel &g, const GridCell<R> &c, R P[8]) {
#pragma unroll
    for (int q = 0; q < 8; q++) P[q] = R(0);
#pragma unroll
    for (int di = 0; di < 2; di++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++) {
            long long row = ((long long)(c.i0 + di) * g.n2 + (c.j0 + dj)) * g.n3;
            R wij = (di ? c.w1 : R(1) - c.w1) * (dj ? c.w2 : R(1) - c.w2);
#pragma unroll
            for (int dk = 0; dk < 2; dk++) {
                long long cell = row + (dk ? c.k1 : c.k0);
                R wt = wij * (dk ? c.w3 : R(1) - c.w3);
                float4 lo = __ldg(g.prims + 2 * cell), hi = __ldg(g.prims + 2 * cell + 1);
                P[0] += wt * R(lo.x);
                P[1] += wt * R(lo.y);
                P[2] += wt * R(lo.z);
                P[3] += wt * R(lo.w);
                P[4] += wt * R(hi.x);
                P[5] += wt * R(hi.y);
                P[6] += wt * R(hi.z);
                P[7] += wt * R(hi.w);
            }
        }
}

// Weights of the trilinear interpolation in the order of grid_interp: corner (di, dj, dk).
template <typename R>
__device__ __forceinline__ R trilinear_weight(const GridCell<R> &c, int di, int dj, int dk) {
    R wij = (di ? c.w1 : R(1) - c.w1) * (dj ? c.w2 : R(1) - c.w2);
    return wij * (dk ? c.w3 : R(1) - c.w3);
}

template <typename R>
__device__ __forceinline__ void grid_state(const GridModel &g, const KS<R> &m, const GridCell<R> &c, const R P[8],
                                           Plasma<R> &o) {
    typedef Mth<R> F;
    o.valid = false;
    const R r = c.r;
    R rho = P[0], uu = P[1];
    if (!(rho > R(0)) || !(uu > R(0))) return;
    R dth2, dd;
    fmks_mu(g, c.w, c.y, &dth2, &dd);
    R dth1 = -pick<R>(g.mks_smooth, g.f_mks_smooth) * c.w * dd;
    R Ut[4] = {R(0), r * P[2], dth1 * P[2] + dth2 * P[3], P[4]};
    R Bi[4] = {R(0), r * P[5], dth1 * P[5] + dth2 * P[6], P[7]};
    // KS lapse 1/sqrt(1+q), shift beta^r = q/(1+q)
    R Ul[4];
    m.lower(Ut, Ul);
    R gam = F::sqrt_(R(1) + Ul[1] * Ut[1] + Ul[2] * Ut[2] + Ul[3] * Ut[3]);
    R sop = F::sqrt_(m.op);
    o.u[0] = gam * sop;
    o.u[1] = Ut[1] - gam * m.q / sop;
    o.u[2] = Ut[2];
    o.u[3] = Ut[3];
    R ul[4];
    m.lower(o.u, ul);
    R bt = Bi[1] * ul[1] + Bi[2] * ul[2] + Bi[3] * ul[3];
    R iut = R(1) / o.u[0];
    o.b[0] = bt;
    o.b[1] = (Bi[1] + bt * o.u[1]) * iut;
    o.b[2] = (Bi[2] + bt * o.u[2]) * iut;
    o.b[3] = (Bi[3] + bt * o.u[3]) * iut;
    R bsq = m.dot(o.b, o.b);
    if (bsq > pick<R>(g.sigma_cut, g.f_sigma_cut) * rho) return;
    R ga = pick<R>(g.gamma_ad, g.f_gamma_ad);
    // R = (R_high beta^2 + R_low)/(1 + beta^2), written in 1/beta so nothing overflows
    R ib = bsq / (R(2) * (ga - R(1)) * uu);
    R ib2 = ib * ib;
    R Rt = ib2 < R(1e30) ? (pick<R>(g.R_high, g.f_R_high) + pick<R>(g.R_low, g.f_R_low) * ib2) / (R(1) + ib2)
                         : pick<R>(g.R_low, g.f_R_low);
    o.ne = rho * pick<R>(g.ne_unit, g.f_ne_unit);
    o.Te = R(kMp / kMe) * (ga - R(1)) * uu / (rho * (R(1) + Rt));
    o.B = F::sqrt_(fmax(bsq, R(0))) * pick<R>(g.b_unit, g.f_b_unit);
    o.valid = true;
}

template <typename R>
__device__ __forceinline__ void grid_plasma(const GridModel &g, const KS<R> &m, double rd, double thd, double phd,
                                            Plasma<R> &o) {
    GridCell<R> c;
    if (!grid_cell(g, rd, thd, phd, c)) {
        o.valid = false;
        return;
    }
    R P[8];
    grid_interp(g, c, P);
    grid_state(g, m, c, P, o);
}

// ------------------------------------------------------------------------------------------
// Fluid tetrad: e3 the unit projection of k = -K normal to u; e2 the unit part of b normal to
// (u, e3) (d_theta if b is along k); e1 = Levi-Civita(e0, e2, e3) so (e1, e2, e3) is right
// handed. Returns w = -k.u = nu/nu_obs, sin and cos of the field angle.
template <typename R>
__device__ __forceinline__ void fluid_tetrad(const KS<R> &m, const R K[4], const R u[4], const R b[4], R e1[4],
                                             R e2[4], R &w, R &sth, R &cth) {
    typedef Mth<R> F;
    w = m.dot(K, u);
    R e3[4];
#pragma unroll
    for (int i = 0; i < 4; i++) e3[i] = -K[i] - w * u[i];
    R n3 = R(1) / F::sqrt_(m.dot(e3, e3));
#pragma unroll
    for (int i = 0; i < 4; i++) e3[i] *= n3;
    // scale b to order one first (only its direction enters), so FP32 cannot underflow
    R bs = fmax(fmax(fabs(b[0]), fabs(b[1])), fmax(fabs(b[2]), fabs(b[3])));
    R bn[4];
    R ibs = bs > R(0) ? R(1) / bs : R(0);
#pragma unroll
    for (int i = 0; i < 4; i++) bn[i] = b[i] * ibs;
    R bb = m.dot(bn, bn), be3 = m.dot(bn, e3);
#pragma unroll
    for (int i = 0; i < 4; i++) e2[i] = bn[i] - be3 * e3[i];
    R n2 = F::sqrt_(fmax(m.dot(e2, e2), R(0)));
    if (bb > R(0)) {
        R ibn = R(1) / F::sqrt_(bb);
        sth = n2 * ibn;
        cth = be3 * ibn;
    } else {  // no field: no emission (the coefficients vanish with B)
        sth = R(0);
        cth = R(1);
    }
    if (!(n2 > R(1e-10) * F::sqrt_(bb))) {
        R v[4] = {R(0), R(0), R(1), R(0)};
        R vu = m.dot(v, u), ve = m.dot(v, e3);
#pragma unroll
        for (int i = 0; i < 4; i++) e2[i] = v[i] + vu * u[i] - ve * e3[i];
        n2 = F::sqrt_(m.dot(e2, e2));
    }
    R in2 = R(1) / n2;
#pragma unroll
    for (int i = 0; i < 4; i++) e2[i] *= in2;
    // e1_mu = -sqrt(-g) eps[mu nu rho sigma] u^nu e2^rho e3^sigma (generalized cross product)
    const R *A = u, *Bv = e2, *Cv = e3;
    auto det3 = [&](int i, int j, int k) {
        return A[i] * (Bv[j] * Cv[k] - Bv[k] * Cv[j]) - A[j] * (Bv[i] * Cv[k] - Bv[k] * Cv[i]) +
               A[k] * (Bv[i] * Cv[j] - Bv[j] * Cv[i]);
    };
    R sg = m.sqrt_mg();
    R low[4] = {-sg * det3(1, 2, 3), sg * det3(0, 2, 3), -sg * det3(0, 1, 3), sg * det3(0, 1, 2)};
    m.raise(low, e1);
    R n1 = R(1) / F::sqrt_(m.dot(e1, e1));
#pragma unroll
    for (int i = 0; i < 4; i++) e1[i] *= n1;
}

}  // namespace prt
