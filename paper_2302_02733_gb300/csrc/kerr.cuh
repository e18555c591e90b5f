// Kerr geometry in spherical Kerr-Schild coordinates (t, r, theta, phi), G = c = M = 1.
//
// With Sigma = r^2 + a^2 cos^2, q = 2r/Sigma and the Kerr-Schild null form
// l_mu = (1, 1, 0, -a sin^2), the metric is g = (oblate flat part) + q l l:
//   g_tt = -1 + q, g_tr = q, g_tphi = -a s^2 q, g_rr = 1 + q, g_rphi = -a s^2 (1 + q),
//   g_thth = Sigma, g_phiphi = s^2 (Sigma + a^2 s^2 (1 + q)),
// and the inverse is g^tt = -(1 + q), g^tr = q, g^rr = Delta/Sigma, g^rphi = a/Sigma,
// g^thth = 1/Sigma, g^phiphi = 1/(Sigma s^2).
//
// Only r and theta enter, so every connection contraction is built from the two partial
// derivatives of g. The geodesic acceleration -Gamma^mu_ab K^a K^b = -g^{mu nu}(A_nu - B_nu),
// with A_nu = (K^a d_a g_{nu b}) K^b and B_nu = 1/2 d_nu g_ab K^a K^b, is evaluated
// directly, without forming the 40 connection coefficients.
#pragma once
#include "ffloat.cuh"
#include "rt_common.cuh"

namespace prt {

template <typename R>
struct Fn;
template <>
struct Fn<double> {
    static __device__ __forceinline__ void sc(double x, double *s, double *c) { sincos(x, s, c); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
};
template <>
struct Fn<float> {
    static __device__ __forceinline__ void sc(float x, float *s, float *c) { sincosf(x, s, c); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rcp(float x) { return 1.0f / x; }
};

// Metric, inverse and the two derivative sets at (r, theta).
template <typename R>
struct KS {
    R a, r, s, c, s2, sc, sig, isig, iss, q, op, dqr, dqt;
    R tt, tr, tp, rr, rp, hh, pp;  // g_{mu nu}
    R Itt, Itr, Irr, Irp, Ihh, Ipp;  // g^{mu nu}

    __device__ __forceinline__ void eval(R a_, R r_, R th) {
        R s_, c_;
        Fn<R>::sc(th, &s_, &c_);
        eval_sc(a_, r_, s_, c_);
    }
    __device__ __forceinline__ void eval_sc(R a_, R r_, R s_, R c_) {
        a = a_;
        r = r_;
        s = s_;
        c = c_;
        s2 = s * s;
        sc = s * c;
        R a2 = a * a;
        sig = r * r + a2 * c * c;
        iss = Fn<R>::rcp(sig * s2);
        isig = iss * s2;
        q = R(2) * r * isig;
        op = R(1) + q;
        dqr = R(2) * isig - q * q;
        dqt = R(2) * a2 * sc * q * isig;
        tt = q - R(1);
        tr = q;
        tp = -a * s2 * q;
        rr = op;
        rp = -a * s2 * op;
        hh = sig;
        pp = s2 * (sig + a2 * s2 * op);
        Itt = -op;
        Itr = q;
        Irr = (r * r - R(2) * r + a2) * isig;
        Irp = a * isig;
        Ihh = isig;
        Ipp = iss;
    }
    __device__ __forceinline__ R dot(const R u[4], const R v[4]) const {
        return tt * u[0] * v[0] + tr * (u[0] * v[1] + u[1] * v[0]) + tp * (u[0] * v[3] + u[3] * v[0]) +
               rr * u[1] * v[1] + rp * (u[1] * v[3] + u[3] * v[1]) + hh * u[2] * v[2] + pp * u[3] * v[3];
    }
    __device__ __forceinline__ void lower(const R u[4], R l[4]) const {
        l[0] = tt * u[0] + tr * u[1] + tp * u[3];
        l[1] = tr * u[0] + rr * u[1] + rp * u[3];
        l[2] = hh * u[2];
        l[3] = tp * u[0] + rp * u[1] + pp * u[3];
    }
    __device__ __forceinline__ void raise(const R l[4], R u[4]) const {
        u[0] = Itt * l[0] + Itr * l[1];
        u[1] = Itr * l[0] + Irr * l[1] + Irp * l[3];
        u[2] = Ihh * l[2];
        u[3] = Irp * l[1] + Ipp * l[3];
    }
    __device__ __forceinline__ R sqrt_mg() const { return sig * s; }  // sqrt(-g) = Sigma sin
};

// Contractions of the metric derivatives with a vector K:
//   D_{nu b} = K^r d_r g_{nu b} + K^th d_th g_{nu b}   (7 unique entries)
//   P_nu = d_r g_{nu a} K^a,  Q_nu = d_th g_{nu a} K^a.
template <typename R>
struct DK {
    R d1, dtp, drp, dhh, dpp;  // D_tt = D_tr = D_rr = d1
    R P[4], Qv[4];
    __device__ __forceinline__ void eval(const KS<R> &m, const R K[4]) {
        R a = m.a, a2 = a * a;
        R W = K[0] + K[1];
        R V = W - a * m.s2 * K[3];
        d1 = K[1] * m.dqr + K[2] * m.dqt;
        R two_sc = R(2) * m.sc;
        dtp = -a * (m.s2 * d1 + two_sc * m.q * K[2]);
        drp = -a * (m.s2 * d1 + two_sc * m.op * K[2]);
        dhh = R(2) * m.r * K[1] - R(2) * a2 * m.sc * K[2];
        R bigp = m.sig + a2 * m.s2 * (R(1) + R(2) * m.q);
        dpp = R(2) * m.r * m.s2 * K[1] + a2 * m.s2 * m.s2 * d1 + two_sc * bigp * K[2];
        P[0] = m.dqr * V;
        P[1] = P[0];
        P[2] = R(2) * m.r * K[2];
        P[3] = -a * m.s2 * m.dqr * V + R(2) * m.r * m.s2 * K[3];
        Qv[0] = m.dqt * V - two_sc * a * m.q * K[3];
        Qv[1] = m.dqt * V - two_sc * a * m.op * K[3];
        Qv[2] = -R(2) * a2 * m.sc * K[2];
        Qv[3] = -a * m.s2 * m.dqt * V - two_sc * a * (m.q * K[0] + m.op * K[1]) + two_sc * bigp * K[3];
    }
    // D_{nu b} as a full symmetric 4x4 accessor
    __device__ __forceinline__ R D(int n, int b) const {
        if (n > b) { int t = n; n = b; b = t; }
        if (n == 2 || b == 2) return (n == 2 && b == 2) ? dhh : R(0);
        if (b == 3) return n == 0 ? dtp : (n == 1 ? drp : dpp);
        return d1;  // (0,0), (0,1), (1,1)
    }
};

// sin and cos of theta for the FP64 geodesic by table-driven angle addition: theta_k from a
// table of (theta_k, sin theta_k, cos theta_k) at spacing h = 1.5 pi / 1023 over
// [-pi/4, 5 pi/4] (24 KB, small enough for shared memory), delta = theta - theta_k
// (|delta| <= h/2 < 2.4e-3), then sin(theta_k + delta) = s_k cos(delta) + c_k sin(delta) with
// the Taylor polynomials sin d = d - d^3/6 + d^5/120 (remainder below 1e-22) and
// cos d = 1 - d^2/2 + d^4/24 (remainder d^6/720 below 2.1e-19, a thousandth of an ulp of 1).
// Outside the table range it falls back to sincos().
constexpr int kSinTab = 1024;
constexpr double kSinLo = -0.25 * kPi;
constexpr double kSinH = 1.5 * kPi / (kSinTab - 1);

__device__ __forceinline__ void sincos_tab(const double *__restrict__ tab, double th, double *s, double *c) {
    // the nearest node from theta rounded to FP32, with integer and FP32 operations (an FP64
    // to int conversion would take the FP64 pipe); a node one off, for a theta halfway between
    // two, leaves |delta| a few 1e-7 above kSinH / 2, well inside the polynomials' accuracy.
    // A NaN or infinite theta gives a k outside the table.
    int k = rint_small(fmaf(d2f_int(th), float(1.0 / kSinH), float(-kSinLo / kSinH)));
    if (k < 1 || k > kSinTab - 2) {  // outside the table
        sincos(th, s, c);
        return;
    }
    const double *e = tab + 3 * k;
    double d = th - e[0];  // |d| <= kSinH / 2
    double sk = e[1], ck = e[2];
    double d2 = d * d;
    double sd = fma(d * d2, fma(d2, 1.0 / 120.0, -1.0 / 6.0), d);       // sin d
    double cm = d2 * fma(d2, 1.0 / 24.0, -0.5);                          // cos d - 1
    *s = fma(sk, cm, fma(ck, sd, sk));
    *c = fma(ck, cm, fma(-sk, sd, ck));
}

// 1/x for positive x between 2^-120 and 2^120: a seed from FP32, x rounded to FP32 and
// rcp.approx.ftz.f32 (relative error of the seed below 2^-22; both conversions on the integer
// pipe, the reciprocal on the special-function unit, so the seed takes no FP64 instruction),
// refined by one third-order step: with e = 1 - x r (exact to its rounding),
// 1/x = r / (1 - e) = r (1 + e + e^2 + ...), so r (1 + e + e^2) leaves a relative error of
// e^3 < 2^-66 before the last rounding. The result is the correctly rounded quotient except,
// rarely, one ulp from it (a quotient within 2^-66 of a rounding boundary).
__device__ __forceinline__ double recip_nr(double x) {
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(d2f_int(x)));
    const double r = f2d_int(rf);
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// Geodesic acceleration dK/dl = -Gamma K K (FP64 path), arranged for the FP64 pipe: every
// product that can be folded into a fused multiply-add is, and products shared by the
// contractions are formed once. Same quantities as DK::eval / connection_T:
//   A_nu = D_{nu b} K^b, B_r = K.P/2, B_th = K.Q/2, F = A - B, acc = -g^{-1} F,
// with the two B terms summed in closed form. With V = l.K = K^t + K^r - a s^2 K^phi:
//   K.P = dq/dr V^2 + 2 r (K^th^2 + s^2 K^phi^2),
//   K.Q = dq/dth V^2 + 2 s c [P K^phi^2 - a^2 K^th^2 - 2 a K^phi (q (K^t + K^r) + K^r)],
// P = Sigma + a^2 s^2 (1 + 2 q): the P and Q contractions of DK::eval summed against K and
// simplified, which takes fewer FP64 operations than forming P_nu and Q_nu and summing them.
//
// The geodesic carries W = K^t + K^r in place of K^t (the stationary metric's K^t enters the
// acceleration only through W): K = (W, K^r, K^theta, K^phi) on input, and acc[0] = dW/dl.
__device__ __forceinline__ void geo_accel(const double *__restrict__ sctab, double a, double r, double th,
                                          const double K[4], double acc[4], double fac[4]) {
    const double a2 = a * a;
    double s, c;
    sincos_tab(sctab, th, &s, &c);
    const double W = K[0], Kr = K[1], Kh = K[2], Kp = K[3];
    // metric pieces
    double s2 = s * s, sc = s * c;
    double a2s2 = a2 * s2;
    double sa = fma(r, r, a2);                 // r^2 + a^2
    double sig = sa - a2s2;                    // Sigma = r^2 + a^2 cos^2 (>= r^2: no cancellation)
    double iss = recip_nr(sig * s2);  // 1/(Sigma sin^2)
    double isig = iss * s2;         // 1/Sigma
    double tr = twice(r);           // 2r (twice, halve: exact, on the integer pipe)
    double q = tr * isig;           // 2r/Sigma
    double dqr = fma(-q, q, twice(isig));      // d q/dr
    double two_sc = twice(sc);
    double dqt = (a2 * two_sc) * (q * isig);   // d q/dtheta
    // contractions with K
    double as2 = a * s2;
    double V = fma(-as2, Kp, W);               // l_mu K^mu
    double d1 = fma(Kr, dqr, Kh * dqt);        // D_tt = D_tr = D_rr
    double scK = two_sc * Kh;
    double m = fma(s2, d1, q * scK);           // -D_tphi / a
    double bigp = fma(twice(q), a2s2, sa);
    double trKr = tr * Kr;
    double dpp = fma(s2, fma(a2s2, d1, trKr), bigp * scK);  // D_phiphi
    // A_nu and F = A - B
    double d1W = d1 * W;
    double aKp = a * Kp;
    double At = fma(-m, aKp, d1W);
    double Ar = fma(-scK, aKp, At);            // -D_rphi = -D_tphi + a scK
    double Ap = fma(dpp, Kp, -a * fma(m, W, scK * Kr));
    double hV2 = halve(V) * V, Kh2 = Kh * Kh, Kp2 = Kp * Kp;
    double Fr = fma(-dqr, hV2, fma(-r, fma(s2, Kp2, Kh2), Ar));
    double t = fma(bigp, Kp2, a2 * Kh2);
    t = fma(-twice(aKp), fma(q, W, Kr), t);
    double Fh = fma(trKr, Kh, fma(-dqt, hV2, -sc * t));
    // acc = -g^{-1} F with g^tt = -(1+q), g^tr = q, g^rr = Delta/Sigma, g^rphi = a/Sigma,
    // g^thth = 1/Sigma, g^phiphi = 1/(Sigma sin^2)
    double del = sa - tr;
    // dK^t = (1 + q) At - q Fr and dK^r = -(isig (del Fr + a Ap) + q At), so
    // dW = At - q Fr - isig (del Fr + a Ap)
    const double X = fma(del, Fr, a * Ap);
    acc[0] = fma(-isig, X, fma(-q, Fr, At));
    acc[1] = -fma(isig, X, q * At);
    // The theta and phi rates are products, acc[2] = fac[0] fac[1] and acc[3] = fac[2] fac[3],
    // rounded here with mul.rn, which the compiler never contracts into a later addition: a
    // caller's sums of these rates then round alike wherever they are compiled. A caller that
    // wants a rate fused into a sum takes its factors (fac) and writes the fma itself.
    fac[0] = -isig;
    fac[1] = Fh;
    fac[2] = -iss;
    fac[3] = fma(as2, Fr, Ap);  // a/Sigma = a s^2 / (Sigma s^2)
    acc[2] = __dmul_rn(fac[0], fac[1]);
    acc[3] = __dmul_rn(fac[2], fac[3]);
}

// T^mu_b = Gamma^mu_{a b} K^a = 1/2 g^{mu nu} (D_{nu b} + [b=r] P_nu + [b=th] Q_nu
//                                              - [nu=r] P_b - [nu=th] Q_b).
template <typename R>
__device__ __forceinline__ void connection_T(const KS<R> &m, const R K[4], R T[4][4]) {
    DK<R> d;
    d.eval(m, K);
    R M[4][4];
#pragma unroll
    for (int n = 0; n < 4; n++)
#pragma unroll
        for (int b = 0; b < 4; b++) {
            R v = d.D(n, b);
            if (b == 1) v += d.P[n];
            if (b == 2) v += d.Qv[n];
            if (n == 1) v -= d.P[b];
            if (n == 2) v -= d.Qv[b];
            M[n][b] = v;
        }
#pragma unroll
    for (int b = 0; b < 4; b++) {
        R col[4] = {M[0][b], M[1][b], M[2][b], M[3][b]}, up[4];
        m.raise(col, up);
        T[0][b] = R(0.5) * up[0];
        T[1][b] = R(0.5) * up[1];
        T[2][b] = R(0.5) * up[2];
        T[3][b] = R(0.5) * up[3];
    }
}

}  // namespace prt
