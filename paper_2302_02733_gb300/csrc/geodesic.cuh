// Geodesic building blocks shared by the per-image and the batched kernels: the initial
// state of a pixel's ray, the radius-scaled step size, one classic RK4 step with polar
// reflection, and the stop tests (the paper's Section 2.1).
#pragma once
#include "camera.cuh"
#include "rt_kernels.cuh"

namespace prt {

// Order of positive doubles by their bit patterns (as signed 64-bit integers a negative
// double orders below every positive one). Comparisons on the integer pipe keep the FP64 pipe,
// the kernel's bound, for arithmetic.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double pos_min(double x, double y) { return dbits(x) < dbits(y) ? x : y; }
__device__ __forceinline__ double pos_max(double x, double y) { return dbits(x) < dbits(y) ? y : x; }

// h = eps / (|K^r|/r + |K^th|/tt + |K^ph| + 1e-40), tt = max(min(th, pi - th), 0.01), taken
// with one reciprocal: h = eps r tt / (|K^r| tt + |K^th| r + |K^ph| r tt). Here 0 <= th <= pi,
// so min and max compare bit patterns. The 1e-40 only keeps the denominator from zero: it is
// below half an ulp of |K^ph| >= 1e-24 and of any denominator above 1e-24 r tt, so it changes
// no rounded result there; a floor on the bit pattern stands in for it, without an FP64
// addition. The floor is 1e-30, inside the reciprocal's range; it differs from the 1e-40 term
// only for denominators below 1e-30, where the step already exceeds 1e27 r tt.
__device__ __forceinline__ double step_size(double eps, const double y[7]) {
    double tt = pos_max(pos_min(y[1], kPi - y[1]), 1e-2);
    double rt = y[0] * tt;
    double den = fma(fabs(y[6]), rt, fma(fabs(y[4]), tt, fabs(y[5]) * y[0]));
    den = pos_max(den, 1e-30);
    return (eps * rt) * recip_nr(den);
}

// y = (r, theta, phi, W, K^r, K^theta, K^phi) with W = K^t + K^r (geo_accel); t is never
// needed (stationary metric). Saved states hold K^t = W - K^r.
//
// The position rates of a stage are the previous stage's K: k1 = y_K and k_j+1 = K of stage
// j+1. So a position and its K component share the sums: with T = k2 + k3 and S = k1 + T of
// the K component, the classic weights give
//   position' = position + h y_K + (h^2 / 6) S,  K' = y_K + (h / 6) (S + T + k4),
// and W' = y_W + h/6 k1 + h/3 k2 + h/3 k3 + h/6 k4, summed in that order.
// h/6 is taken as half of h/3: 1/6 in FP64 is half of 1/3, so the product rounds to the same
// bits.
//
// Two forms with the same arithmetic, hence bit-identical states. LOOP = false writes the four
// right-hand sides out (the faster form in a kernel of its own); LOOP = true runs the stages as
// one loop over a single copy of the right-hand side, a quarter of the instruction footprint,
// for the persistent kernel, whose geodesic and transfer loops compete for the instruction
// cache. No sum is left for the compiler to contract: every addend is an fma, a negated fma or
// a rate rounded by mul.rn (geo_accel), and the last stage's theta and phi rates enter their
// sums through an explicit fma of their factors. (Left to the compiler, the written-out form
// fused rate products into the sums that the loop form keeps in other basic blocks, and the two
// forms' states differed by rounding.)
template <bool LOOP>
__device__ __forceinline__ void rk4_step(const double *__restrict__ tab, double a, double h, const double y[7],
                                         double out[7]) {
    const double h2 = halve(h), h3 = h * (1.0 / 3.0), h6 = halve(h3), hh6 = h * h6;
    double S[3], T[3];
    if (!LOOP) {
        double k1[4], k2[4], k3[4], k4[4], f[4], z[2], zk[4];
        geo_accel(tab, a, y[0], y[1], y + 3, k1, f);  // k = d(W, K^r, K^theta, K^phi)
        z[0] = fma(h2, y[4], y[0]);
        z[1] = fma(h2, y[5], y[1]);
#pragma unroll
        for (int i = 0; i < 4; i++) zk[i] = fma(h2, k1[i], y[3 + i]);
        geo_accel(tab, a, z[0], z[1], zk, k2, f);
        z[0] = fma(h2, zk[1], y[0]);
        z[1] = fma(h2, zk[2], y[1]);
#pragma unroll
        for (int i = 0; i < 4; i++) zk[i] = fma(h2, k2[i], y[3 + i]);
        geo_accel(tab, a, z[0], z[1], zk, k3, f);
        z[0] = fma(h, zk[1], y[0]);
        z[1] = fma(h, zk[2], y[1]);
#pragma unroll
        for (int i = 0; i < 4; i++) zk[i] = fma(h, k3[i], y[3 + i]);
        geo_accel(tab, a, z[0], z[1], zk, k4, f);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            T[i] = k2[1 + i] + k3[1 + i];
            S[i] = k1[1 + i] + T[i];
        }
        out[3] = fma(h6, k4[0], fma(h3, k3[0], fma(h3, k2[0], fma(h6, k1[0], y[3]))));
        out[4] = fma(h6, (S[0] + T[0]) + k4[1], y[4]);
        out[5] = fma(h6, fma(f[0], f[1], S[1] + T[1]), y[5]);
        out[6] = fma(h6, fma(f[2], f[3], S[2] + T[2]), y[6]);
    } else {
        double z[7], k[4], f[4], k1[3], k2[3], w;
#pragma unroll
        for (int i = 0; i < 7; i++) z[i] = y[i];
#pragma unroll 1
        for (int st = 0; st < 4; st++) {
            geo_accel(tab, a, z[0], z[1], z + 3, k, f);
            if (st == 0) {
                w = fma(h6, k[0], y[3]);
#pragma unroll
                for (int i = 0; i < 3; i++) k1[i] = k[1 + i];
            } else if (st == 1) {
                w = fma(h3, k[0], w);
#pragma unroll
                for (int i = 0; i < 3; i++) k2[i] = k[1 + i];
            } else if (st == 2) {
                w = fma(h3, k[0], w);
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    T[i] = k2[i] + k[1 + i];
                    S[i] = k1[i] + T[i];
                }
            } else {
                out[3] = fma(h6, k[0], w);
                out[4] = fma(h6, (S[0] + T[0]) + k[1], y[4]);
                out[5] = fma(h6, fma(f[0], f[1], S[1] + T[1]), y[5]);
                out[6] = fma(h6, fma(f[2], f[3], S[2] + T[2]), y[6]);
                break;
            }
            // the next stage's state from y: positions advance with this stage's K (z[4], z[5])
            const double c = st == 2 ? h : h2;
            const double r = fma(c, z[4], y[0]), th = fma(c, z[5], y[1]);
            z[0] = r;
            z[1] = th;
#pragma unroll
            for (int i = 0; i < 4; i++) z[3 + i] = fma(c, k[i], y[3 + i]);
        }
    }
#pragma unroll
    for (int i = 0; i < 3; i++) out[i] = fma(hh6, S[i], fma(h, y[4 + i], y[i]));
}

// Initial state of the backward ray through pixel (ix, iy): the camera frame's past-directed
// null vector K = -e_0 + s^i e_i at (r_cam, theta_o, 0), the frame computed once per camera.
__device__ __forceinline__ void ray_start(const Camera &c, int ix, int iy, double y[7]) {
    const double(&e)[4][4] = c.e;
    double s[3];
    sky_direction(c, ix, iy, s);
    y[0] = c.r_cam;
    y[1] = c.theta_o;
    y[2] = 0.0;
#pragma unroll
    for (int k = 0; k < 4; k++) y[3 + k] = -e[0][k] + s[0] * e[1][k] + s[1] * e[2][k] + s[2] * e[3][k];
    y[3] += y[4];  // W = K^t + K^r
}

// The camera constants a geodesic step and its stop test read. The batched kernel, whose
// cameras live in a global job table, keeps them in registers for the life of a ray.
struct StepCam {
    double a, eps, r_stop, r_cam;
    int nmax;
};
__device__ __forceinline__ StepCam step_cam(const Camera &c) { return StepCam{c.a, c.eps, c.r_stop, c.r_cam, c.nmax}; }

// One step from y: yn, the step h, and whether it crossed the polar axis (then theta is
// reflected, phi advanced by pi and K^theta reversed). C is Camera or StepCam; LOOP selects
// the form of rk4_step.
template <bool LOOP = false, class C>
__device__ __forceinline__ bool geo_step(const double *__restrict__ tab, const C &c, const double y[7],
                                         double yn[7], double &h) {
    h = step_size(c.eps, y);
    rk4_step<LOOP>(tab, c.a, h, y, yn);
    bool refl = false;
    long long tb = dbits(yn[1]);
    if (tb < 0 && (tb << 1) != 0) {  // theta < 0 (not -0)
        yn[1] = -yn[1];
        yn[2] += kPi;
        yn[5] = -yn[5];
        refl = true;
    } else if (tb > dbits(kPi)) {  // theta > pi
        yn[1] = 2.0 * kPi - yn[1];
        yn[2] += kPi;
        yn[5] = -yn[5];
        refl = true;
    }
    return refl;
}

// Stop test after n steps, in order: non-finite, horizon, escape, step limit; 0 to go on.
template <class C>
__device__ __forceinline__ uint8_t geo_stop(const C &c, const double y[7], int n) {
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 7; k++) bad |= (__double2hiint(y[k]) & 0x7ff00000) == 0x7ff00000;  // inf or NaN
    if (bad) return kNan;
    if (dbits(y[0]) < dbits(c.r_stop)) return kHorizon;
    if (dbits(y[0]) > dbits(c.r_cam) && dbits(y[4]) > 0) return kEscape;
    if (n >= c.nmax) return kNmax;
    return 0;
}

}  // namespace prt
