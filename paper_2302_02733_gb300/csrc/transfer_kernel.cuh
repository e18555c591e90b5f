// The transfer kernel (persistent, one ray per lane, per-lane refill from a work queue). Each
// lane walks its ray's saved states from the far end back to the camera. At every state it
// parallel-transports the screen legs (Heun, connection from the saved K), evaluates the
// plasma, and if the point emits it projects onto the fluid screen and takes the exact
// constant-coefficient step. Instantiated for the FP64 and the mixed (FP32 transfer) forms.
#pragma once
#include <cuda.h>

#include "surrogate.cuh"
#include "tc.cuh"
#include "transfer.cuh"

namespace prt {

// The FP32 form reads the FP64 path with d2f_int (ffloat.cuh): integer operations only.
template <typename R>
__device__ __forceinline__ R to_real(double d);
template <>
__device__ __forceinline__ double to_real<double>(double d) {
    return d;
}
template <>
__device__ __forceinline__ float to_real<float>(double d) {
    return d2f_int(d);
}

// o = T v for a 4x4 matrix
template <typename R>
__device__ __forceinline__ void matvec4(const R T[4][4], const R v[4], R o[4]) {
#pragma unroll
    for (int m = 0; m < 4; m++) o[m] = T[m][0] * v[0] + T[m][1] * v[1] + T[m][2] * v[2] + T[m][3] * v[3];
}

// Heun step of a screen leg held as base + increment, E = eo + u: with a = T(x_{n+1}) E known
// from the previous point and T0 = T(x_n), v = E + h a and E gains (h/2)(a + T0 v). Only the
// increment u changes, so E - e (needed by the compensated re-projection) stays exact.
template <typename R>
__device__ __forceinline__ void heun_leg(const R eo[4], R u[4], const R a[4], const R T0[4][4], R h) {
    R v[4];
#pragma unroll
    for (int m = 0; m < 4; m++) v[m] = (eo[m] + u[m]) + h * a[m];
    R hh = R(0.5) * h;
#pragma unroll
    for (int m = 0; m < 4; m++)
        u[m] += hh * (a[m] + T0[m][0] * v[0] + T0[m][1] * v[1] + T0[m][2] * v[2] + T0[m][3] * v[3]);
}

// Stokes (I, Q, U, V) in the screen (E1, E2) re-expressed on the screen (f1, f2) given as
// lowered legs: n' = C n C^T, C_{ij} = f_i . E_j. Used once, at the camera.
template <typename R>
__device__ __forceinline__ void reproject(const R f1[4], const R f2[4], const R E1[4], const R E2[4], R S[4]) {
    R c11 = f1[0] * E1[0] + f1[1] * E1[1] + f1[2] * E1[2] + f1[3] * E1[3];
    R c12 = f1[0] * E2[0] + f1[1] * E2[1] + f1[2] * E2[2] + f1[3] * E2[3];
    R c21 = f2[0] * E1[0] + f2[1] * E1[1] + f2[2] * E1[2] + f2[3] * E1[3];
    R c22 = f2[0] * E2[0] + f2[1] * E2[1] + f2[2] * E2[2] + f2[3] * E2[3];
    R n11 = R(0.5) * (S[0] + S[1]), n22 = R(0.5) * (S[0] - S[1]), nr = R(0.5) * S[2];
    R m11 = c11 * c11 * n11 + R(2) * c11 * c12 * nr + c12 * c12 * n22;
    R m22 = c21 * c21 * n11 + R(2) * c21 * c22 * nr + c22 * c22 * n22;
    R mr = c11 * c21 * n11 + (c11 * c22 + c12 * c21) * nr + c12 * c22 * n22;
    R det = c11 * c22 - c12 * c21;
    S[0] = m11 + m22;
    S[1] = m11 - m22;
    S[2] = R(2) * mr;
    S[3] = det * S[3];
}

// Stokes re-expressed from the transported screen E_k = eo_k + u_k onto the new fluid screen
// (e1, e2), lowered l1, l2, as a compensated increment. The new coefficients are
// n' = C n C^T with C = G^{-1} A, A_ik = l_i . E_k and G_ij = l_i . e_j: the dual basis of
// (e1, e2), so the rounding of their norms does not scale the intensity. Writing
// E_k = e_k + Delta_k with Delta_k = (eo_k - e_k) + u_k (exact differences of nearby legs plus
// the transport increment) gives C = 1 + D, D = G^{-1} Lambda, Lambda_ik = l_i . Delta_k, and
// n' - n = D n + n D^T + D n D^T; V scales by det C = 1 + tr D + det D. The change is small
// where the screen turns slowly and is added to (S, Slo) without rounding loss.
template <typename R>
__device__ __forceinline__ void reproject_comp(const R l1[4], const R l2[4], const R e1[4], const R e2[4],
                                               const R eo1[4], const R eo2[4], const R u1[4], const R u2[4],
                                               R S[4], R Slo[4]) {
    R L11 = 0, L12 = 0, L21 = 0, L22 = 0, g11 = 0, g12 = 0, g21 = 0, g22 = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        R d1 = (eo1[i] - e1[i]) + u1[i];
        R d2 = (eo2[i] - e2[i]) + u2[i];
        L11 += l1[i] * d1;
        L12 += l1[i] * d2;
        L21 += l2[i] * d1;
        L22 += l2[i] * d2;
        g11 += l1[i] * e1[i];
        g12 += l1[i] * e2[i];
        g21 += l2[i] * e1[i];
        g22 += l2[i] * e2[i];
    }
    R idet = R(1) / (g11 * g22 - g12 * g21);
    R d11 = (g22 * L11 - g12 * L21) * idet, d12 = (g22 * L12 - g12 * L22) * idet;
    R d21 = (g11 * L21 - g21 * L11) * idet, d22 = (g11 * L22 - g21 * L12) * idet;
    R n11 = R(0.5) * (S[0] + S[1]), n22 = R(0.5) * (S[0] - S[1]), nr = R(0.5) * S[2];
    R x11 = d11 * n11 + d12 * nr, x12 = d11 * nr + d12 * n22;
    R x21 = d21 * n11 + d22 * nr, x22 = d21 * nr + d22 * n22;
    R dn11 = R(2) * x11 + (x11 * d11 + x12 * d12);
    R dn22 = R(2) * x22 + (x21 * d21 + x22 * d22);
    R dnr = (x12 + x21) + (x11 * d21 + x12 * d22);
    R dV = ((d11 + d22) + (d11 * d22 - d12 * d21)) * S[3];
    two_sum_add(S[0], Slo[0], dn11 + dn22);
    two_sum_add(S[1], Slo[1], dn11 - dn22);
    two_sum_add(S[2], Slo[2], R(2) * dnr);
    two_sum_add(S[3], Slo[3], dV);
}

// Per-lane transfer state of one ray. S + Slo: Stokes / nu^3 (invariant) as a value and its
// compensation; eo + u: screen legs (base, transport increment); a1, a2: T E of the legs at the
// previous point; tau, phi: optical and Faraday depths with their Kahan compensations.
template <typename R>
struct XLane {
    R S[4], Slo[4], eo1[4], eo2[4], u1[4], u2[4], a1[4], a2[4];
    R tau, tauc, phi, phic;
    bool basis;
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int i = 0; i < 4; i++) S[i] = Slo[i] = R(0);
        tau = tauc = phi = phic = R(0);
        basis = false;
    }
};

// One saved state (q0, q1) of the walk toward the camera: transport the screen legs to it,
// evaluate the plasma, and where it emits, re-project onto the fluid screen and take the
// exact constant-coefficient step. m returns the metric at the state. Returns whether the
// point emits.
// The surrogate's maps (surrogate.cuh) in the transfer's precision R, from the tetrad's sin and
// cos of the field angle (sth >= 0) instead of the angle, for the FP32 render: the prefactors are
// written as in the thermal fits (nu_B / nu and e^2 / (m c) grouped) so every intermediate
// stays within FP32 range.
template <typename R>
struct SurPrefR {
    R Pj, PjV, Pa, PaV, PrQ, PrV, sgn;
};

template <typename R>
__device__ __forceinline__ SurPrefR<R> sur_prefactors_r(R ne, R Te, R B, R nu, R sth, R cth) {
    typedef Mth<R> F;
    const R cB = R(kQe / (2.0 * kPi * kMe * kC));             // nu_B / B
    const R cQ2 = R(kQe * kQe / (kMe * kC));                  // e^2 / (m c)
    const R cJ = R(kQe * kQe / (2.0 * 1.7320508075688772 * kC));
    SurPrefR<R> p;
    R as = fabs(sth), ac = fabs(cth);
    R rb = cB * B / nu;
    R cot = as > R(0) ? ac / as : R(0);
    p.Pj = cJ * ne * nu / (Te * Te);
    p.PjV = p.Pj * (R(4) / (R(3) * Te)) * cot;
    p.Pa = cQ2 * ne / (R(4.0 * 1.7320508075688772) * nu * Te * Te * Te);
    p.PaV = p.Pa * cot;
    R X = Te * F::sqrt_(R(1.4142135623730951) * as * R(1e3) * rb);
    R f = shcherbakov_fX(X);
    p.PrQ = cQ2 * ne * rb * rb / nu * sth * sth * f;
    p.PrV = R(2) * cQ2 * ne * rb / nu * ac * (R(1) - R(0.11) * F::log1p_(R(0.035) * X));
    p.sgn = cth < R(0) ? R(-1) : R(1);
    return p;
}

template <typename R>
__device__ __forceinline__ void sur_features_r(R Te, R B, R nu, R sth, R cth, R kappa, float f[4]) {
    typedef Mth<R> F;
    const R cB = R(kQe / (2.0 * kPi * kMe * kC));
    R tf = F::atan2_(sth, fabs(cth));  // theta_B folded into [0, pi/2]
    f[0] = (float)(-F::log_(R(1.5) * cB * B / nu * sth * Te * Te));
    f[1] = (float)tf;
    f[2] = (float)F::log_(Te);
    f[3] = (float)kappa;
}

template <typename R>
__device__ __forceinline__ void sur_expand_r(const SurPrefR<R> &p, const float y[8], R c[8]) {
    typedef Mth<R> F;
    c[0] = p.Pj * F::exp_(R(y[0]));
    c[1] = p.Pj * F::exp_(R(y[1]));
    c[2] = p.sgn * p.PjV * F::exp_(R(y[2]));
    c[3] = p.Pa * F::exp_(R(y[3]));
    c[4] = p.Pa * F::exp_(R(y[4]));
    c[5] = p.sgn * p.PaV * F::exp_(R(y[5]));
    c[6] = p.PrQ * F::exp_(R(y[6]));
    c[7] = p.sgn * p.PrV * F::exp_(R(y[7]));
    R pj = F::sqrt_(c[1] * c[1] + c[2] * c[2]);
    if (pj > c[0] && pj > R(0)) {
        c[1] *= c[0] / pj;
        c[2] *= c[0] / pj;
    }
    R pa = F::sqrt_(c[4] * c[4] + c[5] * c[5]);
    if (pa > c[3] && pa > R(0)) {
        c[4] *= c[3] / pa;
        c[5] *= c[3] / pa;
    }
}

// Coefficients of an emitting point for kappa electrons: CM 1 by quadrature, CM 2 from the
// surrogate's outputs for this saved state (quadrature outside the network's box).
template <typename R, int CM>
__device__ __forceinline__ void kappa_point_coeffs(const XferArgs *pa, long long st, const Model &mdl,
                                                   const Plasma<R> &pl, R w, R sth, R cth, R nu_obs, R cf[8]) {
    typedef Mth<R> F;
    if (CM == 2) {  // the network, in R, inside its box
        float f[4], xn[4];
        sur_features_r<R>(pl.Te, pl.B, w * nu_obs, sth, cth, R(mdl.kappa), f);
        bool in = true;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float u = (f[j] - pa->sur_lo[j]) / (pa->sur_hi[j] - pa->sur_lo[j]);
            in &= u >= 0.0f && u <= 1.0f;
            xn[j] = 2.0f * u - 1.0f;
        }
        if (in) {
            float phi[kSurBasis], y[8];
            sur_basis(xn, phi);
            const long long row = pa->sur_row ? (long long)pa->sur_row[st] : st;
            const float *nm = pa->sur_norm, *yh = pa->sur_y + 8 * row;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                float b = 0.f;
                for (int q = 0; q < kSurBasis; q++) b += nm[16 + k * kSurBasis + q] * phi[q];
                y[k] = b + nm[k] + nm[8 + k] * yh[k];
            }
            sur_expand_r<R>(sur_prefactors_r<R>(pl.ne, pl.Te, pl.B, w * nu_obs, sth, cth), y, cf);
            if (!(cf[0] > F::jflush))
#pragma unroll
                for (int k = 0; k < 6; k++) cf[k] = R(0);
            return;
        }
    }
    // quadrature (CM 1, or CM 2 outside the network's box), in FP64: the exact grade for the
    // FP64 form, the tabulated one for the FP32 forms
    double thB = atan2((double)sth, (double)cth), nu = (double)(w * nu_obs);
    double cd[8];
    kappa_coeffs_quad<sizeof(R) == 8>(pa->kt, (double)pl.ne, (double)pl.Te, (double)pl.B, nu, thB, mdl.kappa, cd);
#pragma unroll
    for (int k = 0; k < 8; k++) cf[k] = R(cd[k]);
    if (!(cf[0] > F::jflush))  // as for the thermal fits: no relative precision left
#pragma unroll
        for (int k = 0; k < 6; k++) cf[k] = R(0);
}

// pre (optional): the grid cell of this state and its interpolated primitives, fetched by the
// caller (the staged transfer); a null cell pointer means the state lies outside the grid.
template <typename R>
struct PreFetch {
    const GridCell<R> *cell;
    const R *P;
};

template <typename R, int CM = 0, bool PRE = false>
__device__ __forceinline__ bool xfer_point(const Camera &c, const Model &mdl, const double4_32a &q0,
                                           const double4_32a &q1, const R *sgw, XLane<R> &Ln, KS<R> &m,
                                           const XferArgs *pa = nullptr, long long st = 0,
                                           PreFetch<R> pre = PreFetch<R>{nullptr, nullptr}) {
    const R a = pick<R>(c.a, c.f_a);
    R r = to_real<R>(q0.x), th = to_real<R>(q0.y), ph = to_real<R>(q0.z);
    R K[4] = {to_real<R>(q0.w), to_real<R>(q1.x), to_real<R>(q1.y), to_real<R>(q1.z)};
    R hs = to_real<R>(q1.w);
    R h = fabs(hs);
    m.eval(a, r, th);
    if (Ln.basis && hs < R(0)) {  // that step crossed the polar axis: bring n+1 into this chart
        Ln.eo1[2] = -Ln.eo1[2];
        Ln.eo2[2] = -Ln.eo2[2];
        Ln.u1[2] = -Ln.u1[2];
        Ln.u2[2] = -Ln.u2[2];
        Ln.a1[2] = -Ln.a1[2];
        Ln.a2[2] = -Ln.a2[2];
    }
    Plasma<R> pl;
    if (PRE) {
        pl.valid = false;
        if (pre.cell) grid_state(mdl.grid, m, *pre.cell, pre.P, pl);
    } else if (mdl.kind == 1) {
        adaf_plasma(mdl.adaf, a, m, r, pl);
    } else {
        grid_plasma(mdl.grid, m, q0.x, q0.y, q0.z, pl);
    }
    R e1[4], e2[4], w, sth, cth;
    if (pl.valid) fluid_tetrad(m, K, pl.u, pl.b, e1, e2, w, sth, cth);
    if (Ln.basis || pl.valid) {
        // transport the legs from n+1 to n, then T E at n for the next step
        R T0[4][4];
        connection_T(m, K, T0);
        if (Ln.basis) {
            heun_leg(Ln.eo1, Ln.u1, Ln.a1, T0, h);
            heun_leg(Ln.eo2, Ln.u2, Ln.a2, T0, h);
        }
        R E1[4], E2[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            E1[i] = pl.valid ? e1[i] : Ln.eo1[i] + Ln.u1[i];
            E2[i] = pl.valid ? e2[i] : Ln.eo2[i] + Ln.u2[i];
        }
        matvec4(T0, E1, Ln.a1);
        matvec4(T0, E2, Ln.a2);
    }
    if (pl.valid) {
        if (Ln.basis) {
            R l1[4], l2[4];
            m.lower(e1, l1);
            m.lower(e2, l2);
            reproject_comp(l1, l2, e1, e2, Ln.eo1, Ln.eo2, Ln.u1, Ln.u2, Ln.S, Ln.Slo);
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            Ln.eo1[i] = e1[i];
            Ln.eo2[i] = e2[i];
            Ln.u1[i] = Ln.u2[i] = R(0);
        }
        R cf[8];
        if (CM == 0)
            thermal_coeffs(pl.ne, pl.Te, pl.B, w * pick<R>(c.nu_obs, c.f_nu_obs), sth, cth, sgw, cf);
        else
            kappa_point_coeffs<R, CM>(pa, st, mdl, pl, w, sth, cth, pick<R>(c.nu_obs, c.f_nu_obs), cf);
        // invariant form: S holds I/nu^3, so the step takes J/w^3 and the same M
        R ds = w * h * pick<R>(c.L_unit, c.f_L_unit);
        substep(cf, ds, R(1) / (w * w * w), Ln.S, Ln.Slo);
        kahan_add(Ln.tau, Ln.tauc, cf[3] * ds);
        kahan_add(Ln.phi, Ln.phic, cf[7] * ds);
        Ln.basis = true;
    }
    return pl.valid;
}

// At the camera (the last state, metric m): project onto the image basis and write pixel
// (ix, iy) of out (and of depth, if given).
template <typename R, typename OutT>
__device__ __forceinline__ void xfer_finish(const Camera &c, const KS<R> &m, int ix, int iy, XLane<R> &Ln,
                                            void *out, void *depth) {
#pragma unroll
    for (int i = 0; i < 4; i++) Ln.S[i] += Ln.Slo[i];
    if (Ln.basis) {
        // camera screen: x along e_phi, y along -e_theta, each normal to the ray
        R X[4], Y[4];
        if constexpr (sizeof(R) == 4) {
            // the FP32 form: the camera frame from the host (c.f_e), the sky direction in float,
            // with no FP64 instruction (this runs once per ray, on a lane of its own)
            float px = (i2f_small(ix) + 0.5f) * c.f_pix - 0.5f * (c.f_pix * i2f_small(c.nx));
            float py = (i2f_small(iy) + 0.5f) * c.f_pix - 0.5f * (c.f_pix * i2f_small(c.ny));
            float al = px / c.f_r_cam, be = py / c.f_r_cam;
            float n = rsqrtf(1.0f + al * al + be * be);
            float s[3] = {-n, -be * n, al * n};
            float xh[3] = {-s[2] * s[0], -s[2] * s[1], 1.0f - s[2] * s[2]};
            float nx = rsqrtf(xh[0] * xh[0] + xh[1] * xh[1] + xh[2] * xh[2]);
            float yh[3] = {s[1] * s[0], -1.0f + s[1] * s[1], s[1] * s[2]};
#pragma unroll
            for (int k = 0; k < 3; k++) xh[k] *= nx;
            float yx = yh[0] * xh[0] + yh[1] * xh[1] + yh[2] * xh[2];
#pragma unroll
            for (int k = 0; k < 3; k++) yh[k] -= yx * xh[k];
            float ny = rsqrtf(yh[0] * yh[0] + yh[1] * yh[1] + yh[2] * yh[2]);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                X[mu] = xh[0] * c.f_e[0][mu] + xh[1] * c.f_e[1][mu] + xh[2] * c.f_e[2][mu];
                Y[mu] = ny * (yh[0] * c.f_e[0][mu] + yh[1] * c.f_e[1][mu] + yh[2] * c.f_e[2][mu]);
            }
        } else {
            const double(&e)[4][4] = c.e;
            double s[3];
            sky_direction(c, ix, iy, s);
            double xh[3] = {-s[2] * s[0], -s[2] * s[1], 1.0 - s[2] * s[2]};
            double nx = rsqrt(xh[0] * xh[0] + xh[1] * xh[1] + xh[2] * xh[2]);
            double yh[3] = {s[1] * s[0], -1.0 + s[1] * s[1], s[1] * s[2]};
            double yx = yh[0] * xh[0] * nx + yh[1] * xh[1] * nx + yh[2] * xh[2] * nx;
            for (int k = 0; k < 3; k++) {
                xh[k] *= nx;
                yh[k] -= yx * xh[k];
            }
            double ny = rsqrt(yh[0] * yh[0] + yh[1] * yh[1] + yh[2] * yh[2]);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                X[mu] = R(xh[0] * e[1][mu] + xh[1] * e[2][mu] + xh[2] * e[3][mu]);
                Y[mu] = R(ny * (yh[0] * e[1][mu] + yh[1] * e[2][mu] + yh[2] * e[3][mu]));
            }
        }
        R lx[4], ly[4], E1[4], E2[4];
        m.lower(X, lx);
        m.lower(Y, ly);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            E1[i] = Ln.eo1[i] + Ln.u1[i];
            E2[i] = Ln.eo2[i] + Ln.u2[i];
        }
        reproject(lx, ly, E1, E2, Ln.S);
    }
    long long pix = (long long)iy * c.nx + ix;
    OutT *o = reinterpret_cast<OutT *>(out) + 4 * pix;
    o[0] = OutT(Ln.S[0]);
    o[1] = OutT(Ln.S[1]);
    o[2] = OutT(Ln.S[2]);
    o[3] = OutT(Ln.S[3]);
    if (depth) {
        OutT *d = reinterpret_cast<OutT *>(depth) + 2 * pix;
        d[0] = OutT(Ln.tau - Ln.tauc);
        d[1] = OutT(Ln.phi - Ln.phic);
    }
}

// A pixel whose ray has no usable path: zero Stokes (and depths).
template <typename OutT>
__device__ __forceinline__ void xfer_zero(long long pix, void *out, void *depth) {
    OutT *o = reinterpret_cast<OutT *>(out) + 4 * pix;
    o[0] = o[1] = o[2] = o[3] = OutT(0);
    if (depth) {
        OutT *d = reinterpret_cast<OutT *>(depth) + 2 * pix;
        d[0] = d[1] = OutT(0);
    }
}

// Bessel-quadrature weights exp(-(k h)^2) (halved at k = 0) into shared memory.
template <typename R>
__device__ __forceinline__ void fill_bessel_weights(R *sgw) {
    typedef Mth<R> F;
    if (threadIdx.x < BesselCfg<R>::nq) {
        R u = R(threadIdx.x) * BesselCfg<R>::h;
        sgw[threadIdx.x] = F::exp_(-u * u) * (threadIdx.x == 0 ? R(0.5) : R(1));
    }
}

// JOBS: the rays run over a table of images (p.jobs), each with its own camera, model and
// outputs; otherwise over the one image of p.cam, p.model, p.out.
template <typename R, typename OutT, int CM = 0, bool JOBS = false>
__global__ void __launch_bounds__(kXferThreads, sizeof(R) == 4 ? 4 : 1) transfer_kernel(XferArgs p) {
    __shared__ R sgw[32];
    fill_bessel_weights(sgw);
    __syncthreads();
    long long ray = -1;
    int blk = -1, slot = 0, n = 0, rstat = 0, job = 0;
    bool live = false, drained = false;
    XLane<R> Ln;
    unsigned long long my_pts = 0, my_emit = 0;
    // this ray's image: pixel, and (JOBS) the job's camera, model and outputs
    auto gid_of = [&](long long r) { return p.pix_list ? (long long)p.pix_list[r + p.ray_offset] : r + p.ray_offset; };
    auto pixel = [&](int &ix, int &iy) {
        if (JOBS) {
            const JobDev &J = p.jobs[job];
            ray_pixel(gid_of(ray) - J.ray_begin, J.cam.nx, J.cam.ny, ix, iy);
        } else {
            map_pixel(p.pix_list, ray + p.ray_offset, p.cam.nx, p.cam.ny, ix, iy);
        }
    };
    for (;;) {
        bool want = !live && !drained;
        unsigned long long t = warp_pop(&p.ctr->xfer_next, want);
        if (want) {
            if (t < (unsigned long long)p.nrays) {
                ray = (long long)t;
                if (JOBS) job = find_job(p.jobs, p.njobs, gid_of(ray));
                RayRecord rec = p.rec[ray];
                rstat = rec.status;
                if (rec.nstates >= 2) {
                    blk = rec.last_block;
                    slot = (rec.nstates - 1) % kBlockStates;
                    n = rec.nstates - 1;
                    Ln.reset();
                    live = true;
                } else {
                    int ix, iy;
                    pixel(ix, iy);
                    const Camera &c = JOBS ? p.jobs[job].cam : p.cam;
                    void *out = JOBS ? p.jobs[job].out : p.out, *depth = JOBS ? p.jobs[job].depth : p.depth;
                    uint8_t *status = JOBS ? p.jobs[job].status : p.status;
                    long long pix = (long long)iy * c.nx + ix;
                    xfer_zero<OutT>(pix, out, depth);
                    if (status) status[pix] = (uint8_t)rstat;
                }
            } else {
                drained = true;
            }
        }
        if (__all_sync(0xffffffffu, !live && drained)) break;
        if (!live) continue;

        // move from state n to state n-1
        if (--slot < 0) {
            blk = p.arena.prev[blk];
            slot = kBlockStates - 1;
        }
        n--;
        const double4_32a *src = reinterpret_cast<const double4_32a *>(p.arena.states + (long long)blk * kBlockStates + slot);
        double4_32a q0 = src[0], q1 = src[1];
        KS<R> m;
        const Camera &c = JOBS ? p.jobs[job].cam : p.cam;
        const Model &mdl = JOBS ? p.jobs[job].model : p.model;
        if (xfer_point<R, CM>(c, mdl, q0, q1, sgw, Ln, m, &p, (long long)blk * kBlockStates + slot)) my_emit++;
        my_pts++;
        if (n == 0) {
            int ix, iy;
            pixel(ix, iy);
            void *out = JOBS ? p.jobs[job].out : p.out, *depth = JOBS ? p.jobs[job].depth : p.depth;
            uint8_t *status = JOBS ? p.jobs[job].status : p.status;
            xfer_finish<R, OutT>(c, m, ix, iy, Ln, out, depth);
            if (status) status[(long long)iy * c.nx + ix] = (uint8_t)rstat;
            live = false;
        }
    }
    if (my_pts) atomicAdd(&p.ctr->points, my_pts);
    if (my_emit) atomicAdd(&p.ctr->emitting, my_emit);
}

// ---- The grid fetch staged through shared memory by TMA (FP32 form, thermal electrons) ----
// Each lane owns a 256-byte slot of shared memory and an mbarrier. While it works on one saved
// state, the 2 x 2 x 2 cells of the next state's trilinear stencil are copied into its slot by
// one TMA tensor load: a box of 8 floats x 2 x 2 x 2 cells of the grid seen as a 4-d tensor
// [n1][n2][n3][8]. The fetch's latency then hides behind a whole point of work, and the eight
// 32-byte gathers leave the load/store path. At the periodic seam in phi (k1 = 0) the two
// k cells are not adjacent in memory, and the lane copies that stencil with plain loads. The
// interpolation takes the cells in grid_interp's order, so the image is the same bit for bit.

// TMA: the box of the 4-d tensor map at coordinates (c0, c1, c2, c3), innermost first, into
// shared memory at dst, counted on the mbarrier bar's transaction bytes.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Arrive on bar (this thread's one arrival) and expect bytes more of transactions.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// The staged cells of one state in grid_interp's order: cell (di, dj, dk) at float4
// ((di 2 + dj) 2 + dk) 2 (and + 1).
template <typename R>
__device__ __forceinline__ void grid_interp_staged(const GridCell<R> &c, const float4 *s, R P[8]) {
#pragma unroll
    for (int q = 0; q < 8; q++) P[q] = R(0);
#pragma unroll
    for (int di = 0; di < 2; di++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++) {
            R wij = (di ? c.w1 : R(1) - c.w1) * (dj ? c.w2 : R(1) - c.w2);
#pragma unroll
            for (int dk = 0; dk < 2; dk++) {
                R wt = wij * (dk ? c.w3 : R(1) - c.w3);
                const int o = ((di * 2 + dj) * 2 + dk) * 2;
                float4 lo = s[o], hi = s[o + 1];
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

// CM: the coefficients (0: thermal fits; the only one staged so far)
template <int CM = 0>
__global__ void __launch_bounds__(kXferThreads, 4) transfer_kernel_staged(XferArgs p, const __grid_constant__ CUtensorMap tmap) {
    typedef float R;
    __shared__ R sgw[32];
    __shared__ __align__(128) float4 stc[kXferThreads * 16];
    __shared__ __align__(8) unsigned long long bars[kXferThreads];
    fill_bessel_weights(sgw);
    const uint32_t bar = smem_u32(&bars[threadIdx.x]);
    float4 *slot_s = stc + threadIdx.x * 16;
    const uint32_t slot_a = smem_u32(slot_s);
    mbar_init(bar, 1);
    __syncthreads();
    const GridModel &g = p.model.grid;
    long long ray = -1;
    int blk = -1, slot = 0, n = 0, rstat = 0;
    bool live = false, drained = false, failed = false;
    XLane<R> Ln;
    unsigned long long my_pts = 0, my_emit = 0;
    uint32_t phase = 0;
    // the next state's cell, and where its stencil is: 0 nowhere (outside the grid), 1 in
    // flight (TMA), 2 in the slot (plain loads at the seam)
    GridCell<R> nc;
    int nmode = 0;
    auto stage = [&](int b, int s) {
        const double4_32a q = *reinterpret_cast<const double4_32a *>(p.arena.states + (long long)b * kBlockStates + s);
        nmode = 0;
        if (!grid_cell<R>(g, q.x, q.y, q.z, nc)) return;
        if (nc.k1 != 0) {
            fence_smem_async();  // the slot's last reads (generic proxy) before the TMA's writes
            mbar_expect_tx(bar, 16 * sizeof(float4));
            tma_load_4d(slot_a, &tmap, 0, nc.k0, nc.j0, nc.i0, bar);
            nmode = 1;
        } else {
#pragma unroll
            for (int di = 0; di < 2; di++)
#pragma unroll
                for (int dj = 0; dj < 2; dj++) {
                    long long row = ((long long)(nc.i0 + di) * g.n2 + (nc.j0 + dj)) * g.n3;
#pragma unroll
                    for (int dk = 0; dk < 2; dk++) {
                        long long cell = row + (dk ? nc.k1 : nc.k0);
                        const int o = ((di * 2 + dj) * 2 + dk) * 2;
                        slot_s[o] = __ldg(g.prims + 2 * cell);
                        slot_s[o + 1] = __ldg(g.prims + 2 * cell + 1);
                    }
                }
            nmode = 2;
        }
    };
    // the state after (b, s) on the walk toward the camera
    auto step_back = [&](int &b, int &s) {
        if (--s < 0) {
            b = p.arena.prev[b];
            s = kBlockStates - 1;
        }
    };
    for (;;) {
        bool want = !live && !drained;
        unsigned long long t = warp_pop(&p.ctr->xfer_next, want);
        if (want) {
            if (t < (unsigned long long)p.nrays) {
                ray = (long long)t;
                RayRecord rec = p.rec[ray];
                rstat = rec.status;
                if (rec.nstates >= 2) {
                    blk = rec.last_block;
                    slot = (rec.nstates - 1) % kBlockStates;
                    n = rec.nstates - 1;
                    Ln.reset();
                    live = true;
                    int b1 = blk, s1 = slot;
                    step_back(b1, s1);
                    stage(b1, s1);
                } else {
                    int ix, iy;
                    map_pixel(p.pix_list, ray + p.ray_offset, p.cam.nx, p.cam.ny, ix, iy);
                    long long pix = (long long)iy * p.cam.nx + ix;
                    xfer_zero<R>(pix, p.out, p.depth);
                    if (p.status) p.status[pix] = (uint8_t)rstat;
                }
            } else {
                drained = true;
            }
        }
        if (__all_sync(0xffffffffu, !live && drained)) break;
        if (!live) continue;

        step_back(blk, slot);
        n--;
        const double4_32a *src = reinterpret_cast<const double4_32a *>(p.arena.states + (long long)blk * kBlockStates + slot);
        double4_32a q0 = src[0], q1 = src[1];
        // this state's primitives from the slot, then the next state's stencil into it
        const GridCell<R> cc = nc;
        const int cmode = nmode;
        R P[8];
        if (cmode == 1 && !failed) {
            if (mbar_wait(bar, phase))
                phase ^= 1u;
            else
                failed = true;  // the copy is still owed on this phase
        }
        if (cmode != 0) grid_interp_staged(cc, slot_s, P);
        if (n > 0 && !failed) {
            int b1 = blk, s1 = slot;
            step_back(b1, s1);
            stage(b1, s1);
        } else {
            nmode = 0;
        }
        KS<R> m;
        PreFetch<R> pre{cmode != 0 && !failed ? &cc : nullptr, P};
        if (xfer_point<R, CM, true>(p.cam, p.model, q0, q1, sgw, Ln, m, &p, 0, pre)) my_emit++;
        my_pts++;
        if (n == 0) {
            int ix, iy;
            map_pixel(p.pix_list, ray + p.ray_offset, p.cam.nx, p.cam.ny, ix, iy);
            xfer_finish<R, R>(p.cam, m, ix, iy, Ln, p.out, p.depth);
            if (p.status) p.status[(long long)iy * p.cam.nx + ix] = (uint8_t)rstat;
            live = false;
        }
    }
    if (failed) {  // report, and give the copy in flight (bounded) time to land before exit
        atomicAdd(&p.ctr->n_status[kStageStatus], 1u);
        mbar_wait(bar, phase);
    }
    if (my_pts) atomicAdd(&p.ctr->points, my_pts);
    if (my_emit) atomicAdd(&p.ctr->emitting, my_emit);
}

// The surrogate form's features pass: walk each ray's saved states as the transfer will and
// write, for every emitting state, the network's normalised inputs (f mapped from the box to
// [-1, 1]); other states get zeros. Same arithmetic as the transfer's own feature evaluation.
template <typename R>
__global__ void __launch_bounds__(kXferThreads) sur_features_pass(XferArgs p) {
    const Camera &c = p.cam;
    const R a = pick<R>(c.a, c.f_a), nu_obs = pick<R>(c.nu_obs, c.f_nu_obs);
    long long ray = -1, row = 0;
    int blk = -1, slot = 0, n = 0;
    bool live = false, drained = false;
    for (;;) {
        bool want = !live && !drained;
        unsigned long long t = warp_pop(&p.ctr->feat_next, want);
        if (want) {
            if (t < (unsigned long long)p.nrays) {
                ray = (long long)t;
                RayRecord rec = p.rec[ray];
                if (rec.nstates >= 2) {
                    blk = rec.last_block;
                    slot = (rec.nstates - 1) % kBlockStates;
                    n = rec.nstates - 1;
                    live = true;
                    // compact rows: the ray's n states take n consecutive rows
                    if (p.sur_row) row = (long long)atomicAdd(&p.ctr->sur_rows, (unsigned long long)n);
                }
            } else {
                drained = true;
            }
        }
        if (__all_sync(0xffffffffu, !live && drained)) break;
        if (!live) continue;
        if (--slot < 0) {
            blk = p.arena.prev[blk];
            slot = kBlockStates - 1;
        }
        n--;
        const double4_32a *src = reinterpret_cast<const double4_32a *>(p.arena.states + (long long)blk * kBlockStates + slot);
        double4_32a q0 = src[0], q1 = src[1];
        R r = to_real<R>(q0.x), th = to_real<R>(q0.y), ph = to_real<R>(q0.z);
        R K[4] = {to_real<R>(q0.w), to_real<R>(q1.x), to_real<R>(q1.y), to_real<R>(q1.z)};
        KS<R> m;
        m.eval(a, r, th);
        Plasma<R> pl;
        if (p.model.kind == 1)
            adaf_plasma(p.model.adaf, a, m, r, pl);
        else
            grid_plasma(p.model.grid, m, q0.x, q0.y, q0.z, pl);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pl.valid) {
            R e1[4], e2[4], w, sth, cth;
            fluid_tetrad(m, K, pl.u, pl.b, e1, e2, w, sth, cth);
            float f[4], xn[4];
            sur_features_r<R>(pl.Te, pl.B, w * nu_obs, sth, cth, R(p.model.kappa), f);
            if (p.feat_raw) {
                unsigned long long k = atomicAdd(&p.ctr->feat_count, 1ull);
                if ((long long)k < p.feat_cap) p.feat_raw[k] = make_float4(f[0], f[1], f[2], f[3]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) xn[j] = 2.0f * (f[j] - p.sur_lo[j]) / (p.sur_hi[j] - p.sur_lo[j]) - 1.0f;
            o = make_float4(xn[0], xn[1], xn[2], xn[3]);
        }
        if (p.sur_row) {
            p.feat[row + n] = o;
            p.sur_row[(long long)blk * kBlockStates + slot] = (int)(row + n);
        } else if (p.feat) {
            p.feat[(long long)blk * kBlockStates + slot] = o;
        }
        if (n == 0) live = false;
    }
}

// The unpolarized transfer (Stokes I only, for fitting loops): I/nu^3 is a scalar invariant,
// so nothing is transported. At each emitting point: the pitch angle from scalar products
// (the ray's fluid-frame direction is -K - w u, b is spatial in that frame), j_I and a_I, and the
// exact step I <- I e^-tau + (j ds / w^3) (1 - e^-tau)/tau, added as the increment
// (J - tau I) (1 - e^-tau)/tau with TwoSum compensation. Output: one value per pixel.
template <typename R, bool JOBS = false>
__global__ void __launch_bounds__(kXferThreads, 4) unpol_kernel(XferArgs p) {
    typedef Mth<R> F;
    // the ray's camera constants: p.cam's, or (JOBS) its image's
    R a = pick<R>(p.cam.a, p.cam.f_a), nu_obs = pick<R>(p.cam.nu_obs, p.cam.f_nu_obs),
      L = pick<R>(p.cam.L_unit, p.cam.f_L_unit);
    long long ray = -1;
    int blk = -1, slot = 0, n = 0, rstat = 0, job = 0;
    bool live = false, drained = false;
    R I = 0, Ilo = 0;
    unsigned long long my_pts = 0, my_emit = 0;
    auto gid_of = [&](long long r) { return p.pix_list ? (long long)p.pix_list[r + p.ray_offset] : r + p.ray_offset; };
    // this ray's pixel index and its image's outputs
    auto target = [&](long long &pix, R *&out, uint8_t *&status) {
        int ix, iy;
        if (JOBS) {
            const JobDev &J = p.jobs[job];
            ray_pixel(gid_of(ray) - J.ray_begin, J.cam.nx, J.cam.ny, ix, iy);
            pix = (long long)iy * J.cam.nx + ix;
            out = reinterpret_cast<R *>(J.out);
            status = J.status;
        } else {
            map_pixel(p.pix_list, ray + p.ray_offset, p.cam.nx, p.cam.ny, ix, iy);
            pix = (long long)iy * p.cam.nx + ix;
            out = reinterpret_cast<R *>(p.out);
            status = p.status;
        }
    };
    for (;;) {
        bool want = !live && !drained;
        unsigned long long t = warp_pop(&p.ctr->xfer_next, want);
        if (want) {
            if (t < (unsigned long long)p.nrays) {
                ray = (long long)t;
                if (JOBS) {
                    job = find_job(p.jobs, p.njobs, gid_of(ray));
                    const Camera &cj = p.jobs[job].cam;
                    a = pick<R>(cj.a, cj.f_a);
                    nu_obs = pick<R>(cj.nu_obs, cj.f_nu_obs);
                    L = pick<R>(cj.L_unit, cj.f_L_unit);
                }
                RayRecord rec = p.rec[ray];
                rstat = rec.status;
                if (rec.nstates >= 2) {
                    blk = rec.last_block;
                    slot = (rec.nstates - 1) % kBlockStates;
                    n = rec.nstates - 1;
                    I = Ilo = R(0);
                    live = true;
                } else {
                    long long pix;
                    R *out;
                    uint8_t *status;
                    target(pix, out, status);
                    out[pix] = R(0);
                    if (status) status[pix] = (uint8_t)rstat;
                }
            } else {
                drained = true;
            }
        }
        if (__all_sync(0xffffffffu, !live && drained)) break;
        if (!live) continue;
        if (--slot < 0) {
            blk = p.arena.prev[blk];
            slot = kBlockStates - 1;
        }
        n--;
        const double4_32a *src = reinterpret_cast<const double4_32a *>(p.arena.states + (long long)blk * kBlockStates + slot);
        double4_32a q0 = src[0], q1 = src[1];
        R r = to_real<R>(q0.x), th = to_real<R>(q0.y), ph = to_real<R>(q0.z);
        R K[4] = {to_real<R>(q0.w), to_real<R>(q1.x), to_real<R>(q1.y), to_real<R>(q1.z)};
        R h = fabs(to_real<R>(q1.w));
        KS<R> m;
        m.eval(a, r, th);
        Plasma<R> pl;
        const Model &mdl = JOBS ? p.jobs[job].model : p.model;
        if (mdl.kind == 1)
            adaf_plasma(mdl.adaf, a, m, r, pl);
        else
            grid_plasma(mdl.grid, m, q0.x, q0.y, q0.z, pl);
        if (pl.valid) {
            R w = m.dot(K, pl.u);
            R kp[4], bn[4];
            R bs = fmax(fmax(fabs(pl.b[0]), fabs(pl.b[1])), fmax(fabs(pl.b[2]), fabs(pl.b[3])));
            R ibs = bs > R(0) ? R(1) / bs : R(0);
#pragma unroll
            for (int i = 0; i < 4; i++) {
                kp[i] = -K[i] - w * pl.u[i];
                bn[i] = pl.b[i] * ibs;
            }
            R bb = m.dot(bn, bn), kk = m.dot(kp, kp), bk = m.dot(bn, kp);
            R sth = (bb > R(0) && kk > R(0)) ? F::sqrt_(fmax(bb - bk * bk / kk, R(0)) / bb) : R(0);
            R jI, aI;
            thermal_jI_aI(pl.ne, pl.Te, pl.B, w * nu_obs, sth, jI, aI);
            R ds = w * h * L, tau = aI * ds;
            R J = jI * ds / (w * w * w);
            two_sum_add(I, Ilo, (J - tau * I) * phi1(tau));
            my_emit++;
        }
        my_pts++;
        if (n == 0) {
            long long pix;
            R *out;
            uint8_t *status;
            target(pix, out, status);
            out[pix] = I + Ilo;
            if (status) status[pix] = (uint8_t)rstat;
            live = false;
        }
    }
    if (my_pts) atomicAdd(&p.ctr->points, my_pts);
    if (my_emit) atomicAdd(&p.ctr->emitting, my_emit);
}

}  // namespace prt
