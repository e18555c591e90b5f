// The transfer kernel (persistent, one ray per lane, per-lane refill from a work queue). Each
// lane walks its ray's saved states from the far end back to the camera. At every state it
// parallel-transports the screen legs (Heun, connection from the saved K), evaluates the
// plasma, and if the point emits it projects onto the fluid screen and takes the exact
// constant-coefficient step. Instantiated for the FP64 and the mixed (FP32 transfer) forms.
#pragma once
#include "transfer.cuh"

namespace prt {

// double -> float rounded to nearest even with integer operations only, so the FP32 form
// reads the FP64 path without using the FP64 pipe. Magnitudes below the float normal range
// become signed zero; above it, infinity.
__device__ __forceinline__ float d2f_int(double d) {
    unsigned long long x = (unsigned long long)__double_as_longlong(d);
    unsigned hi = (unsigned)(x >> 32), lo = (unsigned)x;
    unsigned sign = hi & 0x80000000u;
    int fe = (int)((hi >> 20) & 0x7ffu) - 896;
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
    unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned rem = lo & 0x1fffffffu;
    unsigned f = sign | ((unsigned)fe << 23) | mant;
    f += (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & (mant & 1u));
    return __uint_as_float(f);
}

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

template <typename R>
__device__ __forceinline__ void heun_transport(R E[4], const R T1[4][4], const R T0[4][4], R h) {
    R a[4], v[4];
#pragma unroll
    for (int m = 0; m < 4; m++) a[m] = T1[m][0] * E[0] + T1[m][1] * E[1] + T1[m][2] * E[2] + T1[m][3] * E[3];
#pragma unroll
    for (int m = 0; m < 4; m++) v[m] = E[m] + h * a[m];
    R hh = R(0.5) * h;
#pragma unroll
    for (int m = 0; m < 4; m++)
        E[m] += hh * (a[m] + T0[m][0] * v[0] + T0[m][1] * v[1] + T0[m][2] * v[2] + T0[m][3] * v[3]);
}

// Stokes (I, Q, U, V) in the screen (E1, E2) re-expressed on the screen (f1, f2) given as
// lowered legs: n' = C n C^T, C_{ij} = f_i . E_j.
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

template <typename R, typename OutT>
__global__ void __launch_bounds__(kXferThreads, sizeof(R) == 4 ? 4 : 1) transfer_kernel(XferArgs p) {
    typedef Mth<R> F;
    __shared__ R sgw[32];
    if (threadIdx.x < BesselCfg<R>::nq) {
        R u = R(threadIdx.x) * BesselCfg<R>::h;
        sgw[threadIdx.x] = F::exp_(-u * u) * (threadIdx.x == 0 ? R(0.5) : R(1));
    }
    __syncthreads();
    const Camera &c = p.cam;
    const R a = R(c.a);
    const R nu_obs = R(c.nu_obs), L = R(c.L_unit);
    long long ray = -1;
    int blk = -1, slot = 0, n = 0, rstat = 0;
    bool live = false, drained = false, basis = false;
    R S[4], E1[4], E2[4], T1[4][4];
    unsigned long long my_pts = 0, my_emit = 0;
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
                    basis = false;
#pragma unroll
                    for (int i = 0; i < 4; i++) S[i] = R(0);
                    live = true;
                } else {
                    int ix, iy;
                    ray_pixel(ray + p.ray_offset, c.nx, c.ny, ix, iy);
                    long long pix = (long long)iy * c.nx + ix;
                    OutT *o = reinterpret_cast<OutT *>(p.out) + 4 * pix;
                    o[0] = o[1] = o[2] = o[3] = OutT(0);
                    if (p.status) p.status[pix] = (uint8_t)rstat;
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
        R r = to_real<R>(q0.x), th = to_real<R>(q0.y), ph = to_real<R>(q0.z);
        R K[4] = {to_real<R>(q0.w), to_real<R>(q1.x), to_real<R>(q1.y), to_real<R>(q1.z)};
        R hs = to_real<R>(q1.w);
        R h = fabs(hs);
        KS<R> m;
        m.eval(a, r, th);
        if (basis) {
            if (hs < R(0)) {  // that step crossed the polar axis: bring n+1 into this chart
                E1[2] = -E1[2];
                E2[2] = -E2[2];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if ((i == 2) != (j == 2)) T1[i][j] = -T1[i][j];
            }
            R T0[4][4];
            connection_T(m, K, T0);
            heun_transport(E1, T1, T0, h);
            heun_transport(E2, T1, T0, h);
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) T1[i][j] = T0[i][j];
        }
        Plasma<R> pl;
        if (p.model.kind == 1)
            adaf_plasma(p.model.adaf, a, m, r, pl);
        else
            grid_plasma(p.model.grid, m, r, th, ph, pl);
        if (pl.valid) {
            R e1[4], e2[4], w, sth, cth;
            fluid_tetrad(m, K, pl.u, pl.b, e1, e2, w, sth, cth);
            if (basis) {
                R l1[4], l2[4];
                m.lower(e1, l1);
                m.lower(e2, l2);
                reproject(l1, l2, E1, E2, S);
            }
            R cf[8];
            thermal_coeffs(pl.ne, pl.Te, pl.B, w * nu_obs, sth, cth, sgw, cf);
            R w3 = w * w * w, iw3 = R(1) / w3;
#pragma unroll
            for (int i = 0; i < 4; i++) S[i] *= w3;
            substep(cf, w * h * L, S);
#pragma unroll
            for (int i = 0; i < 4; i++) {
                S[i] *= iw3;
                E1[i] = e1[i];
                E2[i] = e2[i];
            }
            if (!basis) {
                connection_T(m, K, T1);
                basis = true;
            }
            my_emit++;
        }
        my_pts++;
        if (n == 0) {
            int ix, iy;
            ray_pixel(ray + p.ray_offset, c.nx, c.ny, ix, iy);
            if (basis) {
                // camera screen: x along e_phi, y along -e_theta, each normal to the ray
                double e[4][4], s[3];
                camera_tetrad(c.a, c.r_cam, c.theta_o, e);
                sky_direction(c, ix, iy, s);
                double xh[3] = {-s[2] * s[0], -s[2] * s[1], 1.0 - s[2] * s[2]};
                double nx = rsqrt(xh[0] * xh[0] + xh[1] * xh[1] + xh[2] * xh[2]);
                double yh[3] = {s[1] * s[0], -1.0 + s[1] * s[1], s[1] * s[2]};
                double yx = yh[0] * xh[0] * nx + yh[1] * xh[1] * nx + yh[2] * xh[2] * nx;
                R X[4], Y[4];
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
                R lx[4], ly[4];
                m.lower(X, lx);
                m.lower(Y, ly);
                reproject(lx, ly, E1, E2, S);
            }
            long long pix = (long long)iy * c.nx + ix;
            OutT *o = reinterpret_cast<OutT *>(p.out) + 4 * pix;
            o[0] = OutT(S[0]);
            o[1] = OutT(S[1]);
            o[2] = OutT(S[2]);
            o[3] = OutT(S[3]);
            if (p.status) p.status[pix] = (uint8_t)rstat;
            live = false;
        }
    }
    if (my_pts) atomicAdd(&p.ctr->points, my_pts);
    if (my_emit) atomicAdd(&p.ctr->emitting, my_emit);
}

}  // namespace prt
