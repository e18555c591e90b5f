// Backward null-geodesic integration from the camera (the paper's Section 2.1: one photon
// per pixel, integrated away from the observer and saved).
//
// Persistent kernel, one ray per lane. A lane whose ray stops takes the next ray from a
// global queue (warp-aggregated atomics), so long photon-ring rays do not hold a warp's
// other lanes idle. Every state is written to a block arena, 64 B per state: each lane
// writes two full 32 B sectors. The FP64 pipe bounds this kernel.
#include "camera.cuh"
#include "rt_kernels.cuh"

namespace prt {

// h = eps / (|K^r|/r + |K^th|/tt + |K^ph| + 1e-40), tt = max(min(th, pi - th), 0.01), taken
// with one division: h = eps r tt / (|K^r| tt + |K^th| r + (|K^ph| + 1e-40) r tt).
__device__ __forceinline__ double step_size(double eps, const double y[7]) {
    double tt = fmax(fmin(y[1], kPi - y[1]), 1e-2);
    double rt = y[0] * tt;
    double den = fma(fabs(y[6]) + 1e-40, rt, fma(fabs(y[4]), tt, fabs(y[5]) * y[0]));
    return eps * rt / den;
}

// y = (r, theta, phi, K^t, K^r, K^theta, K^phi); t is never needed (stationary metric).
__device__ __forceinline__ void rk4_step(const double *__restrict__ tab, double a, double h, const double y[7],
                                         double out[7]) {
    double k1[7], k2[7], k3[7], k4[7], t[7];
    auto rhs = [&](const double *z, double *dz) {
        dz[0] = z[4];
        dz[1] = z[5];
        dz[2] = z[6];
        double acc[4];
        geo_accel(tab, a, z[0], z[1], z + 3, acc);
        dz[3] = acc[0];
        dz[4] = acc[1];
        dz[5] = acc[2];
        dz[6] = acc[3];
    };
    const double h2 = 0.5 * h, h3 = h * (1.0 / 3.0), h6 = h * (1.0 / 6.0);
    rhs(y, k1);
#pragma unroll
    for (int i = 0; i < 7; i++) t[i] = fma(h2, k1[i], y[i]);
    rhs(t, k2);
#pragma unroll
    for (int i = 0; i < 7; i++) t[i] = fma(h2, k2[i], y[i]);
    rhs(t, k3);
#pragma unroll
    for (int i = 0; i < 7; i++) t[i] = fma(h, k3[i], y[i]);
    rhs(t, k4);
#pragma unroll
    for (int i = 0; i < 7; i++) out[i] = fma(h6, k4[i], fma(h3, k3[i], fma(h3, k2[i], fma(h6, k1[i], y[i]))));
}

__global__ void __launch_bounds__(kGeoThreads, 4) geodesic_kernel(GeoArgs p) {
    const Camera &c = p.cam;
    double y[7];
    long long ray = -1;
    int n = 0, blk = -1, slot = kBlockStates;
    bool live = false, drained = false;
    unsigned long long my_steps = 0;
    for (;;) {
        bool want = !live && !drained;
        unsigned long long t = warp_pop(&p.ctr->geo_next, want);
        if (want) {
            if (t < (unsigned long long)p.nrays) {
                ray = (long long)t;
                int ix, iy;
                ray_pixel(ray + p.ray_offset, c.nx, c.ny, ix, iy);
                double e[4][4], s[3];
                camera_tetrad(c.a, c.r_cam, c.theta_o, e);
                sky_direction(c, ix, iy, s);
                y[0] = c.r_cam;
                y[1] = c.theta_o;
                y[2] = 0.0;
#pragma unroll
                for (int k = 0; k < 4; k++) y[3 + k] = -e[0][k] + s[0] * e[1][k] + s[1] * e[2][k] + s[2] * e[3][k];
                n = 0;
                blk = -1;
                slot = kBlockStates;
                live = true;
            } else {
                drained = true;
            }
        }
        if (__all_sync(0xffffffffu, !live && drained)) break;
        if (!live) continue;

        double h = step_size(c.eps, y);
        double yn[7];
        rk4_step(p.sctab, c.a, h, y, yn);
        bool refl = false;
        if (yn[1] < 0.0) {
            yn[1] = -yn[1];
            yn[2] += kPi;
            yn[5] = -yn[5];
            refl = true;
        } else if (yn[1] > kPi) {
            yn[1] = 2.0 * kPi - yn[1];
            yn[2] += kPi;
            yn[5] = -yn[5];
            refl = true;
        }
        // save state n with the step taken from it; then n+1 becomes current
        uint8_t status = 0;
        for (int pass = 0; pass < 2; pass++) {
            const double *z = pass ? yn : y;
            double hz = pass ? 0.0 : (refl ? -h : h);
            if (pass == 1 && status == 0) break;
            if (slot == kBlockStates) {
                unsigned long long b = atomicAdd(&p.ctr->arena_next, 1ull);
                if (b >= (unsigned long long)p.arena.nblocks) {
                    status = kOverflow;
                    break;
                }
                p.arena.prev[b] = blk;
                blk = (int)b;
                slot = 0;
            }
            PathState ps = {z[0], z[1], z[2], z[3], z[4], z[5], z[6], hz};
            reinterpret_cast<double4_32a *>(p.arena.states + (long long)blk * kBlockStates + slot)[0] =
                make_double4_32a(ps.r, ps.th, ps.ph, ps.kt);
            reinterpret_cast<double4_32a *>(p.arena.states + (long long)blk * kBlockStates + slot)[1] =
                make_double4_32a(ps.kr, ps.kth, ps.kph, ps.h);
            slot++;
            if (pass == 0) {
                n++;
#pragma unroll
                for (int k = 0; k < 7; k++) y[k] = yn[k];
                bool bad = false;
#pragma unroll
                for (int k = 0; k < 7; k++) bad |= !isfinite(y[k]);
                if (bad)
                    status = kNan;
                else if (y[0] < 1.05 * c.rh)
                    status = kHorizon;
                else if (y[0] > c.r_cam && y[4] > 0.0)
                    status = kEscape;
                else if (n >= c.nmax)
                    status = kNmax;
            }
        }
        if (status) {
            RayRecord rec;
            bool ok = (status != kOverflow && status != kNan);
            rec.last_block = ok ? blk : -1;
            rec.nstates = ok ? n + 1 : 0;
            rec.status = status;
            p.rec[ray] = rec;
            my_steps += (unsigned long long)n;
            atomicAdd(&p.ctr->n_status[status], 1u);
            live = false;
        }
    }
    // one counter update per lane
    if (my_steps) atomicAdd(&p.ctr->steps, my_steps);
}

__global__ void sincos_table_kernel(double *tab) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kSinTab) return;
    double th = kSinLo + k * kSinH;
    double s, c;
    sincos(th, &s, &c);
    tab[3 * k] = th;
    tab[3 * k + 1] = s;
    tab[3 * k + 2] = c;
}

void launch_sincos_table(double *tab, cudaStream_t s) {
    sincos_table_kernel<<<(kSinTab + 255) / 256, 256, 0, s>>>(tab);
}

void launch_geodesic(const GeoArgs &a, int grid, cudaStream_t s) {
    geodesic_kernel<<<grid, kGeoThreads, 0, s>>>(a);
}

int geodesic_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, geodesic_kernel, kGeoThreads, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

}  // namespace prt
