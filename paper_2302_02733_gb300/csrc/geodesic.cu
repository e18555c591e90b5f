// Backward null-geodesic integration from the camera (the paper's Section 2.1: one photon
// per pixel, integrated away from the observer and saved).
//
// Persistent kernel, one ray per lane. A lane whose ray stops takes the next ray from a
// global queue (warp-aggregated atomics), so long photon-ring rays do not hold a warp's
// other lanes idle. Every state is written to a block arena, 64 B per state: each lane
// writes two full 32 B sectors. The FP64 pipe bounds this kernel.
#include <algorithm>

#include "geodesic.cuh"

namespace prt {

static_assert(kSinTabBytes == 3 * kSinTab * sizeof(double), "sin/cos table size");

// JOBS: the rays run over a table of images (p.jobs), each with its own camera; otherwise over
// the one image of p.cam.
template <bool JOBS>
__global__ void __launch_bounds__(kGeoThreads, 4) geodesic_kernel(GeoArgs p) {
    // the sin/cos table in shared memory: the RK4 stages read it at data-dependent indices, and
    // through the texture path those reads queued behind the transfer's gathers
    __shared__ double tab[3 * kSinTab];
    for (int i = threadIdx.x; i < 3 * kSinTab; i += blockDim.x) tab[i] = p.sctab[i];
    __syncthreads();
    const Camera &c = p.cam;
    StepCam sc{};  // JOBS: the current ray's camera constants
    double y[7];
    long long ray = -1;
    int n = 0, blk = -1, slot = kBlockStates, pix = 0;
    bool live = false, drained = false;
    unsigned long long my_steps = 0;
    for (;;) {
        bool want = !live && !drained;
        unsigned long long t = warp_pop(&p.ctr->geo_next, want);
        if (want) {
            if (t < (unsigned long long)p.nrays) {
                ray = (long long)t;
                int ix, iy;
                if (JOBS) {  // the ray's global id (through the order list, if any) and image
                    const long long gid = p.pix_list ? p.pix_list[ray + p.ray_offset] : ray + p.ray_offset;
                    const JobDev &J = p.jobs[find_job(p.jobs, p.njobs, gid)];
                    ray_pixel(gid - J.ray_begin, J.cam.nx, J.cam.ny, ix, iy);
                    ray_start(J.cam, ix, iy, y);
                    sc = step_cam(J.cam);
                    pix = (int)gid;
                } else {
                    map_pixel(p.pix_list, ray + p.ray_offset, c.nx, c.ny, ix, iy);
                    pix = iy * c.nx + ix;
                    ray_start(c, ix, iy, y);
                }
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

        double h, yn[7];
        bool refl = JOBS ? geo_step(tab, sc, y, yn, h) : geo_step(tab, c, y, yn, h);
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
            PathState ps = {z[0], z[1], z[2], z[3] - z[4], z[4], z[5], z[6], hz};  // K^t = W - K^r
            reinterpret_cast<double4_32a *>(p.arena.states + (long long)blk * kBlockStates + slot)[0] =
                make_double4_32a(ps.r, ps.th, ps.ph, ps.kt);
            reinterpret_cast<double4_32a *>(p.arena.states + (long long)blk * kBlockStates + slot)[1] =
                make_double4_32a(ps.kr, ps.kth, ps.kph, ps.h);
            slot++;
            if (pass == 0) {
                n++;
#pragma unroll
                for (int k = 0; k < 7; k++) y[k] = yn[k];
                status = JOBS ? geo_stop(sc, y, n) : geo_stop(c, y, n);
            }
        }
        if (status) {
            RayRecord rec;
            bool ok = (status != kOverflow && status != kNan);
            rec.last_block = ok ? blk : -1;
            rec.nstates = ok ? n + 1 : 0;
            rec.status = status;
            p.rec[ray] = rec;
            if (p.steps_out) p.steps_out[pix] = (uint16_t)min(n, 65535);  // by pixel, or (JOBS) by global id
            my_steps += (unsigned long long)n;
            atomicAdd(&p.ctr->n_status[status], 1u);
            if (p.chunk_done) {
                // release this ray's states and record to the chunk's transfer: the fence orders
                // them before the count; the lane whose count completes the chunk fences again
                // (acquiring the others' and releasing to the host) and raises the flag
                __threadfence();
                const int k = p.layout.chunk_of(ray);
                if (atomicAdd(&p.chunk_done[k], 1u) + 1u == (unsigned)p.layout.size(k)) {
                    __threadfence_system();
                    *(volatile unsigned *)&p.chunk_flag[k] = 1u;
                }
            }
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
    if (a.jobs)
        geodesic_kernel<true><<<grid, kGeoThreads, 0, s>>>(a);
    else
        geodesic_kernel<false><<<grid, kGeoThreads, 0, s>>>(a);
}

static int func_regs(const void *f) {
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, f) != cudaSuccess) {
        cudaGetLastError();
        return 255;
    }
    return a.numRegs;
}

int geodesic_regs() {
    return std::max(func_regs((const void *)geodesic_kernel<false>), func_regs((const void *)geodesic_kernel<true>));
}

int geodesic_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, geodesic_kernel<false>, kGeoThreads, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

}  // namespace prt
