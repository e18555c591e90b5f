// The batched form: geodesics and transfers of many images in one persistent launch.
//
// Each 8-warp block holds both roles of the method (the paper's Section 2.1). Its first
// geo_warps warps integrate backward geodesics (FP64) and save the states. The remaining warps
// walk completed paths toward the camera and do the transfer (FP64 or FP32). The roles share
// the SM, so the FP32 transfer issues while the FP64 pipe is busy with geodesics.
//
// Flow control, all in global memory:
//  - rays come from a queue (geo_next) over all images of the batch;
//  - path blocks come from a free ring, so memory is bounded by the pool, not by the batch. A
//    lane that needs a block takes a ticket (a ring position) and polls only that slot, so
//    blocks are handed out first come, first served and waiting lanes touch no shared counter;
//  - a completed ray is published in a ready list (ready_tail) that the transfer warps
//    consume in order (xfer_next).
// Every wait is bounded, by the global nanosecond timer (sleeps are only hints) or by a poll
// count. A geodesic lane whose block has not come for kPoolStallNs gives its ray up as an
// arena overflow and frees the ray's blocks, so in-flight paths cannot deadlock the pool; it
// keeps its ticket and returns that block when it comes. A transfer lane that waits
// kReadyWaitNs for its ray, a ticket still open after kReadyWaitNs, or a ring slot that stays
// unchanged for kRingSpin polls sets an error bit that the host reports.
#pragma once
#include "geodesic.cuh"
#include "transfer_kernel.cuh"

namespace prt {

constexpr int kRingSpin = 1 << 22;
constexpr unsigned long long kPoolStallNs = 1000000000ull;   // 1 s without a free block
constexpr unsigned long long kReadyWaitNs = 30000000000ull;  // 30 s without the awaited ray

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Return a block to the ring at the next tail position. The slot is written only once the
// ticket of the previous lap has taken its value (that ticket exists: the ring never holds
// more than nblocks free blocks), and only after this lane's accesses to the block.
__device__ __forceinline__ int pool_free(const Pool &P, PipeCounters *c, int b) {
    unsigned long long pos = atomicAdd(&c->pool_tail, 1ull);
    volatile int *slot = P.ring + (pos % (unsigned long long)P.nblocks);
    int spin = 0;
    while (*slot >= 0) {
        if (++spin > kRingSpin) {
            atomicOr(&c->err, kPipeErrRing);
            return spin;
        }
    }
    __threadfence();
    *slot = b;
    return spin;
}

// Free every block of a ray from its current block back to the first (own writes only).
__device__ __forceinline__ int pool_free_chain(const Pool &P, PipeCounters *c, int blk) {
    int spins = 0;
    while (blk >= 0) {
        int pb = P.prev[blk];
        spins += pool_free(P, c, blk);
        blk = pb;
    }
    return spins;
}

__device__ __forceinline__ void save_state(const Pool &P, int blk, int slot, const double y[7], double h) {
    double4_32a *d = reinterpret_cast<double4_32a *>(P.states + (long long)blk * kBlockStates + slot);
    d[0] = make_double4_32a(y[0], y[1], y[2], y[3] - y[4]);  // K^t = W - K^r
    d[1] = make_double4_32a(y[4], y[5], y[6], h);
}

// Loads of data written by other SMs during this launch bypass L1 (a reused block may still
// sit in this SM's L1 from its previous ray).
__device__ __forceinline__ double4_32a load_cg(const double4_32a *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldcg(q), b = __ldcg(q + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}

// Publish a finished ray (record and path written before) to the transfer warps.
__device__ __forceinline__ void publish(const PipeArgs &p, long long ray, const RayRecord &rec) {
    p.rec[ray] = rec;
    __threadfence();
    unsigned long long pos = atomicAdd(&p.ctr->ready_tail, 1ull);
    atomicExch(p.ready + pos, (int)ray);
}

__device__ __forceinline__ void pipe_geodesic(const PipeArgs &p, const double *tab) {
    const unsigned long long nb = (unsigned long long)p.pool.nblocks;
    double y[7];
    StepCam sc{};  // the current ray's camera constants
    long long ray = -1, tk = -1;  // tk: pool ticket whose block has not come yet
    int job = 0, n = 0, blk = -1, slot = 0;
    bool live = false, drained = false, cancel = false;
    unsigned long long my_steps = 0, t0 = 0;
    unsigned long long n_iter = 0, n_sleep = 0, n_tpoll = 0, n_spin = 0, n_tick = 0;
    unsigned backoff = 256;
    for (;;) {
        n_iter++;
        bool want = !live && !drained && tk < 0;
        unsigned long long t = warp_pop(&p.ctr->geo_next, want);
        if (want) {
            if (t < (unsigned long long)p.nrays) {
                ray = (long long)t;
                job = find_job(p.jobs, p.njobs, ray);
                const Camera &c = p.jobs[job].cam;
                int ix, iy;
                ray_pixel(ray - p.jobs[job].ray_begin, c.nx, c.ny, ix, iy);
                ray_start(c, ix, iy, y);
                sc = step_cam(c);
                n = 0;
                blk = -1;
                slot = kBlockStates;
                live = true;
            } else {
                drained = true;
            }
        }
        if (__all_sync(0xffffffffu, !live && drained && tk < 0)) break;
        // a ticket for a block when the current one cannot take the two states of a step
        bool ask = live && tk < 0 && slot > kBlockStates - 2;
        unsigned long long pos = warp_pop(&p.ctr->pool_head, ask);
        if (ask) {
            tk = (long long)pos;
            t0 = global_ns();
            n_tick++;
        }
        bool go = live && tk < 0;
        if (tk >= 0) {
            volatile int *sl = p.pool.ring + ((unsigned long long)tk % nb);
            int b = *sl;
            if (b >= 0) {
                *sl = -1;
                tk = -1;
                if (cancel) {  // the ray was given up: return the late block
                    n_spin += pool_free(p.pool, p.ctr, b);
                    cancel = false;
                } else {
                    if (blk >= 0) p.pool.fill[blk] = slot;
                    p.pool.prev[b] = blk;
                    blk = b;
                    slot = 0;
                    go = true;
                }
            } else if (!cancel && global_ns() - t0 > kPoolStallNs) {
                // no block for too long: give the ray up as an overflow, keep the ticket
                n_spin += pool_free_chain(p.pool, p.ctr, blk);
                RayRecord rec = {-1, 0, kOverflow, 0};
                publish(p, ray, rec);
                atomicAdd(&p.ctr->n_status[kOverflow], 1u);
                my_steps += (unsigned long long)n;
                live = false;
                cancel = true;
                t0 = global_ns();
            } else if (cancel && global_ns() - t0 > kReadyWaitNs) {
                atomicOr(&p.ctr->err, kPipeErrRing);
                tk = -1;
                cancel = false;
            }
            if (tk >= 0) n_tpoll++;
        }
        if (__all_sync(0xffffffffu, !go)) {  // nothing to step in this warp: wait a little
            if (__any_sync(0xffffffffu, live || tk >= 0)) {
                n_sleep++;
                __nanosleep(backoff);
                backoff = min(2u * backoff, 8192u);
            }
            continue;
        }
        backoff = 256;
        if (!go) continue;
        uint8_t status = 0;
        for (int k = 0; k < p.step_tile; k++) {
            double h, yn[7];
            bool refl = geo_step<true>(tab, sc, y, yn, h);
            save_state(p.pool, blk, slot, y, refl ? -h : h);
            slot++;
            n++;
#pragma unroll
            for (int i = 0; i < 7; i++) y[i] = yn[i];
            status = geo_stop(sc, y, n);
            if (status || slot > kBlockStates - 2) break;
        }
        if (status) {
            save_state(p.pool, blk, slot, y, 0.0);
            slot++;
            my_steps += (unsigned long long)n;
            RayRecord rec;
            if (status == kNan) {
                n_spin += pool_free_chain(p.pool, p.ctr, blk);
                rec = RayRecord{-1, 0, kNan, 0};
            } else {
                p.pool.fill[blk] = slot;
                rec = RayRecord{blk, n + 1, status, slot};
            }
            publish(p, ray, rec);
            atomicAdd(&p.ctr->n_status[status], 1u);
            live = false;
        }
    }
    if (my_steps) atomicAdd(&p.ctr->steps, my_steps);
    atomicAdd(&p.ctr->geo_iters, n_iter);
    if (n_sleep) atomicAdd(&p.ctr->geo_sleeps, n_sleep);
    if (n_tpoll) atomicAdd(&p.ctr->ticket_polls, n_tpoll);
    if (n_spin) atomicAdd(&p.ctr->free_spins, n_spin);
    if (n_tick) atomicAdd(&p.ctr->tickets, n_tick);
}

template <typename R, typename OutT>
__device__ __forceinline__ void pipe_transfer(const PipeArgs &p, const R *sgw) {
    long long ray = -1;
    int job = 0, blk = -1, slot = 0, n = 0, rstat = 0;
    unsigned long long ticket = 0, wait_t0 = 0;
    bool live = false, pending = false, drained = false;
    XLane<R> Ln;
    unsigned long long my_pts = 0, my_emit = 0;
    unsigned long long n_iter = 0, n_sleep = 0, n_rpoll = 0, n_spin = 0;
    unsigned backoff = 256;
    for (;;) {
        n_iter++;
        bool want = !live && !pending && !drained;
        unsigned long long t = warp_pop(&p.ctr->xfer_next, want);
        if (want) {
            if (t < (unsigned long long)p.nrays) {
                ticket = t;
                pending = true;
                wait_t0 = global_ns();
            } else {
                drained = true;
            }
        }
        if (pending) {
            int v = *reinterpret_cast<volatile int *>(p.ready + ticket);
            if (v >= 0) {
                __threadfence();
                pending = false;
                ray = v;
                job = find_job(p.jobs, p.njobs, ray);
                int4 rr = __ldcg(reinterpret_cast<const int4 *>(p.rec + ray));
                rstat = rr.z;
                if (rr.y >= 2) {
                    blk = rr.x;
                    slot = rr.w - 1;
                    n = rr.y - 1;
                    Ln.reset();
                    live = true;
                } else {
                    const JobDev &J = p.jobs[job];
                    int ix, iy;
                    ray_pixel(ray - J.ray_begin, J.cam.nx, J.cam.ny, ix, iy);
                    long long pix = (long long)iy * J.cam.nx + ix;
                    xfer_zero<OutT>(pix, J.out, J.depth);
                    if (J.status) J.status[pix] = (uint8_t)rstat;
                }
            } else if (global_ns() - wait_t0 > kReadyWaitNs) {
                atomicOr(&p.ctr->err, kPipeErrReady);
                pending = false;
                drained = true;
            } else {
                n_rpoll++;
            }
        }
        if (__all_sync(0xffffffffu, !live && !pending && drained)) break;
        if (!__any_sync(0xffffffffu, live)) {  // the whole warp waits for rays: back off
            n_sleep++;
            __nanosleep(backoff);
            backoff = min(2u * backoff, 32768u);
            continue;
        }
        backoff = 256;
        if (!live) continue;

        // move from state n to state n-1, returning each block once it is passed
        if (--slot < 0) {
            int pb = __ldcg(p.pool.prev + blk);
            n_spin += pool_free(p.pool, p.ctr, blk);
            blk = pb;
            slot = __ldcg(p.pool.fill + blk) - 1;
        }
        n--;
        const JobDev &J = p.jobs[job];
        const double4_32a *src = reinterpret_cast<const double4_32a *>(p.pool.states + (long long)blk * kBlockStates + slot);
        double4_32a q0 = load_cg(src), q1 = load_cg(src + 1);
        KS<R> m;
        if (xfer_point(J.cam, J.model, q0, q1, sgw, Ln, m)) my_emit++;
        my_pts++;
        if (n == 0) {
            int ix, iy;
            ray_pixel(ray - J.ray_begin, J.cam.nx, J.cam.ny, ix, iy);
            xfer_finish<R, OutT>(J.cam, m, ix, iy, Ln, J.out, J.depth);
            if (J.status) J.status[(long long)iy * J.cam.nx + ix] = (uint8_t)rstat;
            n_spin += pool_free(p.pool, p.ctr, blk);
            live = false;
        }
    }
    if (my_pts) atomicAdd(&p.ctr->points, my_pts);
    if (my_emit) atomicAdd(&p.ctr->emitting, my_emit);
    atomicAdd(&p.ctr->xfer_iters, n_iter);
    if (n_sleep) atomicAdd(&p.ctr->xfer_sleeps, n_sleep);
    if (n_rpoll) atomicAdd(&p.ctr->ready_polls, n_rpoll);
    if (n_spin) atomicAdd(&p.ctr->free_spins, n_spin);
}

template <typename R, typename OutT>
__global__ void __launch_bounds__(kPipeThreads, sizeof(R) == 4 ? 2 : 1) pipe_kernel(PipeArgs p) {
    __shared__ R sgw[32];
    __shared__ double tab[3 * kSinTab];  // the geodesic's sin/cos table
    fill_bessel_weights(sgw);
    for (int i = threadIdx.x; i < 3 * kSinTab; i += blockDim.x) tab[i] = p.sctab[i];
    __syncthreads();
    if ((int)(threadIdx.x >> 5) < ((blockIdx.x & 1) ? p.geo_warps_odd : p.geo_warps))
        pipe_geodesic(p, tab);
    else
        pipe_transfer<R, OutT>(p, sgw);
}

}  // namespace prt
