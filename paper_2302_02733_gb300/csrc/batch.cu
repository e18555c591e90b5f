// Host side of the batched form (include/polrt.h, rt_render_batch): the job table, the bounded
// path pool, capture and replay of the launch as a CUDA graph, and the launch-shape autotuner.
// The kernel is in pipe.cuh.
#include <algorithm>
#include <climits>
#include <cstring>

#include "host_util.cuh"
#include "polrt.h"

using namespace prt;

namespace {

constexpr int kPoolBlocksPerLane = 24;     // pool blocks per resident lane (about 744 states)
constexpr long long kCalibRays = 1ll << 20; // rays in the autotuner's calibration batch

#define BK(x)                     \
    do {                          \
        if ((x) != cudaSuccess) { \
            cudaGetLastError();   \
            return RT_ERR_CUDA;   \
        }                         \
    } while (0)

int fidx(int form) { return form == RT_FP64 ? 0 : 1; }

int check_jobs(const rt_ctx *c, int form, const rt_job *jobs, int njobs, long long *nrays) {
    if (!c || !jobs || njobs < 1 || (form != RT_FP64 && form != RT_MIXED && form != RT_UNPOL)) return RT_ERR_INVALID;
    if (!c->have_model) return RT_ERR_NOT_READY;
    if (c->model.edf != RT_EDF_THERMAL) return RT_ERR_INVALID;  // the batched form renders thermal electrons
    long long tot = 0;
    for (int i = 0; i < njobs; i++) {
        int rv = check_camera(jobs[i].cam);
        if (rv) return rv;
        if (!jobs[i].out_iquv || !is_device_ptr(jobs[i].out_iquv)) return RT_ERR_INVALID;
        if (jobs[i].status && !is_device_ptr(jobs[i].status)) return RT_ERR_INVALID;
        if (jobs[i].out_depth && (form == RT_UNPOL || !is_device_ptr(jobs[i].out_depth))) return RT_ERR_INVALID;
        tot += (long long)jobs[i].cam.nx * jobs[i].cam.ny;
    }
    if (tot > INT_MAX) return RT_ERR_SIZE;
    *nrays = tot;
    return RT_OK;
}

void drop_graph(rt_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    memset(c->gkey, 0, sizeof(c->gkey));
}

template <typename T>
int realloc_dev(T **p, size_t n) {
    cudaFree(*p);
    *p = nullptr;
    if (cudaMalloc(p, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return RT_ERR_NOMEM;
    }
    return RT_OK;
}

int ensure_jobs(rt_ctx *c, int njobs) {
    if (njobs > c->jobs_cap) {
        drop_graph(c);
        if (c->h_jobs) cudaFreeHost(c->h_jobs);
        c->h_jobs = nullptr;
        c->jobs_cap = 0;
        if (realloc_dev(&c->d_jobs, (size_t)njobs)) return RT_ERR_NOMEM;
        if (cudaMallocHost(&c->h_jobs, sizeof(JobDev) * njobs) != cudaSuccess) {
            cudaGetLastError();
            c->h_jobs = nullptr;
            return RT_ERR_NOMEM;
        }
        c->jobs_cap = njobs;
    }
    return RT_OK;
}

void free_pool(rt_ctx *c) {
    cudaFree(c->pool.states);
    cudaFree(c->pool.prev);
    cudaFree(c->pool.fill);
    cudaFree(c->pool.ring);
    c->pool = Pool{};
    cudaGetLastError();
}

int ensure_buffers(rt_ctx *c, int njobs, long long nrays) {
    int rv = ensure_jobs(c, njobs);
    if (rv) return rv;
    if (nrays > c->brays_cap) {
        drop_graph(c);
        c->brays_cap = 0;
        if (realloc_dev(&c->d_brec, (size_t)nrays) || realloc_dev(&c->d_ready, (size_t)nrays)) return RT_ERR_NOMEM;
        c->brays_cap = nrays;
    }
    if (!c->d_pctr || !c->h_pctr) {
        if (realloc_dev(&c->d_pctr, 1)) return RT_ERR_NOMEM;
        if (cudaMallocHost(&c->h_pctr, sizeof(PipeCounters)) != cudaSuccess) {
            cudaGetLastError();
            c->h_pctr = nullptr;
            return RT_ERR_NOMEM;
        }
    }
    if (!c->pool.states) {
        // sized for every lane resident at the largest occupancy, capped at a quarter of free memory
        int bps = std::max(c->pipe_bps[0], c->pipe_bps[1]);
        long long want = (long long)c->nsm * bps * kPipeThreads * kPoolBlocksPerLane;
        size_t per = sizeof(PathState) * kBlockStates + 3 * sizeof(int);
        size_t freeb = 0, total = 0;
        BK(cudaMemGetInfo(&freeb, &total));
        long long cap = (long long)(freeb / 4 / per);
        long long nb = std::min(want, std::min(cap, (long long)INT_MAX / kBlockStates));
        if (nb < 64) return RT_ERR_NOMEM;
        Pool &P = c->pool;
        if (realloc_dev(&P.states, (size_t)nb * kBlockStates) || realloc_dev(&P.prev, (size_t)nb) ||
            realloc_dev(&P.fill, (size_t)nb) || realloc_dev(&P.ring, (size_t)nb)) {
            free_pool(c);  // the part that was allocated; the next call tries again
            return RT_ERR_NOMEM;
        }
        P.nblocks = (int)nb;
        drop_graph(c);
    }
    return RT_OK;
}

void fill_jobs(rt_ctx *c, const rt_job *jobs, int njobs) {
    long long begin = 0;
    for (int i = 0; i < njobs; i++) {
        JobDev &j = c->h_jobs[i];
        memset(&j, 0, sizeof(j));
        j.cam = make_camera(jobs[i].cam, c->eps, c->nmax);
        j.model = make_model(c, j.cam, jobs[i].M_unit, jobs[i].R_high);
        j.ray_begin = begin;
        j.out = jobs[i].out_iquv;
        j.status = jobs[i].status;
        j.depth = jobs[i].out_depth;
        begin += (long long)jobs[i].cam.nx * jobs[i].cam.ny;
    }
}

// Set-up and launch of one batch on stream s (also what the graph captures).
int enqueue(rt_ctx *c, int form, const rt_batch_config &cfg, int njobs, long long nrays, cudaStream_t s) {
    BK(cudaMemcpyAsync(c->d_jobs, c->h_jobs, sizeof(JobDev) * njobs, cudaMemcpyHostToDevice, s));
    BK(cudaMemsetAsync(c->d_pctr, 0, sizeof(PipeCounters), s));
    BK(cudaMemsetAsync(c->d_ready, 0xff, sizeof(int) * (size_t)nrays, s));
    launch_pool_init(c->pool, c->d_pctr, s);
    PipeArgs a{c->d_jobs, njobs, c->d_sctab, c->pool, c->d_brec, c->d_ready, c->d_pctr, nrays, cfg.geo_warps,
               cfg.step_tile, cfg.geo_warps_odd > 0 ? cfg.geo_warps_odd : cfg.geo_warps};
    int grid = c->nsm * cfg.blocks_per_sm;
    if (form == RT_FP64)
        launch_pipe_fp64(a, grid, s);
    else
        launch_pipe_mixed(a, grid, s);
    BK(cudaGetLastError());
    BK(cudaMemcpyAsync(c->h_pctr, c->d_pctr, sizeof(PipeCounters), cudaMemcpyDeviceToHost, s));
    return RT_OK;
}

int finish(rt_ctx *c, long long nrays) {
    BK(cudaStreamSynchronize(c->bstream));
    c->have_pstats = true;
    const PipeCounters &k = *c->h_pctr;
    Counters &h = *c->h_ctr;
    memset(&h, 0, sizeof(h));
    h.steps = k.steps;
    h.points = k.points;
    h.emitting = k.emitting;
    for (int i = 0; i < 8; i++) h.n_status[i] = k.n_status[i];
    h.arena_next = 0;
    c->last_rays = nrays;
    c->last_blocks_total = c->pool.nblocks;
    c->last_was_batch = true;
    c->last_was_overlap = false;
    c->last_was_streamed = false;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->bev[0], c->bev[1]) == cudaSuccess) c->last_ms_total = ms;
    cudaGetLastError();
    if (k.err) return RT_ERR_STALL;
    if (k.n_status[kOverflow] > 0) return RT_ERR_WORKSPACE;
    return RT_OK;
}

bool valid_cfg(const rt_ctx *c, int form, const rt_batch_config &b) {
    if (b.mode == RT_BATCH_CHUNKS) return true;
    return b.mode == RT_BATCH_PERSISTENT && b.geo_warps >= 1 && b.geo_warps <= kPipeThreads / 32 - 1 &&
           b.geo_warps_odd >= 0 && b.geo_warps_odd <= kPipeThreads / 32 - 1 &&
           b.step_tile >= 1 && b.step_tile <= 16 && b.blocks_per_sm >= 1 && b.blocks_per_sm <= c->pipe_bps[fidx(form)];
}

// Mode 1: the job table's images as one ray space through the overlapped two-kernel shape.
int render_chunks(rt_ctx *c, int form, int njobs, long long nrays) {
    BK(cudaMemcpyAsync(c->d_jobs, c->h_jobs, sizeof(JobDev) * njobs, cudaMemcpyHostToDevice, c->stream));
    int rv = render_jobs_overlap(c, form, c->d_jobs, c->h_jobs, njobs, nrays);
    c->last_was_batch = true;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[0], c->ev[2]) == cudaSuccess) c->last_ms_total = ms;
    cudaGetLastError();
    return rv;
}

int autotune(rt_ctx *c, int form, const rt_job *jobs, int njobs, rt_batch_config *best) {
    long long nrays = 0;
    int rv = check_jobs(c, form, jobs, njobs, &nrays);
    if (rv) return rv;
    BK(cudaSetDevice(c->device));
    // calibration batch: the leading images up to about kCalibRays rays
    int k = 0;
    long long rays = 0;
    while (k < njobs && (k == 0 || rays < kCalibRays)) {
        rays += (long long)jobs[k].cam.nx * jobs[k].cam.ny;
        k++;
    }
    rv = ensure_buffers(c, k, rays);
    if (rv) return rv;
    fill_jobs(c, jobs, k);
    BK(cudaEventRecord(c->bev[2], c->stream));
    BK(cudaStreamWaitEvent(c->bstream, c->bev[2], 0));
    // first the number of geodesic warps at step tile 1, then the step tile at the best of
    // them; each shape is timed twice and keeps its faster time (one launch is noisy)
    int maxb = c->pipe_bps[fidx(form)];
    rt_batch_config top{0, 0, 0, 0.f, RT_BATCH_PERSISTENT, 0};
    bool warm = false;
    auto trial = [&](rt_batch_config cand) -> int {
        if (!warm) {  // one untimed launch first
            int r = enqueue(c, form, cand, k, rays, c->bstream);
            if (r) return r;
            BK(cudaStreamSynchronize(c->bstream));
            warm = true;
        }
        float best_ms = -1.f;
        for (int rep = 0; rep < 2; rep++) {
            BK(cudaEventRecord(c->bev[0], c->bstream));
            int r = enqueue(c, form, cand, k, rays, c->bstream);
            if (r) return r;
            BK(cudaEventRecord(c->bev[1], c->bstream));
            BK(cudaStreamSynchronize(c->bstream));
            if (c->h_pctr->err) return RT_OK;  // a shape whose waits ran out is not a candidate
            float ms = 0.f;
            BK(cudaEventElapsedTime(&ms, c->bev[0], c->bev[1]));
            if (best_ms < 0.f || ms < best_ms) best_ms = ms;
        }
        cand.ms = best_ms;
        if (top.geo_warps == 0 || best_ms < top.ms) top = cand;
        return RT_OK;
    };
    for (int g : {2, 3, 4, 5, 6}) {
        rv = trial(rt_batch_config{g, 1, maxb, 0.f, RT_BATCH_PERSISTENT, 0});
        if (rv) return rv;
    }
    // half a warp per block either side of the best split (odd blocks one warp off): the
    // split at which neither role waits for the other usually lies between two whole numbers
    if (top.geo_warps > 0 && maxb >= 2) {
        const int g = top.geo_warps;
        for (int o : {g - 1, g + 1}) {
            if (o < 1 || o > kPipeThreads / 32 - 1) continue;
            rv = trial(rt_batch_config{g, 1, maxb, 0.f, RT_BATCH_PERSISTENT, o});
            if (rv) return rv;
        }
    }
    if (top.geo_warps > 0) {
        const int g = top.geo_warps, go = top.geo_warps_odd;
        for (int t : {2, 4}) {
            rv = trial(rt_batch_config{g, t, maxb, 0.f, RT_BATCH_PERSISTENT, go});
            if (rv) return rv;
        }
    }
    // the overlapped two-kernel shape on the same images
    {
        int r = render_chunks(c, form, k, rays);
        if (r == RT_OK) r = render_chunks(c, form, k, rays);  // the first call allocates
        if (r == RT_OK && (top.geo_warps == 0 || c->last_ms_total < top.ms))
            top = rt_batch_config{top.geo_warps, top.step_tile, top.blocks_per_sm, c->last_ms_total, RT_BATCH_CHUNKS,
                                  top.geo_warps_odd};
        else if (r != RT_OK && r != RT_ERR_NOMEM)
            return r;
    }
    if (top.geo_warps == 0 && top.mode != RT_BATCH_CHUNKS) return RT_ERR_STALL;
    c->bcfg[fidx(form)] = top;
    c->bcal_rays[fidx(form)] = nrays;
    if (best) *best = top;
    return RT_OK;
}

}  // namespace

namespace prt {
void free_batch(rt_ctx *c) {
    drop_graph(c);
    cudaFree(c->d_jobs);
    if (c->h_jobs) cudaFreeHost(c->h_jobs);
    cudaFree(c->d_brec);
    cudaFree(c->d_ready);
    free_pool(c);
    cudaFree(c->d_pctr);
    if (c->h_pctr) cudaFreeHost(c->h_pctr);
    c->d_jobs = c->h_jobs = nullptr;
    c->jobs_cap = 0;
    c->d_brec = nullptr;
    c->d_ready = nullptr;
    c->brays_cap = 0;
    c->d_pctr = c->h_pctr = nullptr;
    for (int i = 0; i < 3; i++)
        if (c->bev[i]) cudaEventDestroy(c->bev[i]);
    for (int i = 0; i < 3; i++) c->bev[i] = nullptr;
    if (c->bstream) cudaStreamDestroy(c->bstream);
    c->bstream = nullptr;
    cudaGetLastError();
}
}  // namespace prt

extern "C" {

int rt_batch_autotune(rt_ctx *c, int form, const rt_job *jobs, int njobs, rt_batch_config *best) {
    if (form == RT_UNPOL) return RT_ERR_INVALID;  // no launch shape to tune: always mode 1
    return autotune(c, form, jobs, njobs, best);
}

int rt_set_batch_config(rt_ctx *c, int form, const rt_batch_config *cfg) {
    if (!c || !cfg || (form != RT_FP64 && form != RT_MIXED) || !valid_cfg(c, form, *cfg)) return RT_ERR_INVALID;
    c->bcfg[fidx(form)] = *cfg;
    c->bcfg[fidx(form)].ms = 0.f;
    c->bcal_rays[fidx(form)] = 0;
    return RT_OK;
}

int rt_get_batch_config(rt_ctx *c, int form, rt_batch_config *cfg) {
    if (!c || !cfg || (form != RT_FP64 && form != RT_MIXED)) return RT_ERR_INVALID;
    *cfg = c->bcfg[fidx(form)];
    return RT_OK;
}

int rt_get_batch_stats(rt_ctx *c, rt_batch_stats *out) {
    if (!c || !out) return RT_ERR_INVALID;
    if (!c->have_pstats) return RT_ERR_NOT_READY;
    BK(cudaSetDevice(c->device));
    BK(cudaStreamSynchronize(c->bstream));
    const PipeCounters &k = *c->h_pctr;
    out->geo_iters = k.geo_iters;
    out->geo_sleeps = k.geo_sleeps;
    out->xfer_iters = k.xfer_iters;
    out->xfer_sleeps = k.xfer_sleeps;
    out->ticket_polls = k.ticket_polls;
    out->ready_polls = k.ready_polls;
    out->free_spins = k.free_spins;
    out->tickets = k.tickets;
    return RT_OK;
}

int rt_render_batch(rt_ctx *c, int form, const rt_job *jobs, int njobs) {
    long long nrays = 0;
    int rv = check_jobs(c, form, jobs, njobs, &nrays);
    if (rv) return rv;
    BK(cudaSetDevice(c->device));
    if (form == RT_UNPOL) {  // the unpolarized form has no persistent kernel: always mode 1
        rv = ensure_jobs(c, njobs);
        if (rv) return rv;
        fill_jobs(c, jobs, njobs);
        return render_chunks(c, form, njobs, nrays);
    }
    // tune on first use, and again when the batch is far larger or smaller than the one the
    // shape was tuned on (a shape set by hand is kept)
    long long cal = c->bcal_rays[fidx(form)];
    const bool tuned = c->bcfg[fidx(form)].geo_warps != 0 || c->bcfg[fidx(form)].mode == RT_BATCH_CHUNKS;
    if (!tuned || (cal > 0 && (nrays > 4 * cal || 4 * nrays < cal))) {
        rv = autotune(c, form, jobs, njobs, nullptr);
        if (rv) return rv;
    }
    rt_batch_config cfg = c->bcfg[fidx(form)];
    rv = ensure_buffers(c, njobs, nrays);
    if (rv) return rv;
    fill_jobs(c, jobs, njobs);
    if (cfg.mode == RT_BATCH_CHUNKS) {
        rv = render_chunks(c, form, njobs, nrays);
        // a batch too large for mode 1's workspace (two chunks of at most 1/kMaxChunks of its
        // rays) runs in the persistent kernel, whose pool bounds its memory
        if (rv != RT_ERR_NOMEM) return rv;
        cfg.mode = RT_BATCH_PERSISTENT;
        if (!valid_cfg(c, form, cfg)) cfg = rt_batch_config{4, 1, c->pipe_bps[fidx(form)], 0.f, RT_BATCH_PERSISTENT, 0};
    }
    long long key[8] = {form + 1,         njobs,          nrays, cfg.geo_warps * 16 + cfg.geo_warps_odd, cfg.step_tile, cfg.blocks_per_sm,
                        c->pool.nblocks, c->jobs_cap};
    if (!c->gexec || memcmp(key, c->gkey, sizeof(key)) != 0) {
        drop_graph(c);
        BK(cudaStreamBeginCapture(c->bstream, cudaStreamCaptureModeThreadLocal));
        rv = enqueue(c, form, cfg, njobs, nrays, c->bstream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->bstream, &g);
        if (rv || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rv ? rv : RT_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            cudaGetLastError();
            return RT_ERR_CUDA;
        }
        memcpy(c->gkey, key, sizeof(key));
    }
    // after the work already on the caller's stream
    BK(cudaEventRecord(c->bev[2], c->stream));
    BK(cudaStreamWaitEvent(c->bstream, c->bev[2], 0));
    BK(cudaEventRecord(c->bev[0], c->bstream));
    BK(cudaGraphLaunch(c->gexec, c->bstream));
    BK(cudaEventRecord(c->bev[1], c->bstream));
    return finish(c, nrays);
}

}  // extern "C"
