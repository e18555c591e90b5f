// Kernel argument blocks and launchers shared by the host API and the kernels.
#pragma once
#include <cuda.h>

#include "rt_common.cuh"

namespace prt {

constexpr int kGeoThreads = 128;
constexpr int kXferThreads = 128;

struct JobDev;

// How n rays are split into K consecutive chunks: the last chunk takes 1/W of a regular one's
// share (W = 1: equal chunks). Ranks of the longest-first sort are dealt in rounds of
// P = (K - 1) W + 1: in each round chunk k < K - 1 takes W consecutive ranks and the last chunk
// one, so every chunk holds the same mix of lengths, longest first. A final partial round
// (n % P ranks) fills the regular chunks in turn.
struct ChunkLayout {
    long long n;
    int K, W;
    __host__ __device__ long long period() const { return (long long)(K - 1) * W + 1; }
    __host__ __device__ long long size(int k) const {
        const long long P = period(), R = n / P, rem = n % P;
        if (k < K - 1) {
            const long long e = rem - (long long)k * W;
            return R * W + (e < 0 ? 0 : (e > W ? W : e));
        }
        return R;  // rem < P: a partial round never reaches the last chunk
    }
    __host__ __device__ long long offset(int k) const {
        const long long P = period(), R = n / P, rem = n % P, kw = (long long)k * W;
        return (long long)k * R * W + (rem < kw ? rem : kw);
    }
    // the largest chunk (the first)
    __host__ __device__ long long max_size() const { return size(0); }
    // the chunk holding index t (0 <= t < n)
    __host__ __device__ int chunk_of(long long t) const {
        int lo = 0, hi = K - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offset(mid) <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    }
    // rank s of the sort -> its index in the order array
    __host__ __device__ long long place(long long s) const {
        const long long P = period(), r = s / P, j = s % P;
        if (j < (long long)(K - 1) * W) return offset((int)(j / W)) + r * W + j % W;
        return offset(K - 1) + r;
    }
};

struct GeoArgs {
    Camera cam;
    const double *sctab;  // (theta, sin, cos) table of the FP64 geodesic, 1024 entries
    Arena arena;
    RayRecord *rec;       // per ray of this chunk
    Counters *ctr;
    long long nrays;      // rays in this chunk
    long long ray_offset; // global id of the chunk's first ray
    const int *pix_list;  // optional: the pixel of each global ray id (adaptive rendering, ray order)
    uint16_t *steps_out;  // optional: per pixel (row-major), the ray's RK4 step count (capped at 65535)
    const JobDev *jobs;   // optional: a table of images; global ray ids then run over all of them, the
    int njobs;            // order list holds global ray ids and steps_out is indexed by them
    // optional (streamed overlapped shape): the rays' chunks; every ray that stops adds one to
    // chunk_done of its chunk, and the lane that completes a chunk sets its chunk_flag (mapped
    // host memory) after a system-scope fence
    unsigned *chunk_done;
    unsigned *chunk_flag;
    ChunkLayout layout;
};

struct XferArgs {
    Camera cam;
    Model model;
    Arena arena;
    const RayRecord *rec;
    Counters *ctr;
    long long nrays, ray_offset;
    void *out;            // image [ny][nx][4] of double (FP64 form) or float (mixed form)
    uint8_t *status;      // optional per-pixel status
    void *depth;          // optional [ny][nx][2] optical and Faraday depths, same type as out
    // kappa electrons (model.edf == 1): the quadrature's tables; for the surrogate form the
    // network's outputs per saved state (8 floats at state index block * 32 + slot), its
    // normalisation (8 means, 8 standard deviations, 8 x 35 baseline) and input box
    KappaTables kt;
    const float *sur_y;
    const float *sur_norm;
    float sur_lo[4], sur_hi[4];
    float4 *feat;         // features pass: network inputs per saved state, or (sur_row) per compact row
    int *sur_row;         // optional: per saved state, its row of feat and sur_y; the features pass
                          // hands each ray consecutive rows (ctr->sur_rows counts them)
    float4 *feat_raw;     // or (rt_render_features) raw inputs of the emitting points, compacted
    long long feat_cap;
    const int *pix_list;  // optional: the pixel of each global ray id (adaptive rendering)
    const JobDev *jobs;   // optional: a table of images (see GeoArgs)
    int njobs;
};

// ---- batched rendering: many images in one persistent launch ----------------------------
// One image of a batch in kernel form. Rays of the batch are numbered image after image.
struct JobDev {
    Camera cam;
    Model model;
    long long ray_begin;  // global id of the image's first ray
    void *out;            // [ny][nx][4] of the form's type
    uint8_t *status;      // optional [ny][nx]
    void *depth;          // optional [ny][nx][2]
};

// Image of a global ray id: the last job whose first ray is <= ray.
__device__ __forceinline__ int find_job(const JobDev *jobs, int njobs, long long ray) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&jobs[mid].ray_begin) <= ray)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// A bounded pool of path blocks with a free ring, so the memory of a batch does not grow
// with its ray count: blocks return to the ring as the transfer walks past them.
struct Pool {
    PathState *states;  // nblocks * kBlockStates
    int *prev;          // previous block of the same ray, -1 for the first
    int *fill;          // states the block holds once closed
    int *ring;          // free-block ring of nblocks slots, -1 marks an empty slot
    int nblocks;
};

struct PipeCounters {
    unsigned long long geo_next, xfer_next, ready_tail;  // work queues
    unsigned long long pool_head, pool_tail;             // free-ring ticket and return positions
    unsigned long long steps, points, emitting;
    unsigned int n_status[8];
    unsigned int err;                                    // kPipeErr* bits
    unsigned int pad1;
    // flow statistics, summed over lanes at their exit (one atomic each): loop iterations of
    // the geodesic and transfer warps, iterations in which the whole warp slept (nothing to
    // step, or no ray published yet), empty polls of a ticket's ring slot and of a ready slot,
    // and polls of a busy slot when returning a block
    unsigned long long geo_iters, geo_sleeps, xfer_iters, xfer_sleeps;
    unsigned long long ticket_polls, ready_polls, free_spins, tickets;
};
constexpr unsigned kPipeErrRing = 1u;   // a free-ring slot never changed
constexpr unsigned kPipeErrReady = 2u;  // a transfer lane never received its ray

constexpr int kPipeThreads = 256;  // 8 warps: geo_warps integrate geodesics, the rest transfer

struct PipeArgs {
    const JobDev *jobs;
    int njobs;
    const double *sctab;
    Pool pool;
    RayRecord *rec;     // per ray of the batch; pad holds the last block's fill
    int *ready;         // completed rays in completion order, -1 until written
    PipeCounters *ctr;
    long long nrays;
    int geo_warps;      // 1..7
    int step_tile;      // RK4 steps per lane between queue and pool checks
    int geo_warps_odd;  // 1..7: the geodesic warps of odd-numbered blocks
};

void launch_pool_init(const Pool &p, PipeCounters *c, cudaStream_t s);
void launch_pipe_fp64(const PipeArgs &a, int grid, cudaStream_t s);
void launch_pipe_mixed(const PipeArgs &a, int grid, cudaStream_t s);
int pipe_blocks_per_sm_fp64();
int pipe_blocks_per_sm_mixed();

// ---- kappa-distribution coefficients by quadrature (kappa.cuh) ---------------------------
constexpr size_t kSynTabBytes = 3 * 4096 * sizeof(double);
int launch_kappa_tables(double *lnk, double *gl16, cudaStream_t s);  // gl16: 8 nodes + 8 weights
void launch_kappa_quad(const KappaTables &T, const double *in, double *out, long long n, int grid, cudaStream_t s);

void launch_geodesic(const GeoArgs &a, int grid, cudaStream_t s);
// Longest-first ray order from the step counts of a previous render of the same camera:
// order[i] is the pixel of ray i, by step count descending (16-step buckets), placed by the
// layout L into its chunks. hist: kOrderBuckets unsigned of scratch.
constexpr int kOrderBuckets = 1024;
void launch_order_build(const uint16_t *steps, const ChunkLayout &L, unsigned *hist, int *order, cudaStream_t s);
// The probe of a new camera: list[i] = the pixel at the centre of S x S block i (row-major over
// blocks, clipped to the image); then every pixel takes its block's probe's step count.
void launch_probe_list(int *list, int nx, int ny, int S, cudaStream_t s);
void launch_steps_fill(uint16_t *steps, int nx, int ny, int S, cudaStream_t s);
void launch_sincos_table(double *tab, cudaStream_t s);
constexpr size_t kSinTabBytes = 1024 * 3 * sizeof(double);
// coef: 0 thermal fits, 1 kappa quadrature at every emitting point, 2 surrogate outputs
void launch_transfer_fp64(const XferArgs &a, int coef, int grid, cudaStream_t s);
void launch_transfer_mixed(const XferArgs &a, int coef, int grid, cudaStream_t s);
// the FP32 transfer (thermal electrons, grid model, one image) with the grid fetch staged
// through shared memory by TMA loads of map: the grid as a 4-d tensor [n1][n2][n3][8] of floats
// with a box of 8 x 2 x 2 x 2
void launch_transfer_staged(const XferArgs &a, const CUtensorMap &map, int grid, cudaStream_t s);
void launch_sur_features(const XferArgs &a, int grid, cudaStream_t s);
void launch_unpol(const XferArgs &a, int grid, cudaStream_t s);  // Stokes I only, FP32
// n rows, capped (when used is given) at used[0] * used_scale, a count an earlier kernel on the
// stream wrote
void launch_mlp_forward(const float *x, float *y, long long n, const void *wpk, unsigned *err, int grid, cudaStream_t s,
                        const unsigned long long *used = nullptr, int used_scale = 1);
void launch_x2_table(const GridModel &g, double *table, float *table_f, cudaStream_t s);
// out[7]: sum I, Q, U, V, flux [Jy], net LP, net CP; out holds 8 + 4 kStatBlocks doubles
constexpr int kStatBlocks = 608;
// form: 0 double IQUV, 1 float IQUV, 2 float I only
void launch_image_sums(const void *img, int form, long long npix, double domega, double *out, cudaStream_t s);
// resident blocks per SM of the persistent kernels (for grid sizing)
int geodesic_blocks_per_sm();
int transfer_blocks_per_sm_fp64();
int transfer_blocks_per_sm_mixed();
int transfer_blocks_per_sm_staged();
// registers per thread of a kernel (cudaFuncGetAttributes), for the overlapped shape's sharing
// of an SM's register file between one geodesic block and the transfer blocks beside it
int geodesic_regs();
int transfer_regs_fp64();
int transfer_regs_mixed();  // the largest of the mixed, staged and unpolarized transfers

}  // namespace prt
