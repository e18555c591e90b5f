// The context behind the opaque rt_ctx handle (shared by the host-side units).
#pragma once
#include "polrt.h"
#include "rt_kernels.cuh"

using prt::RayRecord;

struct rt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nsm = 1;
    rt_camera cam{};
    bool have_cam = false;
    rt_model_params model{};
    bool have_model = false;
    float *d_prims = nullptr;
    size_t prims_bytes = 0;
    double *d_x2 = nullptr;
    float *d_x2f = nullptr;     // float copy of the FMKS inverse table
    double *d_x1c = nullptr;    // 1 / r at the radial cell centres
    int x1c_n = 0;
    // the grid as a 4-d tensor [n1][n2][n3][8] of floats, box 8 x 2 x 2 x 2, for the staged fetch
    CUtensorMap tmap{};
    bool have_tmap = false;
    int fetch = RT_FETCH_AUTO;
    int staged_bps = 1;
    double eps = 0.05;
    int nmax = 20000;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    uint8_t *d_stage_status = nullptr;
    size_t stage_status_bytes = 0;
    void *d_stage_depth = nullptr;
    size_t stage_depth_bytes = 0;
    double *d_stats = nullptr;
    double *d_sctab = nullptr;  // sin/cos table of the FP64 geodesic
    double *d_syn = nullptr;    // ln F, ln G, ln H tables of the kappa quadrature
    double *d_gl = nullptr;     // its Gauss-Legendre nodes and weights
    // surrogate MLP: parameters | Adam m | Adam v | gradient (FP32), tensor-core images, scalars
    float *d_theta = nullptr;
    void *d_wpk = nullptr, *d_tpk = nullptr, *d_mlpaux = nullptr;
    rt_mlp_norm mlp_norm{};
    float *d_gpart = nullptr;   // per-block gradient partials (kMlpParams each) and losses
    long long gpart_cap = 0;    // blocks they hold
    bool have_mlp = false;
    prt::Counters *h_ctr = nullptr;  // pinned
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    long long last_rays = 0, last_blocks_total = 0;
    int geo_bps = 1, fp64_bps = 1, mixed_bps = 1;
    // registers per thread of the geodesic and transfer kernels, and per SM
    int geo_regs = 255, xf_regs_fp64 = 255, xf_regs_mixed = 255, regs_per_sm = 65536;
    float last_ms_total = 0.f;
    bool last_was_batch = false;

    // overlapped rt_render: geodesic of chunk i + 1 on ostream[0] beside the transfer of chunk i
    // on ostream[1]; per chunk the events geodesic start/end, transfer start/end
    static constexpr int kMaxChunks = 256;
    rt_render_config rcfg{};
    cudaStream_t ostream[2] = {nullptr, nullptr};
    cudaEvent_t oev[4 * kMaxChunks] = {};
    bool have_oev = false;
    prt::Counters *h_ctr2 = nullptr;  // pinned: the second half's counters
    // streamed overlapped shape: per chunk the completion flag the geodesic raises (mapped
    // pinned host memory, and its device address)
    unsigned *h_flags = nullptr, *d_flags = nullptr;
    bool last_was_streamed = false;
    int last_pieces = 1;  // pieces of the last streamed render (each last_chunks / last_pieces chunks)
    int last_shape = 0, last_geo_launches = 0, last_xf_launches = 0;  // as rt_counters

    // longest-first ray order (order.cu), from the step counts of the last full render of the
    // same camera and integrator
    uint16_t *d_steps = nullptr;  // per pixel
    int *d_order = nullptr;       // pixel of each ray
    unsigned *d_ohist = nullptr;  // kOrderBuckets counters
    long long order_cap = 0;      // pixels the two arrays hold
    double order_key[8] = {};     // camera and integrator the steps belong to
    bool have_steps = false;
    long long order_K = 0;        // chunks d_order is dealt to; 0: not built
    int order_W = 1;              // and the share divisor of its last chunk (ChunkLayout)
    int *d_probe = nullptr;       // the probe's pixel list (a new camera's predicted order)
    long long probe_cap = 0;
    bool steps_probed = false;    // d_steps holds the probe's predictions, not recorded counts
    // the same for the batched form's mode 1, by global ray id over the job table
    uint16_t *d_bsteps = nullptr;
    int *d_border = nullptr;
    long long border_cap = 0, border_K = 0;
    int border_W = 1;
    unsigned long long bkey = 0;  // hash of the cameras and integrator the steps belong to
    bool have_bsteps = false;
    float last_ms_geo = 0.f, last_ms_xfer = 0.f;
    bool last_was_overlap = false;
    int last_chunks = 0;

    // batched form (rt_render_batch)
    cudaStream_t bstream = nullptr;       // private stream: graph capture needs a non-legacy stream
    cudaEvent_t bev[3] = {nullptr, nullptr, nullptr};
    prt::JobDev *d_jobs = nullptr, *h_jobs = nullptr;  // device table and its pinned staging copy
    int jobs_cap = 0;
    RayRecord *d_brec = nullptr;
    int *d_ready = nullptr;
    long long brays_cap = 0;
    prt::Pool pool{};
    prt::PipeCounters *d_pctr = nullptr, *h_pctr = nullptr;
    bool have_pstats = false;             // h_pctr holds a finished mode-0 batch
    int pipe_bps[2] = {1, 1};             // resident blocks per SM of the fp64 / mixed pipe kernel
    rt_batch_config bcfg[2] = {};         // per form; geo_warps == 0 means not tuned yet
    long long bcal_rays[2] = {0, 0};      // rays of the batch the shape was tuned on (0: set by hand)
    cudaGraphExec_t gexec = nullptr;      // the captured batch of the last call
    long long gkey[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};
