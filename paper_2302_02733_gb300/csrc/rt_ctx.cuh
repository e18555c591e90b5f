// The context behind the opaque rt_ctx handle (shared by the host-side units).
#pragma once
#include "polrt.h"
#include "rt_kernels.cuh"

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
    prt::Counters *h_ctr = nullptr;  // pinned
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    long long last_rays = 0, last_blocks_total = 0;
    int geo_bps = 1, fp64_bps = 1, mixed_bps = 1;
};
