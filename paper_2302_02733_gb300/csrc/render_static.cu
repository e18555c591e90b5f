// rt_render_static: rt_render for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: code that runs under a
// strict memory budget owned by someone else, a host application whose allocator policy
// forbids device allocations after start-up, or code paths that must not touch the
// allocator at all. This entry point renders with its scratch (ray counters, ray records
// and the path arena) in one file-scope static device array of fixed size, which every GPU
// that loads this library holds until the process exits. It allocates nothing: the caller
// passes the device output buffers, and the model and camera come from the context as set
// by rt_load_model and rt_set_camera.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "host_util.cuh"

using namespace prt;

namespace {

constexpr size_t kStaticBytes = 512ull << 20;  // 512 MiB of scratch per device
constexpr size_t kStaticAlign = 256;
constexpr size_t kStaticPerRay = sizeof(RayRecord) + kBudgetBlocksPerRay * kBlockBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

size_t up(size_t x) { return (x + kStaticAlign - 1) / kStaticAlign * kStaticAlign; }

}  // namespace

extern "C" {

// Largest image (nx * ny) one rt_render_static call accepts.
long long rt_render_static_max_pixels(void) {
    size_t room = kStaticBytes - up(sizeof(Counters)) - kStaticAlign;
    return (long long)(room / kStaticPerRay);
}

int rt_render_static(rt_ctx *c, int form, void *out_iquv, uint8_t *status) {
    if (!c || !out_iquv || (form != RT_FP64 && form != RT_MIXED)) return RT_ERR_INVALID;
    if (!c->have_cam || !c->have_model) return RT_ERR_NOT_READY;
    if (c->device < 0 || c->device >= kMaxDevices) return RT_ERR_INVALID;
    const rt_camera &rc = c->cam;
    long long nrays = (long long)rc.nx * rc.ny;
    if (nrays > rt_render_static_max_pixels()) return RT_ERR_SIZE;
    if (!is_device_ptr(out_iquv) || (status && !is_device_ptr(status))) return RT_ERR_INVALID;
    if (cudaSetDevice(c->device) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    // set-up, once per device with that device current: the device address of the array
    if (!g_scratch_ptr[c->device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return RT_ERR_CUDA;
        }
        g_scratch_ptr[c->device] = ptr;
    }
    char *base = (char *)g_scratch_ptr[c->device];

    Camera cam = make_camera(rc, c->eps, c->nmax);
    Model mod = make_model(c, cam);

    // carve the static scratch: counters | ray records | arena states | arena links
    Counters *ctr = (Counters *)base;
    size_t off = up(sizeof(Counters));
    RayRecord *rec = (RayRecord *)(base + off);
    off = up(off + sizeof(RayRecord) * (size_t)nrays);
    long long nblocks = (long long)((kStaticBytes - off - kStaticAlign) / kBlockBytes);
    Arena ar;
    ar.states = (PathState *)(base + off);
    ar.prev = (int *)(base + off + (size_t)nblocks * sizeof(PathState) * kBlockStates);
    ar.nblocks = nblocks;

    // the array keeps the previous call's contents: clear the counters and queue heads
    if (cudaMemsetAsync(ctr, 0, sizeof(Counters), c->stream) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    GeoArgs ga{cam, c->d_sctab, ar, rec, ctr, nrays, 0};
    XferArgs xa{cam, mod, ar, rec, ctr, nrays, 0, out_iquv, status, nullptr};
    cudaEventRecord(c->ev[0], c->stream);
    // the launch shape of rt_set_render_config (blocks per SM), as rt_render's one-pass shape
    const int geo_b = c->rcfg.geo_blocks_per_sm > 0 ? c->rcfg.geo_blocks_per_sm : c->geo_bps;
    const int xf_max = form == RT_FP64 ? c->fp64_bps : c->mixed_bps;
    const int xf_b = c->rcfg.xfer_blocks_per_sm > 0 ? std::min(c->rcfg.xfer_blocks_per_sm, xf_max) : xf_max;
    launch_geodesic(ga, c->nsm * geo_b, c->stream);
    cudaEventRecord(c->ev[1], c->stream);
    xa.kt = KappaTables{c->d_syn, c->d_gl, c->d_gl + 8};
    const int coef = mod.edf == RT_EDF_KAPPA ? 1 : 0;
    if (form == RT_FP64)
        launch_transfer_fp64(xa, coef, c->nsm * xf_b, c->stream);
    else
        launch_transfer_mixed(xa, coef, c->nsm * xf_b, c->stream);
    cudaEventRecord(c->ev[2], c->stream);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
    if (cudaMemcpyAsync(c->h_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    c->last_rays = nrays;
    c->last_blocks_total = nblocks;
    c->last_was_batch = false;
    c->last_was_overlap = false;  // one pass of each kernel: the counters report this call
    c->last_was_streamed = false;
    c->last_chunks = 1;
    c->last_shape = 0;
    c->last_geo_launches = c->last_xf_launches = 1;
    if (c->h_ctr->n_status[kOverflow] > 0) return RT_ERR_WORKSPACE;
    return RT_OK;
}

}  // extern "C"
