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

#include "rt_ctx.cuh"

using namespace prt;

namespace {

constexpr size_t kStaticBytes = 512ull << 20;  // 512 MiB of scratch per device
constexpr size_t kStaticAlign = 256;
constexpr size_t kStaticBlockBytes = sizeof(PathState) * kBlockStates + sizeof(int);
constexpr size_t kStaticPerRay = sizeof(RayRecord) + 20 * kStaticBlockBytes;  // 640 states per ray

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

size_t up(size_t x) { return (x + kStaticAlign - 1) / kStaticAlign * kStaticAlign; }

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

double isco(double a) {
    double z1 = 1.0 + std::cbrt(1.0 - a * a) * (std::cbrt(1.0 + a) + std::cbrt(1.0 - a));
    double z2 = std::sqrt(3.0 * a * a + z1 * z1);
    return 3.0 + z2 - std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

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
    if (!on_device(out_iquv) || (status && !on_device(status))) return RT_ERR_INVALID;
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

    Camera cam{};
    cam.a = rc.a;
    cam.r_cam = rc.r_cam;
    cam.theta_o = rc.incl_deg * kPi / 180.0;
    cam.nu_obs = rc.freq_hz;
    cam.fov = rc.fov_M;
    cam.L_unit = kG * rc.M_bh_g / (kC * kC);
    cam.nx = rc.nx;
    cam.ny = rc.ny;
    cam.eps = c->eps;
    cam.nmax = c->nmax;
    cam.rh = 1.0 + std::sqrt(1.0 - rc.a * rc.a);
    Model mod{};
    mod.kind = c->model.kind;
    if (mod.kind == RT_MODEL_ADAF) {
        const rt_adaf_params &a = c->model.adaf;
        mod.adaf = AdafModel{a.n0, a.T0, a.beta, a.f_kep, a.Ti_over_Te, a.r_out, isco(rc.a)};
    } else {
        const rt_grid_params &g = c->model.grid;
        GridModel &gm = mod.grid;
        gm.n1 = g.n1;
        gm.n2 = g.n2;
        gm.n3 = g.n3;
        gm.r_in = g.r_in;
        gm.r_out = g.r_out;
        gm.x1in = std::log(g.r_in);
        gm.dx1 = (std::log(g.r_out) - gm.x1in) / g.n1;
        gm.dx2 = 1.0 / g.n2;
        gm.dx3 = 2.0 * kPi / g.n3;
        gm.hslope = g.hslope;
        gm.poly_xt = g.poly_xt;
        gm.poly_alpha = g.poly_alpha;
        gm.mks_smooth = g.mks_smooth;
        gm.poly_norm = 0.5 * kPi / (1.0 + 1.0 / ((g.poly_alpha + 1.0) * std::pow(g.poly_xt, g.poly_alpha)));
        gm.prims = reinterpret_cast<const float4 *>(c->d_prims);
        gm.x2_table = c->d_x2;
        double L = cam.L_unit;
        gm.rho_unit = g.M_unit / (L * L * L);
        gm.b_unit = kC * std::sqrt(4.0 * kPi * gm.rho_unit);
        gm.ne_unit = gm.rho_unit / (kMp + kMe);
        gm.R_high = g.R_high;
        gm.R_low = g.R_low;
        gm.sigma_cut = g.sigma_cut;
        gm.gamma_ad = g.gamma_ad;
    }

    // carve the static scratch: counters | ray records | arena states | arena links
    Counters *ctr = (Counters *)base;
    size_t off = up(sizeof(Counters));
    RayRecord *rec = (RayRecord *)(base + off);
    off = up(off + sizeof(RayRecord) * (size_t)nrays);
    long long nblocks = (long long)((kStaticBytes - off - kStaticAlign) / kStaticBlockBytes);
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
    launch_geodesic(ga, c->nsm * c->geo_bps, c->stream);
    cudaEventRecord(c->ev[1], c->stream);
    if (form == RT_FP64)
        launch_transfer_fp64(xa, c->nsm * c->fp64_bps, c->stream);
    else
        launch_transfer_mixed(xa, c->nsm * c->mixed_bps, c->stream);
    cudaEventRecord(c->ev[2], c->stream);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
    if (cudaMemcpyAsync(c->h_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    c->last_rays = nrays;
    c->last_blocks_total = nblocks;
    if (c->h_ctr->n_status[kOverflow] > 0) return RT_ERR_WORKSPACE;
    return RT_OK;
}

}  // extern "C"
