// Host side of the C ABI (include/polrt.h): argument checks, buffers, chunking and launches.
// All arithmetic of the method runs in the kernels. The host derives only constants of the
// parameters (units, horizon radius, grid spacings).
#include <algorithm>
#include <chrono>
#include <climits>
#include <thread>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "host_util.cuh"
#include "kappa.cuh"
#include "polrt.h"

using namespace prt;

namespace {
constexpr size_t kAlign = 256;
constexpr size_t kPerRayBytes = sizeof(RayRecord) + kBudgetBlocksPerRay * kBlockBytes;
// automatic overlapped shape: about 2^kAutoChunkShift rays per chunk, 4 to kAutoChunksMax
// chunks, the last with 1/kAutoLastDiv of a regular chunk's share
constexpr int kAutoChunkShift = 17;
constexpr int kAutoChunksMax = 16;
constexpr int kAutoLastDiv = 1;
// automatic streamed shape: about 2^kStreamChunkShift rays per chunk, at least 16 per piece,
// kStreamGeoBlocks geodesic blocks per SM
constexpr int kStreamChunkShift = 15;
constexpr int kStreamGeoBlocks = 2;
// RT_FETCH_AUTO: the grid fetch measured faster on GB300 for the benchmark image
constexpr bool kStagedByDefault = false;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// The tensor map of the staged grid fetch: the grid's [n1][n2][n3][8] floats as a 4-d tensor
// (innermost first: 8 primitives, n3, n2, n1; rows 32 bytes apart), loaded in boxes of one
// cell's 8 floats x 2 x 2 x 2 cells. The driver's encoder is reached through the runtime, so the
// library links no driver library. False if the grid is too small for the box or the encoder
// refuses it (the fetch then gathers).
bool encode_grid_tmap(CUtensorMap *map, const float *prims, int n1, int n2, int n3) {
    if (n1 < 2 || n2 < 2 || n3 < 2) return false;
    typedef CUresult (*Encode)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                               const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        encode = (Encode)fn;
    }
    const cuuint64_t dims[4] = {8, (cuuint64_t)n3, (cuuint64_t)n2, (cuuint64_t)n1};
    const cuuint64_t strides[3] = {32, 32ull * n3, 32ull * n3 * n2};  // bytes, dims 1..3
    const cuuint32_t box[4] = {8, 2, 2, 2}, estr[4] = {1, 1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)prims, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Whether the FP32 transfer of this render stages its grid fetch (rt_set_grid_fetch).
bool use_staged(const rt_ctx *c, int form, int coef, const Model &mod, const JobDev *jobs) {
    if (form != RT_MIXED || coef != 0 || jobs || mod.kind != RT_MODEL_GRID || !c->have_tmap) return false;
    return c->fetch == RT_FETCH_STAGED || (c->fetch == RT_FETCH_AUTO && kStagedByDefault);
}
}  // namespace


#define CK(x)                                 \
    do {                                      \
        if ((x) != cudaSuccess) {             \
            cudaGetLastError();               \
            return RT_ERR_CUDA;               \
        }                                     \
    } while (0)

extern "C" {

const char *rt_error_string(int code) {
    switch (code) {
        case RT_OK: return "ok";
        case RT_ERR_INVALID: return "invalid argument";
        case RT_ERR_CUDA: return "CUDA runtime error";
        case RT_ERR_NOMEM: return "out of memory";
        case RT_ERR_NOT_READY: return "model or camera not set";
        case RT_ERR_WORKSPACE: return "path arena overflow: enlarge the workspace";
        case RT_ERR_SIZE: return "size beyond the call's fixed limit";
        case RT_ERR_STALL: return "a bounded wait in a kernel ran out";
        default: return "unknown error";
    }
}

size_t rt_workspace_min_bytes(void) { return align_up(sizeof(Counters)) + kPerRayBytes + 4 * kAlign; }

int rt_create(rt_ctx **out, int device, void *stream) {
    if (!out) return RT_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return RT_ERR_INVALID;
    CK(cudaSetDevice(device));
    rt_ctx *c = new (std::nothrow) rt_ctx();
    if (!c) return RT_ERR_NOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return RT_ERR_CUDA;
    }
    c->nsm = prop.multiProcessorCount;
    c->geo_bps = geodesic_blocks_per_sm();
    c->fp64_bps = transfer_blocks_per_sm_fp64();
    c->mixed_bps = transfer_blocks_per_sm_mixed();
    c->staged_bps = transfer_blocks_per_sm_staged();
    c->pipe_bps[0] = pipe_blocks_per_sm_fp64();
    c->pipe_bps[1] = pipe_blocks_per_sm_mixed();
    c->geo_regs = geodesic_regs();
    c->xf_regs_fp64 = transfer_regs_fp64();
    c->xf_regs_mixed = transfer_regs_mixed();
    c->regs_per_sm = prop.regsPerMultiprocessor;
    bool ok = cudaMalloc(&c->d_stats, (8 + 4 * kStatBlocks) * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->d_sctab, kSinTabBytes) == cudaSuccess &&
              cudaMalloc(&c->d_syn, kSynTabBytes) == cudaSuccess && cudaMalloc(&c->d_gl, 16 * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&c->h_ctr, sizeof(Counters)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->bstream, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; i < 3 && ok; i++) ok = cudaEventCreate(&c->ev[i]) == cudaSuccess;
    for (int i = 0; i < 3 && ok; i++) ok = cudaEventCreate(&c->bev[i]) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        rt_destroy(c);
        return RT_ERR_CUDA;
    }
    memset(c->h_ctr, 0, sizeof(Counters));
    launch_sincos_table(c->d_sctab, c->stream);
    if (launch_kappa_tables(c->d_syn, c->d_gl, c->stream) != 0 || cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        rt_destroy(c);
        return RT_ERR_CUDA;
    }
    *out = c;
    return RT_OK;
}

int rt_destroy(rt_ctx *c) {
    if (!c) return RT_ERR_INVALID;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_prims);
    cudaFree(c->d_x2);
    cudaFree(c->d_x2f);
    cudaFree(c->d_x1c);
    for (int i = 0; i < 2; i++)
        if (c->ostream[i]) cudaStreamDestroy(c->ostream[i]);
    if (c->have_oev)
        for (int i = 0; i < 4 * rt_ctx::kMaxChunks; i++) cudaEventDestroy(c->oev[i]);
    if (c->h_ctr2) cudaFreeHost(c->h_ctr2);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    cudaFree(c->d_steps);
    cudaFree(c->d_order);
    cudaFree(c->d_ohist);
    cudaFree(c->d_bsteps);
    cudaFree(c->d_border);
    cudaFree(c->d_probe);
    if (c->ws_owned) cudaFree(c->ws);
    cudaFree(c->d_stage);
    cudaFree(c->d_stage_status);
    cudaFree(c->d_stage_depth);
    cudaFree(c->d_stats);
    cudaFree(c->d_sctab);
    cudaFree(c->d_syn);
    cudaFree(c->d_gl);
    cudaFree(c->d_theta);
    cudaFree(c->d_wpk);
    cudaFree(c->d_tpk);
    cudaFree(c->d_mlpaux);
    cudaFree(c->d_gpart);
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    for (int i = 0; i < 3; i++)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    free_batch(c);
    cudaGetLastError();
    delete c;
    return RT_OK;
}

int rt_set_stream(rt_ctx *c, void *stream) {
    if (!c) return RT_ERR_INVALID;
    c->stream = (cudaStream_t)stream;
    return RT_OK;
}

int rt_get_camera(const rt_ctx *c, rt_camera *cam) {
    if (!c || !cam) return RT_ERR_INVALID;
    if (!c->have_cam) return RT_ERR_NOT_READY;
    *cam = c->cam;
    return RT_OK;
}

int rt_set_integrator(rt_ctx *c, double eps, int nmax) {
    if (!c || !(eps > 0.0) || !(eps < 1.0) || nmax < 1) return RT_ERR_INVALID;
    c->eps = eps;
    c->nmax = nmax;
    return RT_OK;
}

int rt_set_camera(rt_ctx *c, const rt_camera *cam) {
    if (!c || !cam) return RT_ERR_INVALID;
    int rv = check_camera(*cam);
    if (rv) return rv;
    c->cam = *cam;
    c->have_cam = true;
    return RT_OK;
}

int rt_load_model(rt_ctx *c, const rt_model_params *p) {
    if (!c || !p) return RT_ERR_INVALID;
    if (p->edf != RT_EDF_THERMAL && !(p->edf == RT_EDF_KAPPA && p->kappa > 3.0 && p->kappa < 100.0))
        return RT_ERR_INVALID;
    if (p->kind == RT_MODEL_ADAF) {
        const rt_adaf_params &a = p->adaf;
        if (!(a.n0 > 0) || !(a.T0 > 0) || !(a.beta > 0) || !(a.Ti_over_Te >= 0) || !(a.r_out > 0))
            return RT_ERR_INVALID;
    } else if (p->kind == RT_MODEL_GRID) {
        const rt_grid_params &g = p->grid;
        if (g.n1 < 2 || g.n2 < 2 || g.n3 < 1 || !g.prims || !(g.r_in > 0) || !(g.r_out > g.r_in) ||
            !(g.M_unit > 0) || !(g.gamma_ad > 1.0) || !(g.poly_alpha > 0) || !(g.poly_xt > 0))
            return RT_ERR_INVALID;
    } else {
        return RT_ERR_INVALID;
    }
    CK(cudaSetDevice(c->device));
    if (p->kind == RT_MODEL_GRID) {
        const rt_grid_params &g = p->grid;
        // the grid's device buffers change from here on: until they all hold the new grid there
        // is no model (a failure leaves none, rather than the old description over new buffers)
        c->have_model = false;
        size_t bytes = (size_t)g.n1 * g.n2 * g.n3 * 8 * sizeof(float);
        if (bytes != c->prims_bytes) {
            cudaFree(c->d_prims);
            c->d_prims = nullptr;
            c->prims_bytes = 0;
            if (cudaMalloc(&c->d_prims, bytes) != cudaSuccess) {
                cudaGetLastError();
                return RT_ERR_NOMEM;
            }
            c->prims_bytes = bytes;
        }
        cudaMemcpyKind kind = is_device_ptr(g.prims) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CK(cudaMemcpyAsync(c->d_prims, g.prims, bytes, kind, c->stream));
        c->have_tmap = encode_grid_tmap(&c->tmap, c->d_prims, g.n1, g.n2, g.n3);
        if (!c->d_x2) {
            if (cudaMalloc(&c->d_x2, sizeof(double) * kX2TabW * kX2TabT) != cudaSuccess ||
                cudaMalloc(&c->d_x2f, sizeof(float) * kX2TabW * kX2TabT) != cudaSuccess) {
                cudaGetLastError();
                return RT_ERR_NOMEM;
            }
        }
        if (c->x1c_n != g.n1) {
            cudaFree(c->d_x1c);
            c->d_x1c = nullptr;
            c->x1c_n = 0;
            // 1 / r_c as doubles, then as FP32 pairs (value, remainder)
            if (cudaMalloc(&c->d_x1c, (sizeof(double) + sizeof(float2)) * g.n1) != cudaSuccess) {
                cudaGetLastError();
                return RT_ERR_NOMEM;
            }
            c->x1c_n = g.n1;
        }
        {
            // the same X1_in and dx1 as the fetch (make_model)
            double x1in = std::log(g.r_in), dx1 = (std::log(g.r_out) - x1in) / g.n1;
            std::vector<double> irc(g.n1);
            std::vector<float2> irc2(g.n1);
            for (int i = 0; i < g.n1; i++) {
                irc[i] = std::exp(-(x1in + (i + 0.5) * dx1));
                irc2[i].x = (float)irc[i];
                irc2[i].y = (float)(irc[i] - (double)irc2[i].x);
            }
            CK(cudaMemcpyAsync(c->d_x1c, irc.data(), sizeof(double) * g.n1, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->d_x1c + g.n1, irc2.data(), sizeof(float2) * g.n1, cudaMemcpyHostToDevice,
                               c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        GridModel gm{};
        gm.hslope = g.hslope;
        gm.poly_xt = g.poly_xt;
        gm.poly_alpha = g.poly_alpha;
        gm.mks_smooth = g.mks_smooth;
        gm.poly_norm = 0.5 * kPi / (1.0 + 1.0 / ((g.poly_alpha + 1.0) * std::pow(g.poly_xt, g.poly_alpha)));
        launch_x2_table(gm, c->d_x2, c->d_x2f, c->stream);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(c->stream));
    }
    c->model = *p;
    c->model.grid.prims = nullptr;  // the device copy is used from here on
    c->have_model = true;
    return RT_OK;
}

// Wait for the overlapped shapes' internal streams: a render that returned an error part way
// may have left launches on them that still use the workspace. Idle streams return at once.
static int quiesce_overlap(rt_ctx *c) {
    for (int i = 0; i < 2; i++)
        if (c->ostream[i]) CK(cudaStreamSynchronize(c->ostream[i]));
    return RT_OK;
}

int rt_set_workspace(rt_ctx *c, void *dev_ptr, size_t bytes) {
    if (!c) return RT_ERR_INVALID;
    if (dev_ptr && bytes < rt_workspace_min_bytes()) return RT_ERR_INVALID;
    if (dev_ptr && ((uintptr_t)dev_ptr % kAlign) != 0) return RT_ERR_INVALID;
    quiesce_overlap(c);  // no launch of an earlier render may still use the old workspace
    if (c->ws_owned) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->ws);
    }
    c->ws = dev_ptr;
    c->ws_bytes = dev_ptr ? bytes : 0;
    c->ws_owned = false;
    return RT_OK;
}

// Bytes per arena block the surrogate form adds: per saved state, the network's input (float4)
// and output (8 floats), and (streamed) the state's compact row.
constexpr size_t kSurBlockBytes = (size_t)kBlockStates * (16 + 32 + 4);
constexpr size_t kSurPerRayBytes = kPerRayBytes + (size_t)kBudgetBlocksPerRay * kSurBlockBytes;

// Workspace bytes the streamed shape needs for nrays rays: counters, chunk counts, ray records
// and the arena at the per-ray budget (per_ray: kPerRayBytes, or kSurPerRayBytes for the
// surrogate form).
static size_t streamed_bytes(long long nrays, size_t per_ray = kPerRayBytes) {
    return align_up(sizeof(Counters)) + align_up(sizeof(unsigned) * rt_ctx::kMaxChunks) + (size_t)nrays * per_ray +
           8 * kAlign;
}

int rt_workspace_hint(const rt_ctx *c, size_t *bytes) {
    if (!c || !bytes) return RT_ERR_INVALID;
    if (!c->have_cam) return RT_ERR_NOT_READY;
    *bytes = streamed_bytes((long long)c->cam.nx * c->cam.ny);
    return RT_OK;
}

static int ensure_workspace(rt_ctx *c, long long nrays, size_t per_ray = kPerRayBytes) {
    if (c->ws && !c->ws_owned) return RT_OK;
    size_t want = align_up(sizeof(Counters)) + (size_t)nrays * per_ray + 4 * kAlign;
    size_t freeb = 0, total = 0;
    CK(cudaMemGetInfo(&freeb, &total));
    size_t avail = c->ws_bytes + (size_t)(0.6 * (double)freeb);
    size_t bytes = std::min(want, avail);
    if (bytes < rt_workspace_min_bytes()) return RT_ERR_NOMEM;
    if (c->ws_owned && c->ws_bytes >= bytes) return RT_OK;
    if (c->ws_owned) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    if (cudaMalloc(&c->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    c->ws_bytes = bytes;
    c->ws_owned = true;
    return RT_OK;
}

static int ensure_stage(void **buf, size_t *have, size_t need) {
    if (*have >= need) return RT_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    *have = need;
    return RT_OK;
}

// Surrogate-form arguments of a transfer: where the network's inputs and outputs of each
// saved state live, its normalisation and its input box.
static void set_surrogate_args(const rt_ctx *c, XferArgs &xa, float4 *feat, float *sur_y) {
    xa.feat = feat;
    xa.sur_y = sur_y;
    xa.sur_norm = reinterpret_cast<const float *>(c->d_mlpaux) + 4;
    for (int j = 0; j < 4; j++) {
        xa.sur_lo[j] = c->mlp_norm.lo[j];
        xa.sur_hi[j] = c->mlp_norm.hi[j];
    }
}

// The network's inputs for every saved state of a chunk, then one tensor-core pass over
// them; the pass reads the number of arena blocks in use on the device.
static void launch_network_pass(const rt_ctx *c, const XferArgs &xa, float *sur_y, long long nblocks,
                                const unsigned long long *used_blocks, int xf_grid, cudaStream_t s) {
    launch_sur_features(xa, xf_grid, s);
    long long rows = nblocks * kBlockStates;
    launch_mlp_forward(reinterpret_cast<const float *>(xa.feat), sur_y, rows, c->d_wpk,
                       reinterpret_cast<unsigned *>(c->d_mlpaux) + 1,
                       (int)std::min<long long>((rows + 127) / 128, (long long)c->nsm * 4), s, used_blocks,
                       kBlockStates);
}

// The same for the rays of xa in the streamed shape: the features pass hands each ray
// consecutive compact rows (xa.sur_row maps every saved state to its row), and the network runs
// over the rows handed out, a count it reads on the device. max_rows bounds the rows.
static int launch_network_pass_rows(const rt_ctx *c, const XferArgs &xa, float *sur_y, Counters *ctr,
                                    long long max_rows, int xf_grid, cudaStream_t s) {
    CK(cudaMemsetAsync(&ctr->feat_next, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(&ctr->sur_rows, 0, sizeof(unsigned long long), s));
    launch_sur_features(xa, xf_grid, s);
    launch_mlp_forward(reinterpret_cast<const float *>(xa.feat), sur_y, max_rows, c->d_wpk,
                       reinterpret_cast<unsigned *>(c->d_mlpaux) + 1,
                       (int)std::min<long long>((max_rows + 127) / 128, (long long)c->nsm * 4), s, &ctr->sur_rows, 1);
    return RT_OK;
}

// Streams, events and the second pinned counter block of the overlapped render, made on first use.
static int ensure_overlap(rt_ctx *c) {
    for (int i = 0; i < 2; i++)
        if (!c->ostream[i] && cudaStreamCreateWithFlags(&c->ostream[i], cudaStreamNonBlocking) != cudaSuccess)
            return RT_ERR_CUDA;
    if (!c->h_ctr2 && cudaMallocHost(&c->h_ctr2, sizeof(Counters)) != cudaSuccess) return RT_ERR_CUDA;
    if (!c->h_flags) {
        if (cudaHostAlloc(&c->h_flags, sizeof(unsigned) * rt_ctx::kMaxChunks, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            c->h_flags = nullptr;
            return RT_ERR_CUDA;
        }
        if (cudaHostGetDevicePointer((void **)&c->d_flags, c->h_flags, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(c->h_flags);
            c->h_flags = nullptr;
            return RT_ERR_CUDA;
        }
    }
    if (!c->have_oev) {
        for (int i = 0; i < 4 * rt_ctx::kMaxChunks; i++)
            if (cudaEventCreate(&c->oev[i]) != cudaSuccess) {
                for (int j = 0; j < i; j++) cudaEventDestroy(c->oev[j]);
                return RT_ERR_CUDA;
            }
        c->have_oev = true;
    }
    return RT_OK;
}

// Step-count and order arrays for npix pixels; a camera or integrator other than the one the
// recorded steps belong to drops them.
static int prepare_order(rt_ctx *c, const Camera &cam, long long npix) {
    const double key[8] = {cam.a, cam.r_cam, cam.theta_o, cam.fov, (double)cam.nx, (double)cam.ny, cam.eps,
                           (double)cam.nmax};
    if (memcmp(key, c->order_key, sizeof(key)) != 0) {
        memcpy(c->order_key, key, sizeof(key));
        c->have_steps = false;
        c->steps_probed = false;
        c->order_K = 0;
    }
    if (npix > c->order_cap) {
        cudaFree(c->d_steps);
        cudaFree(c->d_order);
        c->d_steps = nullptr;
        c->d_order = nullptr;
        c->order_cap = 0;
        c->have_steps = false;
        c->steps_probed = false;
        c->order_K = 0;
        if (cudaMalloc(&c->d_steps, sizeof(uint16_t) * npix) != cudaSuccess ||
            cudaMalloc(&c->d_order, sizeof(int) * npix) != cudaSuccess) {
            cudaGetLastError();
            return RT_ERR_NOMEM;
        }
        c->order_cap = npix;
    }
    if (!c->d_ohist && cudaMalloc(&c->d_ohist, sizeof(unsigned) * kOrderBuckets) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    return RT_OK;
}

// Predicted step counts for a new camera: trace the ray through the centre of every
// kProbeStride x kProbeStride block (1/64 of the rays) with the one-pass carving of the
// workspace, record their steps, and give every other pixel its block's count. Skipped when
// the workspace's first chunk cannot hold the probe.
constexpr int kProbeStride = 8;
static int probe_steps(rt_ctx *c, const Camera &cam, Counters *ctr, RayRecord *rec, long long cap, const Arena &ar) {
    const long long np = (long long)((cam.nx + kProbeStride - 1) / kProbeStride) *
                         ((cam.ny + kProbeStride - 1) / kProbeStride);
    if (np > cap) return RT_OK;
    if (np > c->probe_cap) {
        cudaFree(c->d_probe);
        c->d_probe = nullptr;
        c->probe_cap = 0;
        if (cudaMalloc(&c->d_probe, sizeof(int) * np) != cudaSuccess) {
            cudaGetLastError();
            return RT_ERR_NOMEM;
        }
        c->probe_cap = np;
    }
    launch_probe_list(c->d_probe, cam.nx, cam.ny, kProbeStride, c->stream);
    CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), c->stream));
    GeoArgs ga{cam, c->d_sctab, ar, rec, ctr, np, 0};
    ga.pix_list = c->d_probe;
    ga.steps_out = c->d_steps;
    launch_geodesic(ga, c->nsm * c->geo_bps, c->stream);
    launch_steps_fill(c->d_steps, cam.nx, cam.ny, kProbeStride, c->stream);
    CK(cudaGetLastError());
    c->have_steps = true;
    c->steps_probed = true;
    c->order_K = 0;
    return RT_OK;
}

// Chunk layout of an overlapped render of nrays rays: at least `chunks` chunks, the last with
// 1/W of a regular one's share, more chunks when a workspace half cannot hold the largest;
// K = 0 when that would need more than kMaxChunks.
static ChunkLayout overlap_chunks(const rt_ctx *c, long long nrays, int chunks, int W, size_t per_ray) {
    const size_t half = (c->ws_bytes / 2) & ~(size_t)(kAlign - 1);
    const size_t off_rec = align_up(sizeof(Counters));
    ChunkLayout L{nrays, 0, W};
    if (half < off_rec + 6 * kAlign + per_ray) return L;
    long long cap = (long long)((half - off_rec - 6 * kAlign) / per_ray);
    long long K = std::min<long long>(std::max<long long>(chunks, (nrays + cap - 1) / cap), nrays);
    for (; K <= rt_ctx::kMaxChunks; K++) {
        L.K = (int)K;
        if (L.max_size() <= cap) return L;
    }
    L.K = 0;
    return L;
}

// Registers of a block (allocated per warp, in units of 256) and the transfer blocks per SM that
// fit in the register file beside geo_b geodesic blocks, at most xf_b and at least 1.
static int block_regs(int regs, int threads) { return ((regs * 32 + 255) / 256) * 256 * ((threads + 31) / 32); }
static int xf_beside_geo(const rt_ctx *c, int form, int geo_b, int xf_b) {
    const int xr = block_regs(form == RT_FP64 ? c->xf_regs_fp64 : c->xf_regs_mixed, kXferThreads);
    const int room = c->regs_per_sm - geo_b * block_regs(c->geo_regs, kGeoThreads);
    const int fit = room > 0 ? room / xr : 0;
    return std::max(1, std::min(xf_b, fit));
}

// Overlapped render. The rays are split into K chunks that alternate between two halves of the
// workspace, each half with its own counters, ray records and arena. Chunk i's geodesic runs on
// ostream[0] once the transfer of chunk i - 2 (the same half) has finished, and its transfer on
// ostream[1] once its geodesic has; so the geodesic of chunk i + 1 shares the SMs with the
// transfer of chunk i. (A second geodesic stream, letting chunk i + 1's geodesic start beside
// chunk i's, was slower: the two geodesics crowded the transfer out of the SMs.) Returns
// RT_ERR_NOMEM when a half cannot hold a chunk of at most kMaxChunks-th of the rays.
static int render_overlap(rt_ctx *c, int form, int coef, const Camera &cam, const Model &mod, const int *list,
                          uint16_t *steps_out, const ChunkLayout &L, void *d_out, uint8_t *d_status,
                          void *d_depth, int geo_grid, int xf_grid, const JobDev *jobs = nullptr, int njobs = 0) {
    const long long K = L.K;
    const bool sur = form == RT_SURROGATE;
    // per arena block: the states and the prev link, and for the surrogate form the network's
    // inputs and outputs of each state (16 + 32 bytes)
    const size_t per_block = kBlockBytes + (sur ? (size_t)kBlockStates * 48 : 0);
    int rv = ensure_overlap(c);
    if (rv) return rv;
    const size_t half = (c->ws_bytes / 2) & ~(size_t)(kAlign - 1);
    const size_t off_rec = align_up(sizeof(Counters));
    // chunk k: L.size(k) rays from L.offset(k) (the layout of a longest-first order)
    const long long chunk = L.max_size();
    Counters *ctr[2];
    RayRecord *rec[2];
    Arena ar[2];
    float4 *feat[2] = {nullptr, nullptr};
    float *sur_y[2] = {nullptr, nullptr};
    for (int h = 0; h < 2; h++) {
        char *base = (char *)c->ws + h * half;
        ctr[h] = (Counters *)base;
        rec[h] = (RayRecord *)(base + off_rec);
        size_t off = align_up(off_rec + sizeof(RayRecord) * chunk);
        long long nb = (long long)((half - off - 5 * kAlign) / per_block);
        ar[h].states = (PathState *)(base + off);
        ar[h].prev = (int *)(base + off + (size_t)nb * sizeof(PathState) * kBlockStates);
        ar[h].nblocks = nb;
        if (sur) {
            off = align_up(off + (size_t)nb * kBlockBytes);
            feat[h] = (float4 *)(base + off);
            off = align_up(off + (size_t)nb * kBlockStates * sizeof(float4));
            sur_y[h] = (float *)(base + off);
        }
    }
    cudaStream_t sg = c->ostream[0], st = c->ostream[1];
    cudaEvent_t *gs = c->oev, *ge = c->oev + rt_ctx::kMaxChunks, *ts = c->oev + 2 * rt_ctx::kMaxChunks,
                *te = c->oev + 3 * rt_ctx::kMaxChunks;
    CK(cudaMemsetAsync(ctr[0], 0, sizeof(Counters), c->stream));
    CK(cudaMemsetAsync(ctr[1], 0, sizeof(Counters), c->stream));
    CK(cudaEventRecord(c->ev[0], c->stream));
    CK(cudaStreamWaitEvent(sg, c->ev[0], 0));
    CK(cudaStreamWaitEvent(st, c->ev[0], 0));
    for (long long i = 0; i < K; i++) {
        const int h = (int)(i & 1);
        const long long o = L.offset((int)i), n = L.size((int)i);
        if (i >= 2) CK(cudaStreamWaitEvent(sg, te[i - 2], 0));
        CK(cudaMemsetAsync(ctr[h], 0, 4 * sizeof(unsigned long long), sg));  // queues + arena
        GeoArgs ga{cam, c->d_sctab, ar[h], rec[h], ctr[h], n, o};
        ga.pix_list = list;
        ga.steps_out = steps_out;
        ga.jobs = jobs;
        ga.njobs = njobs;
        XferArgs xa{cam, mod, ar[h], rec[h], ctr[h], n, o, d_out, d_status, d_depth};
        xa.pix_list = list;
        xa.kt = KappaTables{c->d_syn, c->d_gl, c->d_gl + 8};
        xa.jobs = jobs;
        xa.njobs = njobs;
        if (sur) set_surrogate_args(c, xa, feat[h], sur_y[h]);
        CK(cudaEventRecord(gs[i], sg));
        launch_geodesic(ga, geo_grid, sg);
        CK(cudaEventRecord(ge[i], sg));
        CK(cudaStreamWaitEvent(st, ge[i], 0));
        CK(cudaEventRecord(ts[i], st));
        if (sur) launch_network_pass(c, xa, sur_y[h], ar[h].nblocks, &ctr[h]->arena_next, xf_grid, st);
        if (form == RT_FP64)
            launch_transfer_fp64(xa, coef, xf_grid, st);
        else if (form == RT_UNPOL)
            launch_unpol(xa, xf_grid, st);
        else if (use_staged(c, form, coef, mod, jobs))
            launch_transfer_staged(xa, c->tmap, xf_grid, st);
        else
            launch_transfer_mixed(xa, coef, xf_grid, st);
        CK(cudaEventRecord(te[i], st));
        CK(cudaGetLastError());
    }
    CK(cudaStreamWaitEvent(c->stream, te[K - 1], 0));  // after every geodesic and transfer (in order)
    CK(cudaEventRecord(c->ev[2], c->stream));
    CK(cudaMemcpyAsync(c->h_ctr2, ctr[1], sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->h_ctr, ctr[0], sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    Counters &a = *c->h_ctr, &b = *c->h_ctr2;
    a.steps += b.steps;
    a.points += b.points;
    a.emitting += b.emitting;
    a.arena_next = std::max(a.arena_next, b.arena_next);
    for (int k = 0; k < 8; k++) a.n_status[k] += b.n_status[k];
    // spans: first geodesic start to last geodesic end, first transfer start to last end
    float g = 0.f, x = 0.f;
    if (cudaEventElapsedTime(&g, gs[0], ge[K - 1]) != cudaSuccess) g = 0.f;
    if (cudaEventElapsedTime(&x, ts[0], te[K - 1]) != cudaSuccess) x = 0.f;
    cudaGetLastError();
    c->last_ms_geo = g;
    c->last_ms_xfer = x;
    c->last_chunks = (int)K;
    c->last_shape = 1;
    c->last_geo_launches = c->last_xf_launches = (int)K;
    c->last_blocks_total = ar[0].nblocks;
    c->last_was_streamed = false;
    return RT_OK;
}

// Whether the workspace holds, or (when the library owns it) can grow to hold, the streamed
// shape's nrays rays; grows it then.
static bool prepare_streamed(rt_ctx *c, long long nrays, size_t per_ray = kPerRayBytes) {
    const size_t need = streamed_bytes(nrays, per_ray);
    if (c->ws_bytes >= need) return true;
    if (c->ws && !c->ws_owned) return false;
    size_t freeb = 0, total = 0;
    if (cudaMemGetInfo(&freeb, &total) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (need > c->ws_bytes + (size_t)(0.6 * (double)freeb)) return false;
    return ensure_workspace(c, nrays + 1, per_ray) == RT_OK && c->ws_bytes >= need;
}

// Pieces of a streamed render of nrays rays: 1 when the workspace holds (or can grow to hold)
// every path; otherwise as many as the workspace needs, after growing a library-owned one as
// far as ensure_workspace allows; 0 (no streamed render) beyond kMaxStreamPieces.
constexpr int kMaxStreamPieces = 64;
static int plan_pieces(rt_ctx *c, long long nrays, size_t per_ray = kPerRayBytes) {
    if (prepare_streamed(c, nrays, per_ray)) return 1;
    if (!c->ws || c->ws_owned) ensure_workspace(c, nrays + 1, per_ray);
    const size_t fixed = streamed_bytes(0, per_ray);
    if (c->ws_bytes <= fixed) return 0;
    const long long cap = (long long)((c->ws_bytes - fixed) / per_ray);
    if (cap < 1) return 0;
    for (long long P = (nrays + cap - 1) / cap; P <= kMaxStreamPieces; P++)
        if (ChunkLayout{nrays, (int)P, 1}.max_size() <= cap) return (int)P;
    return 0;
}

// Chunks per piece of a streamed render: `chunks` (set) or automatic, within kMaxChunks in all.
static int stream_chunks(long long nrays, int P, int chunks, bool automatic) {
    const long long np = ChunkLayout{nrays, P, 1}.max_size(), most = rt_ctx::kMaxChunks / P;
    long long K = automatic ? std::max<long long>(16, np >> kStreamChunkShift) : chunks;
    return (int)std::max<long long>(1, std::min(std::min(K, most), np));
}

// Longest wait of the host for one chunk of a streamed render. Every geodesic ends (its rays
// take at most nmax steps), and when it has, every chunk is complete; the bound only keeps a
// host thread from waiting without end on a GPU that no longer answers.
constexpr double kStreamWaitSeconds = 600.0;

// Streamed overlapped render, in P pieces (1 when the workspace holds every ray's path). The
// longest-first order is dealt to the pieces (ChunkLayout {n, P, 1}), so each piece holds the
// same mix of lengths, longest first, and is cut into K contiguous chunks. For each piece, one
// geodesic launch on ostream[0] traces its rays into the arena. Every ray that stops counts
// toward its chunk, and the lane that completes a chunk raises the chunk's flag in mapped host
// memory. The host watches the flags and launches the transfers of complete chunks on
// ostream[1], beside the geodesic still running, so no chunk boundary makes the geodesic's
// lanes drain; a piece ends when its last transfer has. The transfers read only the paths of
// complete chunks: each ray's states and record are released by a fence before its count, and
// a transfer is launched after the host has seen its chunks' flags.
static int render_streamed(rt_ctx *c, int form, int coef, const Camera &cam, const Model &mod, const int *list,
                           uint16_t *steps_out, long long nrays, int P, int K, void *d_out, uint8_t *d_status,
                           void *d_depth, int geo_grid, int xf_grid, int xf_grid_alone, const JobDev *jobs = nullptr,
                           int njobs = 0) {
    int rv = ensure_overlap(c);
    if (rv) return rv;
    // the surrogate form: per run of chunks, its features pass, the network over the run's
    // compact rows, then its transfer
    const bool sur = form == RT_SURROGATE;
    const size_t per_ray = sur ? kSurPerRayBytes : kPerRayBytes;
    const ChunkLayout Lp{nrays, P, 1};
    if (P < 1 || K < 1 || (long long)P * K > rt_ctx::kMaxChunks || c->ws_bytes < streamed_bytes(Lp.max_size(), per_ray))
        return RT_ERR_NOMEM;
    char *base = (char *)c->ws;
    Counters *ctr = (Counters *)base;
    size_t off = align_up(sizeof(Counters));
    unsigned *done = (unsigned *)(base + off);
    off = align_up(off + sizeof(unsigned) * rt_ctx::kMaxChunks);
    RayRecord *rec = (RayRecord *)(base + off);
    off = align_up(off + sizeof(RayRecord) * Lp.max_size());
    Arena ar;
    ar.nblocks = (long long)((c->ws_bytes - off - 6 * kAlign) / (kBlockBytes + (sur ? kSurBlockBytes : 0)));
    ar.states = (PathState *)(base + off);
    ar.prev = (int *)(base + off + (size_t)ar.nblocks * sizeof(PathState) * kBlockStates);
    float4 *feat = nullptr;
    float *sur_y = nullptr;
    int *sur_row = nullptr;
    if (sur) {
        ar.nblocks = std::min<long long>(ar.nblocks, INT_MAX / kBlockStates);  // rows are int
        ar.prev = (int *)(base + off + (size_t)ar.nblocks * sizeof(PathState) * kBlockStates);
        const size_t rows = (size_t)ar.nblocks * kBlockStates;
        off = align_up(off + (size_t)ar.nblocks * kBlockBytes);
        feat = (float4 *)(base + off);
        off = align_up(off + rows * sizeof(float4));
        sur_y = (float *)(base + off);
        off = align_up(off + rows * 8 * sizeof(float));
        sur_row = (int *)(base + off);
    }
    cudaStream_t sg = c->ostream[0], st = c->ostream[1];
    cudaEvent_t *gs = c->oev, *ge = c->oev + rt_ctx::kMaxChunks, *ts = c->oev + 2 * rt_ctx::kMaxChunks,
                *te = c->oev + 3 * rt_ctx::kMaxChunks;
    // no launch of an earlier call may still write the flags
    CK(cudaStreamSynchronize(sg));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), c->stream));
    CK(cudaEventRecord(c->ev[0], c->stream));
    CK(cudaStreamWaitEvent(sg, c->ev[0], 0));
    CK(cudaStreamWaitEvent(st, c->ev[0], 0));
    const auto t0 = std::chrono::steady_clock::now();
    unsigned long long arena_max = 0;
    int first = -1, last = -1, xf_launches = 0;
    for (int p = 0; p < P; p++) {
        const long long o_p = Lp.offset(p), n_p = Lp.size(p);
        const ChunkLayout L{n_p, (int)std::min<long long>(K, std::max<long long>(n_p, 1)), 1};
        const int base_k = p * K;  // this piece's chunks are base_k .. base_k + L.K - 1
        if (p > 0) {  // the previous piece has ended: its arena and records are free
            CK(cudaStreamSynchronize(st));
            CK(cudaMemcpyAsync(&c->h_ctr2->arena_next, &ctr->arena_next, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, sg));
            CK(cudaStreamSynchronize(sg));
            arena_max = std::max(arena_max, (unsigned long long)c->h_ctr2->arena_next);
        }
        memset(c->h_flags, 0, sizeof(unsigned) * L.K);
        CK(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), sg));  // queues + arena
        CK(cudaMemsetAsync(done, 0, sizeof(unsigned) * L.K, sg));
        GeoArgs ga{cam, c->d_sctab, ar, rec, ctr, n_p, o_p};
        ga.pix_list = list;
        ga.steps_out = steps_out;
        ga.jobs = jobs;
        ga.njobs = njobs;
        ga.chunk_done = done;
        ga.chunk_flag = c->d_flags;
        ga.layout = L;
        CK(cudaEventRecord(gs[p], sg));
        if (n_p > 0) launch_geodesic(ga, geo_grid, sg);
        CK(cudaEventRecord(ge[p], sg));
        CK(cudaGetLastError());

        // Launch every run of consecutive chunks that are complete and not yet launched as one
        // transfer (a chunk of long rays may complete after later ones), at the occupancy that
        // fits beside the geodesic, or at the transfer's own once the geodesic has ended. At
        // most one launch waits behind the running one: a new launch is made once the previous
        // has started, so the chunks that complete meanwhile join one launch instead of queueing
        // one each (a launch lasts at least as long as its longest ray's transfer).
        std::vector<char> launched(L.K, 0);
        int left = L.K, prev = -1;
        for (int k = 0; k < L.K; k++)
            if (L.size(k) == 0) {
                launched[k] = 1;
                left--;
            }
        while (left > 0) {
            const cudaError_t q = cudaEventQuery(ge[p]);  // before the flags: then all are final
            if (q != cudaSuccess && q != cudaErrorNotReady) {
                cudaGetLastError();
                cudaStreamSynchronize(st);
                return RT_ERR_CUDA;
            }
            cudaGetLastError();  // a not-ready query
            bool any = false, ready = false;
            bool may = prev < 0 || cudaEventQuery(ts[base_k + prev]) == cudaSuccess;
            cudaGetLastError();
            for (int a = 0; a < L.K;) {
                if (launched[a] || !__atomic_load_n(&c->h_flags[a], __ATOMIC_ACQUIRE)) {
                    a++;
                    continue;
                }
                ready = true;
                if (!may) break;
                int b = a + 1;
                while (b < L.K && !launched[b] && __atomic_load_n(&c->h_flags[b], __ATOMIC_ACQUIRE)) b++;
                const long long o = L.offset(a), n = L.offset(b - 1) + L.size(b - 1) - o;
                XferArgs xa{cam, mod, ar, rec + o, ctr, n, o_p + o, d_out, d_status, d_depth};
                xa.pix_list = list;
                xa.kt = KappaTables{c->d_syn, c->d_gl, c->d_gl + 8};
                xa.jobs = jobs;
                xa.njobs = njobs;
                const int grid = q == cudaSuccess ? xf_grid_alone : xf_grid;
                CK(cudaMemsetAsync(&ctr->xfer_next, 0, sizeof(unsigned long long), st));
                for (int k = a; k < b; k++) CK(cudaEventRecord(ts[base_k + k], st));
                if (sur) {
                    set_surrogate_args(c, xa, feat, sur_y);
                    xa.sur_row = sur_row;
                    rv = launch_network_pass_rows(c, xa, sur_y, ctr, (long long)ar.nblocks * kBlockStates, grid, st);
                    if (rv) return rv;
                }
                if (form == RT_FP64)
                    launch_transfer_fp64(xa, coef, grid, st);
                else if (form == RT_UNPOL)
                    launch_unpol(xa, grid, st);
                else if (use_staged(c, form, coef, mod, jobs))
                    launch_transfer_staged(xa, c->tmap, grid, st);
                else
                    launch_transfer_mixed(xa, coef, grid, st);
                for (int k = a; k < b; k++) {
                    CK(cudaEventRecord(te[base_k + k], st));
                    launched[k] = 1;
                }
                CK(cudaGetLastError());
                if (first < 0) first = base_k + a;
                last = base_k + b - 1;
                xf_launches++;
                prev = a;
                left -= b - a;
                any = true;
                may = false;  // the next launch waits until this one has started
                a = b;
            }
            if (any || left == 0) continue;
            if (q == cudaSuccess && !ready) {  // the geodesic has ended, and a chunk is still incomplete
                cudaStreamSynchronize(st);
                return RT_ERR_CUDA;
            }
            if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > kStreamWaitSeconds)
                return RT_ERR_STALL;
            std::this_thread::yield();
        }
    }
    CK(cudaStreamWaitEvent(c->stream, ge[P - 1], 0));
    if (last >= 0) CK(cudaStreamWaitEvent(c->stream, te[last], 0));  // the transfers run in order on st
    CK(cudaEventRecord(c->ev[2], c->stream));
    CK(cudaMemcpyAsync(c->h_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->h_ctr->arena_next = std::max(arena_max, (unsigned long long)c->h_ctr->arena_next);
    float g = 0.f, x = 0.f;
    if (cudaEventElapsedTime(&g, gs[0], ge[P - 1]) != cudaSuccess) g = 0.f;
    if (first >= 0 && cudaEventElapsedTime(&x, ts[first], te[last]) != cudaSuccess) x = 0.f;
    cudaGetLastError();
    c->last_ms_geo = g;
    c->last_ms_xfer = x;
    c->last_chunks = P * K;
    c->last_pieces = P;
    c->last_shape = 2;
    c->last_geo_launches = P;
    c->last_xf_launches = xf_launches;
    c->last_blocks_total = ar.nblocks;
    c->last_was_streamed = true;
    return RT_OK;
}

}  // extern "C"

// The batched form in the overlapped two-kernel shape: the rays of njobs images (the job table
// d_jobs on the device, h_jobs its host copy, ray_begin filled) form one ray space, chunked and
// overlapped like one large image, on the context's stream. Thermal electrons, RT_FP64 or
// RT_MIXED. Synchronizes; the counters describe the whole batch.
int render_jobs_overlap(rt_ctx *c, int form, const JobDev *d_jobs, const JobDev *h_jobs, int njobs, long long nrays) {
    const size_t per_ray = kPerRayBytes;
    const int chunks = (int)std::min<long long>(64, std::max<long long>(2, nrays >> kAutoChunkShift));
    // streamed, in pieces of the ray space that the workspace holds (up to kMaxStreamPieces),
    // else in two halves
    const int P = plan_pieces(c, nrays), Kp = P > 0 ? stream_chunks(nrays, P, 0, true) : 0;
    const bool streamed = P > 0;
    ChunkLayout L{nrays, (int)std::min<long long>(chunks, nrays), kAutoLastDiv};
    if (!streamed) {
        long long ws_rays = 2 * L.max_size() +
                            2 * (long long)((align_up(sizeof(Counters)) + 6 * kAlign + per_ray - 1) / per_ray) + 1;
        int rv = ensure_workspace(c, ws_rays, per_ray);
        if (rv) return rv;
        L = overlap_chunks(c, nrays, chunks, kAutoLastDiv, per_ray);
        if (L.K == 0) return RT_ERR_NOMEM;
    }
    const long long K = L.K;
    int rv = RT_OK;
    const int xf_own = form == RT_FP64 ? c->fp64_bps : c->mixed_bps, geo_b = streamed ? kStreamGeoBlocks : 1;
    const int geo_grid = c->nsm * geo_b, xf_grid = c->nsm * xf_beside_geo(c, form, geo_b, xf_own);
    // longest first, as for one image, once a batch of the same cameras has recorded its steps
    unsigned long long key = 1469598103934665603ull;  // FNV-1a over the cameras and integrator
    auto mix = [&](const void *v, size_t n) {
        for (size_t i = 0; i < n; i++) key = (key ^ ((const unsigned char *)v)[i]) * 1099511628211ull;
    };
    for (int j = 0; j < njobs; j++) {
        const Camera &cj = h_jobs[j].cam;
        const double f[6] = {cj.a, cj.r_cam, cj.theta_o, cj.fov, cj.eps, (double)cj.nmax};
        const int d[2] = {cj.nx, cj.ny};
        mix(f, sizeof(f));
        mix(d, sizeof(d));
    }
    if (key != c->bkey || nrays > c->border_cap) {
        c->bkey = key;
        c->have_bsteps = false;
        c->border_K = 0;
    }
    if (nrays > c->border_cap) {
        cudaFree(c->d_bsteps);
        cudaFree(c->d_border);
        c->d_bsteps = nullptr;
        c->d_border = nullptr;
        c->border_cap = 0;
        if (cudaMalloc(&c->d_bsteps, sizeof(uint16_t) * nrays) != cudaSuccess ||
            cudaMalloc(&c->d_border, sizeof(int) * nrays) != cudaSuccess) {
            cudaGetLastError();
            return RT_ERR_NOMEM;
        }
        c->border_cap = nrays;
    }
    if (!c->d_ohist && cudaMalloc(&c->d_ohist, sizeof(unsigned) * kOrderBuckets) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    const int *list = nullptr;
    if (c->have_bsteps) {
        // streamed: one longest-first order, cut into contiguous chunks; halves: dealt
        const ChunkLayout Lord = streamed ? ChunkLayout{nrays, P, 1} : L;
        if (c->border_K != Lord.K || c->border_W != Lord.W) {
            launch_order_build(c->d_bsteps, Lord, c->d_ohist, c->d_border, c->stream);
            CK(cudaGetLastError());
            c->border_K = Lord.K;
            c->border_W = Lord.W;
        }
        list = c->d_border;
    }
    if (streamed)
        rv = render_streamed(c, form, 0, h_jobs[0].cam, h_jobs[0].model, list, c->d_bsteps, nrays, P, Kp, nullptr,
                             nullptr, nullptr, geo_grid, xf_grid, c->nsm * xf_own, d_jobs, njobs);
    else
        rv = render_overlap(c, form, 0, h_jobs[0].cam, h_jobs[0].model, list, c->d_bsteps, L, nullptr, nullptr,
                            nullptr, geo_grid, xf_grid, d_jobs, njobs);
    if (rv) return rv;
    c->last_rays = nrays;
    c->last_was_overlap = true;
    if (c->h_ctr->n_status[kOverflow] > 0) return RT_ERR_WORKSPACE;
    c->have_bsteps = true;
    return RT_OK;
}

extern "C" {

static int render_impl(rt_ctx *c, int form, void *out_iquv, uint8_t *status, void *depth, const int *list = nullptr,
                       long long nlist = 0) {
    if (!c || !out_iquv || form < RT_FP64 || form > RT_UNPOL) return RT_ERR_INVALID;
    if (form == RT_UNPOL && depth) return RT_ERR_INVALID;
    if (!c->have_cam || !c->have_model) return RT_ERR_NOT_READY;
    CK(cudaSetDevice(c->device));
    int qv = quiesce_overlap(c);
    if (qv) return qv;
    const rt_camera &rc = c->cam;
    long long nrays = list ? nlist : (long long)rc.nx * rc.ny;
    if (nrays == 0) return RT_OK;
    const long long npix_img = (long long)rc.nx * rc.ny;

    // camera and model in kernel form
    Camera cam = make_camera(rc, c->eps, c->nmax);
    Model mod = make_model(c, cam);
    const bool sur = form == RT_SURROGATE;
    if (sur && (mod.edf != RT_EDF_KAPPA || !c->have_mlp)) return RT_ERR_NOT_READY;
    if (form == RT_UNPOL && mod.edf != RT_EDF_THERMAL) return RT_ERR_INVALID;
    const size_t ncomp = form == RT_UNPOL ? 1 : 4;  // values per pixel
    const int coef = mod.edf != RT_EDF_KAPPA ? 0 : (sur ? 2 : 1);
    if (sur) CK(cudaMemsetAsync(reinterpret_cast<unsigned *>(c->d_mlpaux) + 1, 0, sizeof(unsigned), c->stream));

    // workspace carving; the surrogate form adds, per saved state, the network's inputs and
    // outputs (16 + 32 bytes)
    const size_t per_ray = kPerRayBytes + (sur ? (size_t)kBudgetBlocksPerRay * kBlockStates * 48 : 0);

    // launch shape: the configured one, or automatic. RT_MIXED and RT_UNPOL overlap images of
    // 2^19 rays or more: streamed (chunks of about 2^15 rays, the geodesic at 2 blocks per SM)
    // when the workspace holds a piece of at least 1/64 of the rays, else in two workspace
    // halves (4 to 16 chunks of about 2^17 rays, the geodesic at 1 block per SM beside the
    // transfer). Smaller images run one pass of each kernel, and so do RT_FP64 (its FP64
    // transfer competes with the geodesic for the same pipe) and RT_SURROGATE (the network pass
    // beside the geodesic measured slower than one pass: 859 against 536 ms).
    int chunks = c->rcfg.chunks, geo_b = c->rcfg.geo_blocks_per_sm, W = c->rcfg.last_chunk_div;
    const bool auto_shape = chunks == 0;
    if (auto_shape)
        chunks = nrays >= (1ll << 19) && (form == RT_MIXED || form == RT_UNPOL)
                     ? (int)std::min<long long>(kAutoChunksMax, std::max<long long>(4, nrays >> kAutoChunkShift))
                     : 1;
    bool ovl = chunks >= 2 && nrays >= 2;
    // the streamed shape, in pieces that the workspace holds (the surrogate form's network then
    // runs over compact rows of each transfer launch's rays); else two halves of the workspace
    // that hold a chunk each, with their own counters
    int rv = RT_OK, P = ovl ? plan_pieces(c, nrays, sur ? kSurPerRayBytes : kPerRayBytes) : 0, Kp = 0;
    const bool streamed = P > 0;
    ChunkLayout L{nrays, 1, 1};
    if (streamed) {
        // contiguous ranges of each piece's longest-first order; the automatic shape takes finer
        // chunks and a second geodesic block per SM
        Kp = stream_chunks(nrays, P, chunks, auto_shape);
        if (geo_b == 0) geo_b = kStreamGeoBlocks;
    } else {
        if (ovl && geo_b == 0) geo_b = 1;
        if (W == 0) W = auto_shape ? kAutoLastDiv : 1;
        long long ws_rays = nrays;
        if (ovl)
            ws_rays = 2 * ChunkLayout{nrays, chunks, W}.max_size() +
                      2 * (long long)((align_up(sizeof(Counters)) + 6 * kAlign + per_ray - 1) / per_ray) + 1;
        rv = ensure_workspace(c, ws_rays, per_ray);
        if (rv) return rv;
        if (ovl) {
            // a workspace too small for kMaxChunks (256) overlapped chunks (a caller's, or a
            // nearly full device) renders in one pass of each kernel per chunk instead
            L = overlap_chunks(c, nrays, chunks, W, per_ray);
            if (L.K == 0) {
                ovl = false;
                L = ChunkLayout{nrays, 1, 1};
            }
        }
    }

    // one-pass shape: as many rays per chunk as the workspace holds; the Kseq chunks are those of
    // the layout {n, Kseq, 1} (chunk k from k (n / Kseq) + min(k, n % Kseq)), so that with the
    // longest-first order every chunk holds the same mix of lengths and none outgrows the
    // arena's per-ray budget
    const size_t per_block = kBlockBytes + (sur ? (size_t)kBlockStates * 48 : 0);
    char *base = (char *)c->ws;
    Counters *ctr = (Counters *)base;
    size_t off = align_up(sizeof(Counters));
    size_t room = c->ws_bytes - off - 3 * kAlign;
    long long chunk = std::min<long long>(nrays, (long long)(room / per_ray));
    if (chunk < 1) return RT_ERR_NOMEM;
    const long long Kseq = (nrays + chunk - 1) / chunk;

    RayRecord *rec = (RayRecord *)(base + off);
    off = align_up(off + sizeof(RayRecord) * chunk);
    long long nblocks = (long long)((c->ws_bytes - off - 3 * kAlign) / per_block);
    Arena ar;
    ar.states = (PathState *)(base + off);
    ar.prev = (int *)(base + off + (size_t)nblocks * sizeof(PathState) * kBlockStates);
    ar.nblocks = nblocks;
    float4 *feat = nullptr;
    float *sur_y = nullptr;
    if (sur) {
        off = align_up(off + (size_t)nblocks * kBlockBytes);
        feat = (float4 *)(base + off);
        off = align_up(off + (size_t)nblocks * kBlockStates * sizeof(float4));
        sur_y = (float *)(base + off);
    }

    // ray order: longest first once a render of this camera has recorded its step counts, or,
    // for a new camera of 2^18 rays or more, as a probe of one ray per 8 x 8 block predicts them
    const int *ray_list = list;
    uint16_t *steps_out = nullptr;
    if (!list) {
        rv = prepare_order(c, cam, npix_img);
        if (rv) return rv;
        steps_out = c->d_steps;
        // streamed: one longest-first order, cut into contiguous chunks; halves and one pass: dealt
        const ChunkLayout Lord = streamed ? ChunkLayout{npix_img, P, 1}
                                 : ovl    ? ChunkLayout{npix_img, L.K, L.W}
                                          : ChunkLayout{npix_img, (int)Kseq, 1};
        if (!c->have_steps && nrays >= (1ll << 18)) {
            rv = probe_steps(c, cam, ctr, rec, chunk, ar);
            if (rv) return rv;
        }
        if (c->have_steps) {
            if (c->order_K != Lord.K || c->order_W != Lord.W) {
                launch_order_build(c->d_steps, Lord, c->d_ohist, c->d_order, c->stream);
                CK(cudaGetLastError());
                c->order_K = Lord.K;
                c->order_W = Lord.W;
            }
            ray_list = c->d_order;
        }
    }

    // outputs: device directly, or staged
    size_t esz = form == RT_FP64 ? sizeof(double) : sizeof(float);
    bool out_dev = is_device_ptr(out_iquv);
    bool st_dev = status ? is_device_ptr(status) : true;
    void *d_out = out_iquv;
    uint8_t *d_status = status;
    if (!out_dev) {
        rv = ensure_stage(&c->d_stage, &c->stage_bytes, (size_t)npix_img * ncomp * esz);
        if (rv) return rv;
        d_out = c->d_stage;
    }
    if (status && !st_dev) {
        rv = ensure_stage((void **)&c->d_stage_status, &c->stage_status_bytes, (size_t)npix_img);
        if (rv) return rv;
        d_status = c->d_stage_status;
    }
    bool dep_dev = depth ? is_device_ptr(depth) : true;
    void *d_depth = depth;
    if (depth && !dep_dev) {
        rv = ensure_stage(&c->d_stage_depth, &c->stage_depth_bytes, (size_t)npix_img * 2 * esz);
        if (rv) return rv;
        d_depth = c->d_stage_depth;
    }

    const int xf_max = form == RT_FP64 ? c->fp64_bps : c->mixed_bps;
    const int geo_bps = geo_b > 0 ? geo_b : c->geo_bps;
    const int geo_grid = c->nsm * geo_bps;
    const int xf_own = c->rcfg.xfer_blocks_per_sm > 0 ? std::min(c->rcfg.xfer_blocks_per_sm, xf_max) : xf_max;
    // overlapped: no more transfer blocks per SM than fit beside the geodesic's
    const int xf_grid = c->nsm * (ovl ? xf_beside_geo(c, form, geo_bps, xf_own) : xf_own);
    c->last_was_overlap = false;
    c->last_was_streamed = false;
    if (ovl) {
        if (streamed)
            rv = render_streamed(c, form, coef, cam, mod, ray_list, steps_out, nrays, P, Kp, d_out, d_status, d_depth,
                                 geo_grid, xf_grid, c->nsm * xf_own);
        else
            rv = render_overlap(c, form, coef, cam, mod, ray_list, steps_out, L, d_out, d_status, d_depth, geo_grid,
                                xf_grid);
        if (rv) return rv;
        c->last_was_overlap = true;
    } else {
        CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), c->stream));
        c->last_chunks = (int)Kseq;
        c->last_shape = 0;
        c->last_geo_launches = c->last_xf_launches = (int)Kseq;
        const long long base_n = nrays / Kseq, extra = nrays % Kseq;
        for (long long k = 0; k < Kseq; k++) {
            const long long o = k * base_n + std::min(k, extra), n = base_n + (k < extra ? 1 : 0);
            CK(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), c->stream));  // queues + arena
            GeoArgs ga{cam, c->d_sctab, ar, rec, ctr, n, o};
            ga.pix_list = ray_list;
            ga.steps_out = steps_out;
            XferArgs xa{cam, mod, ar, rec, ctr, n, o, d_out, d_status, d_depth};
            xa.pix_list = ray_list;
            xa.kt = KappaTables{c->d_syn, c->d_gl, c->d_gl + 8};
            if (sur) set_surrogate_args(c, xa, feat, sur_y);
            if (k == 0) CK(cudaEventRecord(c->ev[0], c->stream));
            launch_geodesic(ga, geo_grid, c->stream);
            if (sur) launch_network_pass(c, xa, sur_y, nblocks, &ctr->arena_next, xf_grid, c->stream);
            if (k == 0) CK(cudaEventRecord(c->ev[1], c->stream));
            if (form == RT_FP64)
                launch_transfer_fp64(xa, coef, xf_grid, c->stream);
            else if (form == RT_UNPOL)
                launch_unpol(xa, xf_grid, c->stream);
            else if (use_staged(c, form, coef, mod, nullptr))
                launch_transfer_staged(xa, c->tmap, xf_grid, c->stream);
            else
                launch_transfer_mixed(xa, coef, xf_grid, c->stream);
            CK(cudaGetLastError());
        }
        CK(cudaEventRecord(c->ev[2], c->stream));
        CK(cudaMemcpyAsync(c->h_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
        c->last_blocks_total = nblocks;
    }
    if (!out_dev) CK(cudaMemcpyAsync(out_iquv, d_out, (size_t)npix_img * ncomp * esz, cudaMemcpyDeviceToHost, c->stream));
    if (status && !st_dev)
        CK(cudaMemcpyAsync(status, d_status, (size_t)npix_img, cudaMemcpyDeviceToHost, c->stream));
    if (depth && !dep_dev)
        CK(cudaMemcpyAsync(depth, d_depth, (size_t)npix_img * 2 * esz, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->last_rays = nrays;
    c->last_was_batch = false;
    if (sur) {  // a bounded wait of the network pass that ran out
        unsigned err = 0;
        CK(cudaMemcpy(&err, reinterpret_cast<unsigned *>(c->d_mlpaux) + 1, sizeof(unsigned), cudaMemcpyDeviceToHost));
        if (err) return RT_ERR_STALL;
    }
    if (c->h_ctr->n_status[kStageStatus] > 0) return RT_ERR_STALL;
    if (c->h_ctr->n_status[kOverflow] > 0) return RT_ERR_WORKSPACE;
    if (steps_out) {  // every ray of this camera recorded its steps
        c->have_steps = true;
        if (c->steps_probed) {  // the order came from the probe: rebuild it from the counts
            c->steps_probed = false;
            c->order_K = 0;
        }
    }
    return RT_OK;
}

int rt_render_features(rt_ctx *c, float *feat, long long cap, long long *count) {
    if (!c || !feat || cap < 0 || !count) return RT_ERR_INVALID;
    if (!c->have_cam || !c->have_model) return RT_ERR_NOT_READY;
    if (!is_device_ptr(feat)) return RT_ERR_INVALID;
    CK(cudaSetDevice(c->device));
    int qv = quiesce_overlap(c);
    if (qv) return qv;
    const rt_camera &rc = c->cam;
    long long nrays = (long long)rc.nx * rc.ny;
    int rv = ensure_workspace(c, nrays);
    if (rv) return rv;
    Camera cam = make_camera(rc, c->eps, c->nmax);
    Model mod = make_model(c, cam);
    char *base = (char *)c->ws;
    Counters *ctr = (Counters *)base;
    size_t off = align_up(sizeof(Counters));
    long long chunk = std::min<long long>(nrays, (long long)((c->ws_bytes - off - kAlign) / kPerRayBytes));
    if (chunk < 1) return RT_ERR_NOMEM;
    RayRecord *rec = (RayRecord *)(base + off);
    off = align_up(off + sizeof(RayRecord) * chunk);
    long long nblocks = (long long)((c->ws_bytes - off - kAlign) / kBlockBytes);
    Arena ar;
    ar.states = (PathState *)(base + off);
    ar.prev = (int *)(base + off + (size_t)nblocks * sizeof(PathState) * kBlockStates);
    ar.nblocks = nblocks;
    CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), c->stream));
    for (long long o = 0; o < nrays; o += chunk) {
        long long n = std::min(chunk, nrays - o);
        CK(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), c->stream));
        GeoArgs ga{cam, c->d_sctab, ar, rec, ctr, n, o};
        XferArgs xa{cam, mod, ar, rec, ctr, n, o, nullptr, nullptr, nullptr};
        for (int j = 0; j < 4; j++) {
            xa.sur_lo[j] = 0.f;
            xa.sur_hi[j] = 1.f;
        }
        xa.feat_raw = reinterpret_cast<float4 *>(feat);
        xa.feat_cap = cap;
        launch_geodesic(ga, c->nsm * c->geo_bps, c->stream);
        launch_sur_features(xa, c->nsm * c->mixed_bps, c->stream);
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(c->h_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *count = (long long)c->h_ctr->feat_count;
    return RT_OK;
}

int rt_render(rt_ctx *c, int form, void *out_iquv, uint8_t *status) {
    return render_impl(c, form, out_iquv, status, nullptr);
}

}  // extern "C"

namespace prt {
// Render only the listed pixels (device list of iy nx + ix) into the full-size device outputs.
int render_pixel_list(rt_ctx *c, int form, void *out, uint8_t *status, const int *list, long long n) {
    return render_impl(c, form, out, status, nullptr, list, n);
}
}  // namespace prt

extern "C" {

int rt_render_depths(rt_ctx *c, int form, void *out_iquv, uint8_t *status, void *out_depth) {
    if (!out_depth) return RT_ERR_INVALID;
    return render_impl(c, form, out_iquv, status, out_depth);
}

int rt_image_stats(rt_ctx *c, const void *iquv, int form, double *flux_jy, double *lp_frac, double *cp_frac) {
    if (!c || !iquv || form < RT_FP64 || form > RT_UNPOL) return RT_ERR_INVALID;
    if (!c->have_cam) return RT_ERR_NOT_READY;
    CK(cudaSetDevice(c->device));
    long long npix = (long long)c->cam.nx * c->cam.ny;
    size_t esz = form == RT_FP64 ? sizeof(double) : sizeof(float);
    size_t ncomp = form == RT_UNPOL ? 1 : 4;
    const void *d_img = iquv;
    if (!is_device_ptr(iquv)) {
        int rv = ensure_stage(&c->d_stage, &c->stage_bytes, (size_t)npix * ncomp * esz);
        if (rv) return rv;
        CK(cudaMemcpyAsync(c->d_stage, iquv, (size_t)npix * ncomp * esz, cudaMemcpyHostToDevice, c->stream));
        d_img = c->d_stage;
    }
    double L = kG * c->cam.M_bh_g / (kC * kC);
    double pix = c->cam.fov_M * L / (c->cam.nx * c->cam.dist_cm);
    launch_image_sums(d_img, form == RT_FP64 ? 0 : (form == RT_UNPOL ? 2 : 1), npix, pix * pix, c->d_stats, c->stream);
    CK(cudaGetLastError());
    double h[8];
    CK(cudaMemcpyAsync(h, c->d_stats, 7 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (flux_jy) *flux_jy = h[4];
    if (lp_frac) *lp_frac = h[5];
    if (cp_frac) *cp_frac = h[6];
    return RT_OK;
}

int rt_kappa_coeffs(rt_ctx *c, const double *in, long long n, double *out) {
    if (!c || !in || !out || n < 0) return RT_ERR_INVALID;
    if (n == 0) return RT_OK;
    CK(cudaSetDevice(c->device));
    const double *d_in = in;
    double *d_out = out;
    void *tmp = nullptr;
    bool in_dev = is_device_ptr(in), out_dev = is_device_ptr(out);
    cudaError_t e = cudaSuccess;
    if (!in_dev || !out_dev) {
        if (cudaMalloc(&tmp, (size_t)n * 14 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return RT_ERR_NOMEM;
        }
        if (!in_dev) {
            d_in = (const double *)tmp;
            e = cudaMemcpyAsync((void *)d_in, in, (size_t)n * 6 * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        }
        if (!out_dev) d_out = (double *)tmp + 6 * n;
    }
    if (e == cudaSuccess) {
        KappaTables T{c->d_syn, c->d_gl, c->d_gl + 8};
        launch_kappa_quad(T, d_in, d_out, n, c->nsm * 8, c->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !out_dev)
        e = cudaMemcpyAsync(out, d_out, (size_t)n * 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    return RT_OK;
}

int rt_set_grid_fetch(rt_ctx *c, int mode) {
    if (!c || mode < RT_FETCH_AUTO || mode > RT_FETCH_STAGED) return RT_ERR_INVALID;
    c->fetch = mode;
    return RT_OK;
}

int rt_get_grid_fetch(rt_ctx *c, int *mode) {
    if (!c || !mode) return RT_ERR_INVALID;
    *mode = c->fetch;
    return RT_OK;
}

int rt_set_render_config(rt_ctx *c, const rt_render_config *cfg) {
    if (!c || !cfg) return RT_ERR_INVALID;
    if (cfg->geo_blocks_per_sm < 0 || cfg->geo_blocks_per_sm > c->geo_bps) return RT_ERR_INVALID;
    if (cfg->xfer_blocks_per_sm < 0 || cfg->xfer_blocks_per_sm > std::max(c->mixed_bps, c->fp64_bps))
        return RT_ERR_INVALID;
    if (cfg->chunks < 0 || cfg->chunks > rt_ctx::kMaxChunks) return RT_ERR_INVALID;
    if (cfg->last_chunk_div < 0 || cfg->last_chunk_div > 16) return RT_ERR_INVALID;
    c->rcfg = *cfg;
    return RT_OK;
}

int rt_get_render_config(rt_ctx *c, rt_render_config *cfg) {
    if (!c || !cfg) return RT_ERR_INVALID;
    *cfg = c->rcfg;
    return RT_OK;
}

int rt_last_counters(rt_ctx *c, rt_counters *out) {
    if (!c || !out) return RT_ERR_INVALID;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    const Counters &k = *c->h_ctr;
    memset(out, 0, sizeof(*out));
    out->rays = (uint64_t)c->last_rays;
    out->steps = k.steps;
    out->points = k.points;
    out->emitting_points = k.emitting;
    out->arena_blocks_used = k.arena_next;
    out->arena_blocks_total = (uint64_t)c->last_blocks_total;
    out->n_horizon = k.n_status[kHorizon];
    out->n_escape = k.n_status[kEscape];
    out->n_nmax = k.n_status[kNmax];
    out->n_nan = k.n_status[kNan];
    out->n_overflow = k.n_status[kOverflow];
    float ms = 0.f;
    if (c->last_was_batch) {
        out->ms_total = c->last_ms_total;
    } else {
        out->chunks = (uint32_t)c->last_chunks;
        out->shape = (uint32_t)c->last_shape;
        out->geodesic_launches = (uint32_t)c->last_geo_launches;
        out->transfer_launches = (uint32_t)c->last_xf_launches;
        if (c->last_was_overlap) {
            out->ms_geodesic = c->last_ms_geo;
            out->ms_transfer = c->last_ms_xfer;
        } else {
            if (cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) == cudaSuccess) out->ms_geodesic = ms;
            if (cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]) == cudaSuccess) out->ms_transfer = ms;
        }
        if (cudaEventElapsedTime(&ms, c->ev[0], c->ev[2]) == cudaSuccess) out->ms_total = ms;
    }
    cudaGetLastError();
    return RT_OK;
}

int rt_last_timeline(rt_ctx *c, float *out, int cap, int *n) {
    if (!c || !n || cap < 0 || (cap > 0 && !out)) return RT_ERR_INVALID;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    const int K = c->last_was_overlap ? c->last_chunks : 0;
    cudaEvent_t *gs = c->oev, *ge = c->oev + rt_ctx::kMaxChunks, *ts = c->oev + 2 * rt_ctx::kMaxChunks,
                *te = c->oev + 3 * rt_ctx::kMaxChunks;
    const int per_piece = c->last_was_streamed ? std::max(1, K / std::max(1, c->last_pieces)) : 1;
    for (int k = 0; k < std::min(K, cap); k++) {
        // the streamed shape has one geodesic launch per piece for all its chunks
        const int g = c->last_was_streamed ? k / per_piece : k;
        cudaEvent_t ev[4] = {gs[g], ge[g], ts[k], te[k]};
        for (int j = 0; j < 4; j++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, gs[0], ev[j]) != cudaSuccess) ms = 0.f;
            out[4 * k + j] = ms;
        }
    }
    cudaGetLastError();
    *n = K;
    return RT_OK;
}

}  // extern "C"
