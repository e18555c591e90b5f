// Kernel argument blocks and launchers shared by the host API and the kernels.
#pragma once
#include "rt_common.cuh"

namespace prt {

constexpr int kGeoThreads = 128;
constexpr int kXferThreads = 128;

struct GeoArgs {
    Camera cam;
    const double *sctab;  // (theta, sin, cos) table of the FP64 geodesic, 2048 entries
    Arena arena;
    RayRecord *rec;       // per ray of this chunk
    Counters *ctr;
    long long nrays;      // rays in this chunk
    long long ray_offset; // global id of the chunk's first ray
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
};

void launch_geodesic(const GeoArgs &a, int grid, cudaStream_t s);
void launch_sincos_table(double *tab, cudaStream_t s);
constexpr size_t kSinTabBytes = 2048 * 3 * sizeof(double);
void launch_transfer_fp64(const XferArgs &a, int grid, cudaStream_t s);
void launch_transfer_mixed(const XferArgs &a, int grid, cudaStream_t s);
void launch_x2_table(const GridModel &g, double *table, cudaStream_t s);
// out[7]: sum I, Q, U, V, flux [Jy], net LP, net CP
void launch_image_sums(const void *img, int form, long long npix, double domega, double *out, cudaStream_t s);
// resident blocks per SM of the persistent kernels (for grid sizing)
int geodesic_blocks_per_sm();
int transfer_blocks_per_sm_fp64();
int transfer_blocks_per_sm_mixed();

}  // namespace prt
