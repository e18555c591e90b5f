// Device-side shared definitions of the polrt CUDA library (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace prt {

// cgs constants (CODATA 2018)
constexpr double kG = 6.67430e-8;
constexpr double kC = 2.99792458e10;
constexpr double kMe = 9.1093837015e-28;
constexpr double kMp = 1.67262192369e-24;
constexpr double kQe = 4.80320471257e-10;
constexpr double kKb = 1.380649e-16;
constexpr double kH = 6.62607015e-27;
constexpr double kPi = 3.14159265358979323846;

enum RayStatus : uint8_t { kHorizon = 1, kEscape = 2, kNmax = 3, kNan = 4, kOverflow = 5 };
// Counters::n_status slot that counts lanes whose staged grid fetch's wait ran out
constexpr int kStageStatus = 7;

// One saved geodesic state: r, theta, phi, K^t, K^r, K^theta, K^phi and the step h taken
// from it (negative when that step was reflected through the polar axis). 64 bytes.
struct __align__(16) PathState {
    double r, th, ph, kt, kr, kth, kph, h;
};

// The path arena: fixed-size blocks of kBlockStates states, handed out by a bump counter.
// Each block records the block that precedes it on the same ray, so the transfer can walk
// a ray's states backward.
constexpr int kBlockStates = 32;
// Bytes of one arena block (states plus its back link), and the arena budget per ray: 20 blocks,
// 640 saved states per ray on average over a chunk (the mean is about 300).
constexpr size_t kBlockBytes = sizeof(PathState) * kBlockStates + sizeof(int);
constexpr int kBudgetBlocksPerRay = 20;

struct Camera {
    double a, r_cam, theta_o, nu_obs, fov, L_unit;
    int nx, ny;
    double eps;
    int nmax;
    double rh;             // outer horizon radius
    double r_stop;         // 1.05 rh: the horizon stop
    float f_a, f_nu_obs, f_L_unit;  // float copies for the FP32 transfer (no per-point conversion)
    // the camera frame (static observer; rows e_t, e_r, e_theta, e_phi, KS components) from
    // the host, the pixel side fov / nx [M] and 1 / r_cam: per-ray constants that would
    // otherwise be recomputed in FP64 on a lane of their own at every ray's start and end
    double e[4][4];
    double pix, inv_r_cam;
    // the same for the FP32 transfer's camera reading: spatial legs (rows e_r, e_theta, e_phi)
    float f_e[3][4];
    float f_pix, f_r_cam;
};

struct AdafModel {
    double n0, T0, beta, f_kep, ti_te, r_out, r_isco;
    // derived on the host: Theta_e and B at r = 1 (T_e = te0 / r, B = b0 r^-5/4)
    double te0, b0;
    float f_n0, f_te0, f_b0, f_f_kep, f_r_out, f_r_isco;
};

struct GridModel {
    int n1, n2, n3;
    double r_in, r_out, x1in, dx1, dx2, dx3;
    double hslope, poly_xt, poly_alpha, mks_smooth, poly_norm;
    const float4 *prims;   // [n1][n2][n3] cells of two float4: (rho,u,U1,U2),(U3,B1,B2,B3)
    const double *x2_table;  // inverse FMKS guess table [kX2TabW][kX2TabT]
    const double *x1_irc;    // 1 / r at the radial cell centres [n1]
    const float2 *x1_irc_f2; // the same as FP32 pairs (value, remainder), for the FP32 transfer
    double idx3;             // 1 / dx3
    float f_idx3_hi, f_idx3_lo;  // 1 / dx3 as an FP32 pair
    double rho_unit, b_unit, ne_unit, R_high, R_low, sigma_cut, gamma_ad;
    // float copies for the FP32 transfer (no per-point conversion); poly_alpha1 = poly_alpha + 1
    const float *x2_table_f;
    float f_r_in, f_r_out, f_x1in, f_dx1, f_dx2, f_dx3, f_hslope, f_poly_xt, f_poly_alpha, f_poly_alpha1, f_poly_norm,
        f_mks_smooth, f_b_unit, f_ne_unit, f_R_high, f_R_low, f_sigma_cut, f_gamma_ad;
};

// The constant of the transfer's precision: the double for the FP64 form, the float copy for
// the FP32 form.
template <typename R>
__host__ __device__ __forceinline__ R pick(double d, float f);
template <>
__host__ __device__ __forceinline__ double pick<double>(double d, float) {
    return d;
}
template <>
__host__ __device__ __forceinline__ float pick<float>(double, float f) {
    return f;
}
constexpr int kX2TabW = 64;     // blend weight w = exp(s (X1_in - X1)) in [0, 1]
constexpr int kX2TabT = 1024;   // theta in [0, pi]

struct Model {
    int kind;  // 1 ADAF, 2 grid
    AdafModel adaf;
    GridModel grid;
    int edf;       // 0 thermal (Maxwell-Juttner fits), 1 kappa distribution
    double kappa;  // its index (> 3)
};

// Tables of the kappa quadrature (kappa.cuh): ln F, ln G, ln H and the Gauss-Legendre rule.
struct KappaTables {
    const double *lnk;  // [3][4096]
    const double *glx;  // 8 nodes on [-1, 1]
    const double *glw;  // and weights
};

struct Counters {
    // the first four are reset before every chunk of rays
    unsigned long long geo_next, xfer_next;   // work-queue heads
    unsigned long long feat_next;             // queue of the surrogate's features pass
    unsigned long long arena_next;            // next free arena block
    unsigned long long feat_count;            // emitting points written by rt_render_features
    unsigned long long steps, points, emitting;
    unsigned int n_status[8];
    unsigned long long sur_rows;              // rows of the surrogate's compact features (streamed)
};

struct RayRecord {
    int last_block;  // arena block holding the last state, -1 if none
    int nstates;     // saved states (steps + 1); 0 if the ray has no usable path
    int status;      // RayStatus
    int pad;
};

struct Arena {
    PathState *states;   // nblocks * kBlockStates
    int *prev;           // nblocks: previous block of the same ray, -1 for the first
    long long nblocks;
};

// --------------------------------------------------------------------------------------
// Warp-aggregated pop of `want` lanes from a global queue: returns each requesting lane's
// ticket (>= limit means empty).
__device__ __forceinline__ unsigned long long warp_pop(unsigned long long *head, bool want) {
    unsigned mask = __ballot_sync(0xffffffffu, want);
    unsigned long long base = 0;
    int leader = __ffs(mask) - 1;
    int lane = threadIdx.x & 31;
    if (mask) {
        if (lane == leader) base = atomicAdd(head, (unsigned long long)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
    }
    return base + __popc(mask & ((1u << lane) - 1u));
}

// Pixel of ray `id`: rays are numbered in 8x4 tiles so that a warp's rays are neighbours.
__device__ __forceinline__ void ray_pixel(long long id, int nx, int ny, int &ix, int &iy) {
    if ((nx & 7) == 0 && (ny & 3) == 0) {
        long long tile = id >> 5;
        int l = (int)(id & 31);
        int tx = (int)(tile % (nx >> 3)), ty = (int)(tile / (nx >> 3));
        ix = tx * 8 + (l & 7);
        iy = ty * 4 + (l >> 3);
    } else {
        ix = (int)(id % nx);
        iy = (int)(id / nx);
    }
}

// Pixel of ray id: from an explicit pixel list (p = iy nx + ix) when one is given (adaptive
// rendering), else the 8x4-tiled order.
__device__ __forceinline__ void map_pixel(const int *list, long long id, int nx, int ny, int &ix, int &iy) {
    if (list) {
        int p = list[id];
        ix = p % nx;
        iy = p / nx;
    } else {
        ray_pixel(id, nx, ny, ix, iy);
    }
}

}  // namespace prt
