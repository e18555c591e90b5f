// Adaptive ray tracing (the paper's outlook: trace rays densely only near image features).
//
// The image is traced on a lattice of every s-th pixel (s = base_step, a power of two; the
// last row and column included). Then, level by level, each block of side s between traced
// corners is either refined or filled:
//  - its centre is traced first, and the block is refined when a Stokes parameter at the
//    centre differs from the corners' bilinear prediction by more than tol times the
//    lattice's largest intensity, or when the corner and centre rays ended differently (say,
//    one in the hole and one escaping). Its edge midpoints then join the next list of rays,
//    and its four children are examined at side s/2. (A block too thin to have a centre is
//    refined when its corners differ by more than that.)
//  - otherwise its untraced pixels are filled by bilinear interpolation of the corners.
// A pixel queued for tracing by one block is never filled by a neighbour (a traced value
// wins). The lists are rendered with the same kernels as rt_render, addressed by pixel.
#include <algorithm>
#include <vector>

#include "host_util.cuh"
#include "polrt.h"

using namespace prt;

namespace prt {
int render_pixel_list(rt_ctx *c, int form, void *out, uint8_t *status, const int *list, long long n);
}

namespace {

enum : int { kUntouched = 0, kTraced = 1, kFilled = 2 };

__device__ __forceinline__ void queue_pixel(int *state, int p, int *list, unsigned *count) {
    int old = atomicCAS(state + p, kUntouched, kTraced);
    if (old == kFilled) old = atomicCAS(state + p, kFilled, kTraced);
    if (old != kTraced) list[atomicAdd(count, 1u)] = p;
}

__global__ void lattice_kernel(int nx, int ny, int s, int *state, int *list, unsigned *count) {
    long long n = (long long)nx * ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int i = (int)(q % nx), j = (int)(q / nx);
        bool on = (i % s == 0 || i == nx - 1) && (j % s == 0 || j == ny - 1);
        if (on) queue_pixel(state, (int)q, list, count);
    }
}

// largest intensity among the traced pixels, as ordered integer bits of a non-negative float
template <typename T>
__global__ void imax_kernel(const T *img, int nc, const int *state, long long n, unsigned long long *mx) {
    double m = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        if (state[q] == kTraced) m = fmax(m, (double)img[nc * q]);
    atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

struct Block {
    int i0, j0, i1, j1, im, jm;  // corners and midlines (-1 when the block has none)
};

__device__ __forceinline__ Block block_at(long long b, int nbx, int s, int nx, int ny) {
    Block k;
    int bi = (int)(b % nbx), bj = (int)(b / nbx), h = s / 2;
    k.i0 = bi * s;
    k.j0 = bj * s;
    k.i1 = min(k.i0 + s, nx - 1);
    k.j1 = min(k.j0 + s, ny - 1);
    k.im = k.i0 + h < k.i1 ? k.i0 + h : -1;
    k.jm = k.j0 + h < k.j1 ? k.j0 + h : -1;
    return k;
}

// Pass 1 of a level: the centres of the active blocks join the list of rays.
__global__ void centre_kernel(int nx, int ny, int s, int nbx, int nby, const int *active, int *state, int *list,
                              unsigned *count) {
    long long nb = (long long)nbx * nby;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
        if (!active[b]) continue;
        Block k = block_at(b, nbx, s, nx, ny);
        if (k.im >= 0 && k.jm >= 0) queue_pixel(state, k.jm * nx + k.im, list, count);
    }
}

// Pass 2 of a level: refine (edge midpoints, children) or fill each active block.
template <typename T>
__global__ void decide_kernel(T *img, int nc, const uint8_t *st, int nx, int ny, int s, int nbx, int nby,
                              const int *active, int *next_active, int nbx2, int *state, int *list,
                              unsigned *count, const unsigned long long *imax_bits, double tol) {
    long long nb = (long long)nbx * nby;
    double thr = tol * __longlong_as_double((long long)*imax_bits);
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
        if (!active[b]) continue;
        Block k = block_at(b, nbx, s, nx, ny);
        int bi = (int)(b % nbx), bj = (int)(b / nbx), h = s / 2;
        // pixel indices fit an int; times nc they need not
        long long c00 = k.j0 * nx + k.i0, c10 = k.j0 * nx + k.i1, c01 = k.j1 * nx + k.i0, c11 = k.j1 * nx + k.i1;
        bool centre = k.im >= 0 && k.jm >= 0;
        long long cc = centre ? k.jm * nx + k.im : c00;
        bool refine = st && (st[c00] != st[c10] || st[c00] != st[c01] || st[c00] != st[c11] || st[c00] != st[cc]);
        for (int q = 0; q < nc && !refine; q++) {
            double a = img[nc * c00 + q], bb = img[nc * c10 + q], c = img[nc * c01 + q], d = img[nc * c11 + q];
            if (centre) {
                double fx = (double)(k.im - k.i0) / (k.i1 - k.i0), fy = (double)(k.jm - k.j0) / (k.j1 - k.j0);
                double pred = (1 - fx) * (1 - fy) * a + fx * (1 - fy) * bb + (1 - fx) * fy * c + fx * fy * d;
                refine = fabs((double)img[nc * cc + q] - pred) > thr;
            } else {
                refine = fmax(fmax(a, bb), fmax(c, d)) - fmin(fmin(a, bb), fmin(c, d)) > thr;
            }
        }
        if (refine) {
            if (k.im >= 0) {
                queue_pixel(state, k.j0 * nx + k.im, list, count);
                queue_pixel(state, k.j1 * nx + k.im, list, count);
            }
            if (k.jm >= 0) {
                queue_pixel(state, k.jm * nx + k.i0, list, count);
                queue_pixel(state, k.jm * nx + k.i1, list, count);
            }
            if (next_active)  // children at side h (non-degenerate ones); none below side 2
                for (int dj = 0; dj < 2; dj++)
                    for (int di = 0; di < 2; di++) {
                        int ci = 2 * bi + di, cj = 2 * bj + dj;
                        if (ci * h < k.i1 && cj * h < k.j1 && ci * h < nx - 1 && cj * h < ny - 1)
                            next_active[(long long)cj * nbx2 + ci] = 1;
                    }
        } else {
            for (int j = k.j0; j <= k.j1; j++)
                for (int i = k.i0; i <= k.i1; i++) {
                    long long p = j * nx + i;
                    if (atomicCAS(state + p, kUntouched, kFilled) != kUntouched) continue;
                    double fx = (double)(i - k.i0) / (k.i1 - k.i0), fy = (double)(j - k.j0) / (k.j1 - k.j0);
                    for (int q = 0; q < nc; q++) {
                        double v = (1 - fx) * (1 - fy) * img[nc * c00 + q] + fx * (1 - fy) * img[nc * c10 + q] +
                                   (1 - fx) * fy * img[nc * c01 + q] + fx * fy * img[nc * c11 + q];
                        img[nc * p + q] = (T)v;
                    }
                }
        }
    }
}

int blocks_at(int n, int s) { return (n - 1 + s - 1) / s; }  // blocks of side s over n pixels

}  // namespace

extern "C" {

int rt_render_adaptive(rt_ctx *c, int form, void *out, uint8_t *status, int base_step, double tol,
                       long long *rays_traced) {
    if (!c || !out || (form != RT_FP64 && form != RT_MIXED && form != RT_UNPOL)) return RT_ERR_INVALID;
    if (base_step < 2 || (base_step & (base_step - 1)) || !(tol >= 0.0)) return RT_ERR_INVALID;
    if (!c->have_cam || !c->have_model) return RT_ERR_NOT_READY;
    if (!is_device_ptr(out) || (status && !is_device_ptr(status))) return RT_ERR_INVALID;
    if (cudaSetDevice(c->device) != cudaSuccess) return RT_ERR_CUDA;
    const int nx = c->cam.nx, ny = c->cam.ny;
    if (nx < 2 || ny < 2) return RT_ERR_INVALID;
    const long long npix = (long long)nx * ny;
    const int nc = form == RT_UNPOL ? 1 : 4;
    // buffers: state, list, status (if not given), two activity maps, counters
    const int nbx_f = blocks_at(nx, 2), nby_f = blocks_at(ny, 2);
    size_t act_n = (size_t)(nbx_f + 1) * (nby_f + 1);
    size_t bytes = npix * 2 * sizeof(int) + (status ? 0 : npix) + 2 * act_n * sizeof(int) + 64;
    char *buf = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    int *state = (int *)buf, *list = state + npix;
    int *act[2] = {list + npix, list + npix + act_n};
    uint8_t *own_st = (uint8_t *)(act[1] + act_n);  // status, when the caller gives none
    uint8_t *st = status ? status : own_st;
    // the counters always live in this buffer, after the own status area (reserved or not)
    unsigned long long *scal = (unsigned long long *)(((uintptr_t)(own_st + (status ? 0 : npix)) + 15) & ~(uintptr_t)15);
    unsigned *count = (unsigned *)scal;
    unsigned long long *imax = scal + 1;
    int rv = RT_OK;
    int overflow = RT_OK;  // RT_ERR_WORKSPACE once a level's rays overflowed the arena
    long long traced = 0;
    cudaStream_t s = c->stream;
    int grid = c->nsm * 4;
    auto step = [&](auto dummy) -> int {
        using T = decltype(dummy);
        T *img = (T *)out;
        if (cudaMemsetAsync(state, 0, npix * sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(scal, 0, 16, s) != cudaSuccess)
            return RT_ERR_CUDA;
        lattice_kernel<<<grid, 256, 0, s>>>(nx, ny, base_step, state, list, count);
        unsigned n = 0;
        if (cudaMemcpyAsync(&n, count, sizeof(n), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return RT_ERR_CUDA;
        int r = render_pixel_list(c, form, out, st, list, n);
        if (r != RT_OK && r != RT_ERR_WORKSPACE) return r;
        if (r) overflow = r;
        traced += n;
        imax_kernel<T><<<grid, 256, 0, s>>>(img, nc, state, npix, imax);
        // every lattice block starts active
        int nbx = blocks_at(nx, base_step), nby = blocks_at(ny, base_step);
        std::vector<int> ones((size_t)nbx * nby, 1);
        if (cudaMemcpyAsync(act[0], ones.data(), ones.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return RT_ERR_CUDA;
        int cur = 0;
        for (int side = base_step; side >= 2; side /= 2) {
            nbx = blocks_at(nx, side);
            nby = blocks_at(ny, side);
            // the next level's activity map (blocks of side side/2, the last level has none)
            const bool deeper = side / 2 >= 2;
            int nbx2 = deeper ? blocks_at(nx, side / 2) : 0, nby2 = deeper ? blocks_at(ny, side / 2) : 0;
            if ((deeper && cudaMemsetAsync(act[1 - cur], 0, (size_t)nbx2 * nby2 * sizeof(int), s) != cudaSuccess) ||
                cudaMemsetAsync(count, 0, sizeof(unsigned), s) != cudaSuccess)
                return RT_ERR_CUDA;
            centre_kernel<<<grid, 128, 0, s>>>(nx, ny, side, nbx, nby, act[cur], state, list, count);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(&n, count, sizeof(n), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return RT_ERR_CUDA;
            if (n > 0) {
                r = render_pixel_list(c, form, out, st, list, n);
                if (r != RT_OK && r != RT_ERR_WORKSPACE) return r;
                if (r) overflow = r;
                traced += n;
            }
            if (cudaMemsetAsync(count, 0, sizeof(unsigned), s) != cudaSuccess) return RT_ERR_CUDA;
            decide_kernel<T><<<grid, 128, 0, s>>>(img, nc, st, nx, ny, side, nbx, nby, act[cur],
                                                  deeper ? act[1 - cur] : nullptr, nbx2, state, list, count, imax,
                                                  tol);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(&n, count, sizeof(n), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return RT_ERR_CUDA;
            if (n > 0) {
                r = render_pixel_list(c, form, out, st, list, n);
                if (r != RT_OK && r != RT_ERR_WORKSPACE) return r;
                if (r) overflow = r;
                traced += n;
            }
            cur = 1 - cur;
        }
        return RT_OK;
    };
    rv = form == RT_FP64 ? step(0.0) : step(0.0f);
    if (rv == RT_OK) rv = overflow;  // the refinement went on; the overflowed rays are marked
    cudaFree(buf);
    cudaGetLastError();
    if (rays_traced) *rays_traced = traced;
    c->last_rays = traced;
    return rv;
}

}  // extern "C"
