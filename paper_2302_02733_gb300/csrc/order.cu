// Longest-first ray order. A persistent kernel's launch ends when its slowest lanes finish
// their last rays; if those rays are long (the photon ring), the SMs idle meanwhile. The step
// counts of a previous render of the same camera (geodesics depend on the camera only) give
// the order: a counting sort by step count, descending, dealt to the chunks in rounds
// (ChunkLayout) so that every chunk holds the same mix of lengths, longest first. The image does not depend on
// the order: every ray takes the same arithmetic.
#include <algorithm>

#include "rt_kernels.cuh"

namespace prt {

// bucket 0 holds the longest rays: 16 steps per bucket, 16368 or more steps share bucket 0
__device__ __forceinline__ int order_bucket(uint16_t steps) {
    return kOrderBuckets - 1 - min((int)(steps >> 4), kOrderBuckets - 1);
}

__global__ void order_hist_kernel(const uint16_t *steps, long long n, unsigned *hist) {
    __shared__ unsigned h[kOrderBuckets];
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        atomicAdd(&h[order_bucket(steps[p])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// exclusive prefix sum of the bucket counts, in place (one thread: 1024 additions)
__global__ void order_scan_kernel(unsigned *hist) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned run = 0;
    for (int i = 0; i < kOrderBuckets; i++) {
        unsigned v = hist[i];
        hist[i] = run;
        run += v;
    }
}

// rank s (unique within the sort) -> its place in the chunk layout
__global__ void order_scatter_kernel(const uint16_t *steps, ChunkLayout L, unsigned *offs, int *order) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L.n;
         p += (long long)gridDim.x * blockDim.x) {
        long long s = atomicAdd(&offs[order_bucket(steps[p])], 1u);
        order[L.place(s)] = (int)p;
    }
}

// The probe of a new camera: the pixel at the centre of each S x S block (clipped to the image).
__device__ __forceinline__ int probe_pixel(int bx, int by, int nx, int ny, int S) {
    return min(S * by + S / 2, ny - 1) * nx + min(S * bx + S / 2, nx - 1);
}

__global__ void probe_list_kernel(int *list, int nx, int ny, int S) {
    const int px = (nx + S - 1) / S, py = (ny + S - 1) / S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)px * py;
         i += (long long)gridDim.x * blockDim.x)
        list[i] = probe_pixel((int)(i % px), (int)(i / px), nx, ny, S);
}

// every other pixel takes the step count of its block's probe (which keeps its own)
__global__ void steps_fill_kernel(uint16_t *steps, int nx, int ny, int S) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < (long long)nx * ny;
         p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % nx), y = (int)(p / nx);
        const int q = probe_pixel(x / S, y / S, nx, ny, S);
        if (q != p) steps[p] = steps[q];
    }
}

void launch_probe_list(int *list, int nx, int ny, int S, cudaStream_t s) {
    long long n = (long long)((nx + S - 1) / S) * ((ny + S - 1) / S);
    probe_list_kernel<<<(int)std::min<long long>((n + 255) / 256, 1024), 256, 0, s>>>(list, nx, ny, S);
}

void launch_steps_fill(uint16_t *steps, int nx, int ny, int S, cudaStream_t s) {
    long long n = (long long)nx * ny;
    steps_fill_kernel<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(steps, nx, ny, S);
}

void launch_order_build(const uint16_t *steps, const ChunkLayout &L, unsigned *hist, int *order, cudaStream_t s) {
    int grid = (int)std::min<long long>((L.n + 255) / 256, 1024);
    cudaMemsetAsync(hist, 0, kOrderBuckets * sizeof(unsigned), s);
    order_hist_kernel<<<grid, 256, 0, s>>>(steps, L.n, hist);
    order_scan_kernel<<<1, 32, 0, s>>>(hist);
    order_scatter_kernel<<<grid, 256, 0, s>>>(steps, L, hist, order);
}

}  // namespace prt
