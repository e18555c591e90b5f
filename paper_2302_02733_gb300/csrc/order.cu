// Longest-first ray order. A persistent kernel's launch ends when its slowest lanes finish
// their last rays; if those rays are long (the photon ring), the SMs idle meanwhile. The step
// counts of a previous render of the same camera (geodesics depend on the camera only) give
// the order: a counting sort by step count, descending, dealt round-robin to the chunks so
// that every chunk holds the same mix of lengths, longest first. The image does not depend on
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

// rank s (unique within the sort) -> chunk k = s % K, position s / K in it
__global__ void order_scatter_kernel(const uint16_t *steps, long long n, int K, unsigned *offs, int *order) {
    const long long base = n / K, extra = n % K;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        long long s = atomicAdd(&offs[order_bucket(steps[p])], 1u);
        long long k = s % K, q = s / K;
        order[k * base + min(k, extra) + q] = (int)p;
    }
}

void launch_order_build(const uint16_t *steps, long long n, int K, unsigned *hist, int *order, cudaStream_t s) {
    int grid = (int)std::min<long long>((n + 255) / 256, 1024);
    cudaMemsetAsync(hist, 0, kOrderBuckets * sizeof(unsigned), s);
    order_hist_kernel<<<grid, 256, 0, s>>>(steps, n, hist);
    order_scan_kernel<<<1, 32, 0, s>>>(hist);
    order_scatter_kernel<<<grid, 256, 0, s>>>(steps, n, K, hist, order);
}

}  // namespace prt
