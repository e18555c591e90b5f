// Batched form, FP64 transfer, and the pool set-up kernel.
#include "pipe.cuh"

namespace prt {

__global__ void pool_init_kernel(Pool P, PipeCounters *c) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.nblocks) P.ring[i] = (int)i;
    if (i == 0) {
        c->pool_head = 0;
        c->pool_tail = (unsigned long long)P.nblocks;
    }
}

void launch_pool_init(const Pool &p, PipeCounters *c, cudaStream_t s) {
    pool_init_kernel<<<(unsigned)((p.nblocks + 255) / 256), 256, 0, s>>>(p, c);
}

void launch_pipe_fp64(const PipeArgs &a, int grid, cudaStream_t s) {
    pipe_kernel<double, double><<<grid, kPipeThreads, 0, s>>>(a);
}

int pipe_blocks_per_sm_fp64() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pipe_kernel<double, double>, kPipeThreads, 0) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}

}  // namespace prt
