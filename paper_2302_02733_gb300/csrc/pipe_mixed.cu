// Batched form, FP32 transfer (the mixed form).
#include "pipe.cuh"

namespace prt {

void launch_pipe_mixed(const PipeArgs &a, int grid, cudaStream_t s) {
    pipe_kernel<float, float><<<grid, kPipeThreads, 0, s>>>(a);
}

int pipe_blocks_per_sm_mixed() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pipe_kernel<float, float>, kPipeThreads, 0) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}

}  // namespace prt
