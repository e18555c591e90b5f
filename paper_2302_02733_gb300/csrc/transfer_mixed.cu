// Mixed form of the transfer kernel: the FP64 geodesic path is read back, and the plasma
// fetch, coefficients and transfer run in float.
#include "transfer_kernel.cuh"

namespace prt {
void launch_transfer_mixed(const XferArgs &a, int grid, cudaStream_t s) {
    transfer_kernel<float, float><<<grid, kXferThreads, 0, s>>>(a);
}
int transfer_blocks_per_sm_mixed() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transfer_kernel<float, float>, kXferThreads, 0) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}
}  // namespace prt
