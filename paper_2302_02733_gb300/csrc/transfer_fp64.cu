// FP64 form of the transfer kernel: plasma, coefficients and transfer in double.
#include "transfer_kernel.cuh"

namespace prt {
void launch_transfer_fp64(const XferArgs &a, int grid, cudaStream_t s) {
    transfer_kernel<double, double><<<grid, kXferThreads, 0, s>>>(a);
}
int transfer_blocks_per_sm_fp64() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transfer_kernel<double, double>, kXferThreads, 0) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}
}  // namespace prt
