// FP64 form of the transfer kernel: plasma, coefficients and transfer in double.
#include "transfer_kernel.cuh"

namespace prt {
void launch_transfer_fp64(const XferArgs &a, int coef, int grid, cudaStream_t s) {
    switch (coef) {
        case 0:
            if (a.jobs)
                transfer_kernel<double, double, 0, true><<<grid, kXferThreads, 0, s>>>(a);
            else
                transfer_kernel<double, double, 0><<<grid, kXferThreads, 0, s>>>(a);
            break;
        case 1: transfer_kernel<double, double, 1><<<grid, kXferThreads, 0, s>>>(a); break;
        default: break;
    }
}
int transfer_regs_fp64() {
    cudaFuncAttributes a{}, b{};
    if (cudaFuncGetAttributes(&a, (const void *)transfer_kernel<double, double, 0>) != cudaSuccess ||
        cudaFuncGetAttributes(&b, (const void *)transfer_kernel<double, double, 0, true>) != cudaSuccess) {
        cudaGetLastError();
        return 255;
    }
    return a.numRegs > b.numRegs ? a.numRegs : b.numRegs;
}
int transfer_blocks_per_sm_fp64() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transfer_kernel<double, double>, kXferThreads, 0) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}
}  // namespace prt
