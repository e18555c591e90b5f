// Mixed form of the transfer kernel: the FP64 geodesic path is read back, and the plasma
// fetch, coefficients and transfer run in float.
#include <algorithm>

#include "transfer_kernel.cuh"

namespace prt {
void launch_transfer_mixed(const XferArgs &a, int coef, int grid, cudaStream_t s) {
    switch (coef) {
        case 0:
            if (a.jobs)
                transfer_kernel<float, float, 0, true><<<grid, kXferThreads, 0, s>>>(a);
            else
                transfer_kernel<float, float, 0><<<grid, kXferThreads, 0, s>>>(a);
            break;
        case 1: transfer_kernel<float, float, 1><<<grid, kXferThreads, 0, s>>>(a); break;
        case 2: transfer_kernel<float, float, 2><<<grid, kXferThreads, 0, s>>>(a); break;
        default: break;
    }
}
void launch_transfer_staged(const XferArgs &a, const CUtensorMap &map, int grid, cudaStream_t s) {
    transfer_kernel_staged<0><<<grid, kXferThreads, 0, s>>>(a, map);
}
int transfer_blocks_per_sm_staged() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transfer_kernel_staged<0>, kXferThreads, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}
void launch_unpol(const XferArgs &a, int grid, cudaStream_t s) {
    if (a.jobs)
        unpol_kernel<float, true><<<grid, kXferThreads, 0, s>>>(a);
    else
        unpol_kernel<float><<<grid, kXferThreads, 0, s>>>(a);
}
void launch_sur_features(const XferArgs &a, int grid, cudaStream_t s) {
    sur_features_pass<float><<<grid, kXferThreads, 0, s>>>(a);
}
static int func_regs(const void *f) {
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, f) != cudaSuccess) {
        cudaGetLastError();
        return 255;
    }
    return a.numRegs;
}
int transfer_regs_mixed() {
    int r = func_regs((const void *)transfer_kernel<float, float, 0>);
    r = std::max(r, func_regs((const void *)transfer_kernel<float, float, 0, true>));
    r = std::max(r, func_regs((const void *)transfer_kernel_staged<0>));
    r = std::max(r, func_regs((const void *)unpol_kernel<float>));
    return std::max(r, func_regs((const void *)unpol_kernel<float, true>));
}
int transfer_blocks_per_sm_mixed() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transfer_kernel<float, float>, kXferThreads, 0) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}
}  // namespace prt
