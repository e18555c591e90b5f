// Measured FP64 FMA throughput of the device: the denominator of the geodesic's roofline
// fraction beside the nominal 2 DFMA per clock per SM. A measurement helper of this library
// (the paper has no counterpart).
#include <cuda_runtime.h>

#include "polrt.h"

namespace {

constexpr int kChains = 8, kIters = 2048;

// kChains independent FMA chains per thread (enough in flight to keep the FP64 pipe busy);
// the result is stored so that nothing is optimised away.
__global__ void dfma_chains_kernel(double *out, double seed) {
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = seed + threadIdx.x * 1e-3 + j;
    for (int i = 0; i < kIters; i++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) a[j] = fma(a[j], 0.999999, 1e-7);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; j++) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

int rt_fp64_fma_peak(int device, double *tflops) {
    if (!tflops) return RT_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_CUDA;
    }
    const int threads = 256, blocks = nsm * 8, reps = 5;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rv = RT_OK;
    if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rv = RT_ERR_CUDA;
    } else {
        dfma_chains_kernel<<<blocks, threads>>>(out, 1.0);  // warm-up
        cudaEventRecord(e0);
        for (int r = 0; r < reps; r++) dfma_chains_kernel<<<blocks, threads>>>(out, 1.0 + r);
        cudaEventRecord(e1);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
            rv = RT_ERR_CUDA;
        else
            *tflops = 2.0 * reps * (double)blocks * threads * kIters * kChains / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaGetLastError();
    return rv;
}

}  // extern "C"
