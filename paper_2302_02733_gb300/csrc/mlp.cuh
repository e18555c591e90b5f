// The coefficient surrogate: a 4 -> 64 -> 64 -> 64 -> 8 multilayer perceptron with SiLU hidden
// units, evaluated and trained on the tensor cores (BF16 operands, FP32 accumulation in TMEM).
//
// Parameters (FP32 master copy, one vector): per layer L a matrix [out][in + 1] whose last
// column is the bias, layers (4 -> 64), (64 -> 64), (64 -> 64), (64 -> 8): 9160 floats.
// The bias multiplies a constant-1 input column, so a layer is one matrix product and the
// bias gradient comes out of the weight-gradient product.
//
// Tensor-core images (BF16, canonical K-major tiles, see tc.cuh), built from the master copy:
//   W1 [64 x 16]  (inputs 0-3, the 1 column at 4), W2, W3 [64 x 80] (units 0-63, the 1 at 64),
//   W4 [16 x 80]  (outputs 0-7, rows 8-15 zero): the B operands of the forward products;
//   T2, T3 [80 x 64], T4 [80 x 16]: their transposes, the B operands of the backward products.
#pragma once
#include "tc.cuh"

namespace prt {

constexpr int kMlpIn = 4, kMlpHid = 64, kMlpOut = 8;
constexpr int kMlpParams = 64 * 5 + 64 * 65 + 64 * 65 + 8 * 65;  // 9160
constexpr int kMlpOff1 = 0, kMlpOff2 = 64 * 5, kMlpOff3 = kMlpOff2 + 64 * 65, kMlpOff4 = kMlpOff3 + 64 * 65;

// byte sizes and offsets of the packed images
constexpr int kPkW1 = 0, kPkW2 = kPkW1 + 64 * 16 * 2, kPkW3 = kPkW2 + 64 * 80 * 2, kPkW4 = kPkW3 + 64 * 80 * 2;
constexpr int kPkWBytes = kPkW4 + 16 * 80 * 2;  // 25088
constexpr int kPkT2 = 0, kPkT3 = kPkT2 + 80 * 64 * 2, kPkT4 = kPkT3 + 80 * 64 * 2;
constexpr int kPkTBytes = kPkT4 + 80 * 16 * 2;  // 23040

// SiLU z sigma(z) with sigma(z) = (1 + tanh(z / 2)) / 2 from the PTX tanh.approx.f32 (one
// special-function instruction, relative error about 2^-11, below the BF16 rounding of the
// activations that follows); training and inference share it.
__device__ __forceinline__ float sigmoid_fast(float z) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
    return fmaf(0.5f, t, 0.5f);
}
__device__ __forceinline__ float silu(float z) { return z * sigmoid_fast(z); }
__device__ __forceinline__ float silu_grad(float z) {
    float s = sigmoid_fast(z);
    return s * (1.0f + z * (1.0f - s));
}

// Store row r of a canonical K-major BF16 tile with K columns from v[0..K) (K multiple of 8).
template <int K>
__device__ __forceinline__ void store_row(unsigned char *tile, int r, const float *v) {
#pragma unroll
    for (int j = 0; j < K / 8; j++) {
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v[8 * j + 0], v[8 * j + 1]);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(v[8 * j + 2], v[8 * j + 3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(v[8 * j + 4], v[8 * j + 5]);
        __nv_bfloat162 p3 = __floats2bfloat162_rn(v[8 * j + 6], v[8 * j + 7]);
        uint4 u;
        u.x = *reinterpret_cast<uint32_t *>(&p0);
        u.y = *reinterpret_cast<uint32_t *>(&p1);
        u.z = *reinterpret_cast<uint32_t *>(&p2);
        u.w = *reinterpret_cast<uint32_t *>(&p3);
        *reinterpret_cast<uint4 *>(tile + kmaj_off(r, 8 * j, K)) = u;
    }
}

}  // namespace prt
