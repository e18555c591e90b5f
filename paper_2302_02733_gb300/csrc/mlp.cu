// Surrogate MLP kernels: packing of the BF16 tensor-core images, inference, one training
// step's gradient (forward and backward on the tensor cores), Adam.
#include "mlp.cuh"
#include "rt_kernels.cuh"

namespace prt {

// ---- packing -------------------------------------------------------------------------------
// master index of weight (o, i) of layer L (i == in is the bias)
__device__ __forceinline__ int mlp_index(int L, int o, int i) {
    switch (L) {
        case 1: return kMlpOff1 + o * 5 + i;
        case 2: return kMlpOff2 + o * 65 + i;
        case 3: return kMlpOff3 + o * 65 + i;
        default: return kMlpOff4 + o * 65 + i;
    }
}

// value of the forward image W_L at (row o, column k): weight, bias on the 1 column, else 0
__device__ __forceinline__ float mlp_wval(const float *th, int L, int o, int k) {
    int in = L == 1 ? 4 : 64, out = L == 4 ? 8 : 64;
    if (o >= out || k > in) return 0.0f;
    return th[mlp_index(L, o, k)];
}

__global__ void mlp_pack_kernel(const float *th, unsigned char *wpk, unsigned char *tpk) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    // forward images: element e of W1 | W2 | W3 | W4 in (row, col) order
    const int n1 = 64 * 16, n2 = 64 * 80, n4 = 16 * 80;
    if (e < n1 + 2 * n2 + n4) {
        int L, r, k, K, base;
        if (e < n1) {
            L = 1, K = 16, r = e / 16, k = e % 16, base = kPkW1;
        } else if (e < n1 + n2) {
            L = 2, K = 80, r = (e - n1) / 80, k = (e - n1) % 80, base = kPkW2;
        } else if (e < n1 + 2 * n2) {
            L = 3, K = 80, r = (e - n1 - n2) / 80, k = (e - n1 - n2) % 80, base = kPkW3;
        } else {
            L = 4, K = 80, r = (e - n1 - 2 * n2) / 80, k = (e - n1 - 2 * n2) % 80, base = kPkW4;
        }
        *reinterpret_cast<__nv_bfloat16 *>(wpk + base + kmaj_off(r, k, K)) = __float2bfloat16_rn(mlp_wval(th, L, r, k));
    }
    // transposed images T_L [rows = input index k][cols = output index o]
    const int t2 = 80 * 64, t4 = 80 * 16;
    if (e < 2 * t2 + t4) {
        int L, k, o, K, base;
        if (e < t2) {
            L = 2, K = 64, k = e / 64, o = e % 64, base = kPkT2;
        } else if (e < 2 * t2) {
            L = 3, K = 64, k = (e - t2) / 64, o = (e - t2) % 64, base = kPkT3;
        } else {
            L = 4, K = 16, k = (e - 2 * t2) / 16, o = (e - 2 * t2) % 16, base = kPkT4;
        }
        *reinterpret_cast<__nv_bfloat16 *>(tpk + base + kmaj_off(k, o, K)) = __float2bfloat16_rn(mlp_wval(th, L, o, k));
    }
}

// ---- shared helpers of the tensor-core kernels --------------------------------------------
struct TcSync {
    uint32_t bar, phase;
    bool ok;
};

// all threads' shared-memory writes visible to the tensor core, TMEM reads finished
__device__ __forceinline__ void tc_barrier() {
    fence_smem_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// wait for the MMAs thread 0 committed; block-uniform success flag
__device__ __forceinline__ void tc_wait(TcSync &s) {
    bool ok = mbar_wait(s.bar, s.phase);
    s.phase ^= 1u;
    fence_after_sync();
    s.ok = __syncthreads_and(ok && s.ok) != 0;
}

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float v[64]) {
#pragma unroll
    for (int j = 0; j < 4; j++) tmem_ld16(taddr + 16 * j, v + 16 * j);
}

// ---- inference -----------------------------------------------------------------------------
constexpr int kFwdA0 = kPkWBytes, kFwdA = kFwdA0 + 128 * 16 * 2, kFwdBar = kFwdA + 128 * 80 * 2;
constexpr int kFwdSmem = kFwdBar + 16;

// y[n][8] = MLP(x[n][4]) (x already normalised), tiles of 128 rows, one row per thread. With
// used, n is capped at used[0] * used_scale rows (32 per arena block in use, or a row count), a
// count an earlier kernel on the stream wrote (so the host need not wait for it).
__global__ void __launch_bounds__(128, 1) mlp_forward_kernel(const float4 *__restrict__ x, float *__restrict__ y,
                                                             long long n, const uint4 *__restrict__ wpk,
                                                             unsigned *err, const unsigned long long *used,
                                                             int used_scale) {
    extern __shared__ __align__(128) unsigned char sm[];
    if (used) n = min(n, (long long)(*used * (unsigned long long)used_scale));
    const int r = threadIdx.x, warp = r >> 5;
    for (int i = r; i < kPkWBytes / 16; i += 128) reinterpret_cast<uint4 *>(sm)[i] = wpk[i];
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + kFwdBar + 8);
    if (warp == 0) tmem_alloc(smem_u32(slot), 128);
    if (r == 0) mbar_init(smem_u32(sm + kFwdBar), 1);
    tc_barrier();
    const uint32_t tm = *slot, lane = (uint32_t)(warp * 32) << 16;
    const uint32_t sW = smem_u32(sm), sA0 = smem_u32(sm + kFwdA0), sA = smem_u32(sm + kFwdA);
    TcSync s{smem_u32(sm + kFwdBar), 0u, true};
    float v[80];
    for (long long t0 = (long long)blockIdx.x * 128; t0 < n && s.ok; t0 += (long long)gridDim.x * 128) {
        long long row = t0 + r;
        float4 in = row < n ? x[row] : make_float4(0.f, 0.f, 0.f, 0.f);
        float a0[16] = {in.x, in.y, in.z, in.w, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        store_row<16>(sm + kFwdA0, r, a0);
        tc_barrier();
        if (r == 0) {
            tc_gemm(tm, sA0, sW + kPkW1, 64, 16, false);
            tc_commit(s.bar);
        }
        tc_wait(s);
        for (int L = 2; L <= 4 && s.ok; L++) {
            tmem_ld64(tm + lane, v);
#pragma unroll
            for (int k = 0; k < 64; k++) v[k] = silu(v[k]);
            v[64] = 1.f;
#pragma unroll
            for (int k = 65; k < 80; k++) v[k] = 0.f;
            store_row<80>(sm + kFwdA, r, v);
            tc_barrier();
            if (r == 0) {
                tc_gemm(tm, sA, sW + (L == 2 ? kPkW2 : L == 3 ? kPkW3 : kPkW4), L == 4 ? 16 : 64, 80, false);
                tc_commit(s.bar);
            }
            tc_wait(s);
        }
        float o[16];
        tmem_ld16(tm + lane, o);
        if (row < n) {
            float4 *d = reinterpret_cast<float4 *>(y + 8 * row);
            d[0] = make_float4(o[0], o[1], o[2], o[3]);
            d[1] = make_float4(o[4], o[5], o[6], o[7]);
        }
        fence_before_sync();
        __syncthreads();
    }
    if (!s.ok && r == 0) atomicOr(err, 1u);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tm, 128);
}

// ---- one training step's gradient ----------------------------------------------------------
// Shared memory: W | T | A0 | A1 | A2 | A3 | dZ [128 x <=80] | dZT [64 x 128] | AT [128 x 128]
constexpr int kTrT = kPkWBytes, kTrA0 = kTrT + kPkTBytes, kTrA1 = kTrA0 + 128 * 16 * 2;
constexpr int kTrA2 = kTrA1 + 128 * 80 * 2, kTrA3 = kTrA2 + 128 * 80 * 2, kTrDZ = kTrA3 + 128 * 80 * 2;
constexpr int kTrDZT = kTrDZ + 128 * 80 * 2, kTrAT = kTrDZT + 64 * 128 * 2, kTrBar = kTrAT + 128 * 128 * 2;
constexpr int kTrSmem = kTrBar + 32;  // mbarrier, TMEM slot, the warps' losses
// TMEM columns: pre-activations Z1-Z3, scratch S (outputs, then dA), weight-gradient images G1-G4
constexpr uint32_t kCZ1 = 0, kCZ2 = 64, kCZ3 = 128, kCS = 192, kCG1 = 288, kCG2 = 352, kCG3 = 416, kCG4 = 480;

// AT[k][r] = A[r][k] for this thread's sample r and k < K (the transpose, as a canonical
// K-major tile with 128 columns)
template <int K>
__device__ __forceinline__ void transpose_row(const unsigned char *A, unsigned char *AT, int r) {
#pragma unroll
    for (int k = 0; k < K; k++)
        *reinterpret_cast<__nv_bfloat16 *>(AT + kmaj_off(k, r, 128)) =
            *reinterpret_cast<const __nv_bfloat16 *>(A + kmaj_off(r, k, K));
}

// gpart[block] (the FP32 master layout) = d loss / d theta over this block's 128 samples, with
// loss = sum over samples and outputs of (y - t)^2 / (ntot * 8); lpart[block] = this block's
// loss. Every element is written once (no atomics), so that a fixed-order sum over the blocks
// (mlp_sum_kernel, mlp_adam_kernel) makes a training run depend only on its seed.
__global__ void __launch_bounds__(128, 1) mlp_grad_kernel(const float4 *__restrict__ x, const float *__restrict__ t,
                                                          long long n, long long ntot, const uint4 *__restrict__ wpk,
                                                          const uint4 *__restrict__ tpk, float *gpart, float *lpart,
                                                          unsigned *err) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int r = threadIdx.x, warp = r >> 5;
    for (int i = r; i < kPkWBytes / 16; i += 128) reinterpret_cast<uint4 *>(sm)[i] = wpk[i];
    for (int i = r; i < kPkTBytes / 16; i += 128) reinterpret_cast<uint4 *>(sm + kTrT)[i] = tpk[i];
    for (int i = r; i < 128 * 128 * 2 / 16; i += 128) reinterpret_cast<uint4 *>(sm + kTrAT)[i] = make_uint4(0, 0, 0, 0);
    for (int i = r; i < 64 * 128 * 2 / 16; i += 128) reinterpret_cast<uint4 *>(sm + kTrDZT)[i] = make_uint4(0, 0, 0, 0);
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + kTrBar + 8);
    if (warp == 0) tmem_alloc(smem_u32(slot), 512);
    if (r == 0) mbar_init(smem_u32(sm + kTrBar), 1);
    tc_barrier();
    const uint32_t tm = *slot, lane = (uint32_t)(warp * 32) << 16;
    const uint32_t sW = smem_u32(sm), sT = smem_u32(sm + kTrT);
    const uint32_t sA0 = smem_u32(sm + kTrA0), sA1 = smem_u32(sm + kTrA1), sA2 = smem_u32(sm + kTrA2),
                   sA3 = smem_u32(sm + kTrA3), sDZ = smem_u32(sm + kTrDZ), sDZT = smem_u32(sm + kTrDZT),
                   sAT = smem_u32(sm + kTrAT);
    TcSync s{smem_u32(sm + kTrBar), 0u, true};
    const long long row = (long long)blockIdx.x * 128 + r;
    const bool valid = row < n;
    float v[80], z[64];

    // forward: Z_L kept in TMEM, activations A_L in shared memory
    float4 in = valid ? x[row] : make_float4(0.f, 0.f, 0.f, 0.f);
    float a0[16] = {in.x, in.y, in.z, in.w, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    store_row<16>(sm + kTrA0, r, a0);
    tc_barrier();
    if (r == 0) {
        tc_gemm(tm + kCZ1, sA0, sW + kPkW1, 64, 16, false);
        tc_commit(s.bar);
    }
    tc_wait(s);
    const uint32_t zc[3] = {kCZ1, kCZ2, kCZ3};
    const int aoff[3] = {kTrA1, kTrA2, kTrA3};
    for (int L = 0; L < 3 && s.ok; L++) {
        tmem_ld64(tm + lane + zc[L], v);
#pragma unroll
        for (int k = 0; k < 64; k++) v[k] = silu(v[k]);
        v[64] = 1.f;
#pragma unroll
        for (int k = 65; k < 80; k++) v[k] = 0.f;
        store_row<80>(sm + aoff[L], r, v);
        tc_barrier();
        if (r == 0) {
            uint32_t a = smem_u32(sm + aoff[L]);
            if (L < 2)
                tc_gemm(tm + zc[L + 1], a, sW + (L == 0 ? kPkW2 : kPkW3), 64, 80, false);
            else
                tc_gemm(tm + kCS, a, sW + kPkW4, 16, 80, false);
            tc_commit(s.bar);
        }
        tc_wait(s);
    }

    // loss and dY (scaled by 2 / (ntot 8)); dY as the A operand [128 x 16] and transposed [16 x 128]
    float yo[16], dy[16];
    tmem_ld16(tm + lane + kCS, yo);
    float lsum = 0.f;
    const float sc = 2.0f / (8.0f * (float)ntot);
#pragma unroll
    for (int k = 0; k < 16; k++) {
        float d = 0.f;
        if (k < 8 && valid) {
            d = yo[k] - t[8 * row + k];
            lsum += d * d;
        }
        dy[k] = sc * d;
    }
    store_row<16>(sm + kTrDZ, r, dy);
#pragma unroll
    for (int k = 0; k < 16; k++)
        *reinterpret_cast<__nv_bfloat16 *>(sm + kTrDZT + kmaj_off(k, r, 128)) = __float2bfloat16_rn(dy[k]);
    transpose_row<80>(sm + kTrA3, sm + kTrAT, r);
    for (int o = 16; o >= 1; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    float *wl = reinterpret_cast<float *>(sm + kTrBar + 12);  // 4 floats after the TMEM slot
    if ((r & 31) == 0) wl[warp] = lsum;
    tc_barrier();
    if (r == 0) lpart[blockIdx.x] = (((wl[0] + wl[1]) + wl[2]) + wl[3]) / (8.0f * (float)ntot);
    if (r == 0 && s.ok) {
        tc_gemm(tm + kCG4, sAT, sDZT, 16, 128, false);  // dW4^T = A3^T dY
        tc_gemm(tm + kCS, sDZ, sT + kPkT4, 80, 16, false);  // dA3 = dY W4
        tc_commit(s.bar);
    }
    tc_wait(s);

    // hidden layers 3, 2, 1: dZ_L = dA_L * silu'(Z_L); dW_L^T = A_{L-1}^T dZ_L; dA_{L-1} = dZ_L W_L
    for (int L = 3; L >= 1 && s.ok; L--) {
        tmem_ld64(tm + lane + kCS, v);
        tmem_ld64(tm + lane + zc[L - 1], z);
#pragma unroll
        for (int k = 0; k < 64; k++) v[k] *= silu_grad(z[k]);
        store_row<64>(sm + kTrDZ, r, v);
#pragma unroll
        for (int k = 0; k < 64; k++)
            *reinterpret_cast<__nv_bfloat16 *>(sm + kTrDZT + kmaj_off(k, r, 128)) = __float2bfloat16_rn(v[k]);
        if (L == 1)
            transpose_row<16>(sm + kTrA0, sm + kTrAT, r);
        else
            transpose_row<80>(sm + (L == 3 ? kTrA2 : kTrA1), sm + kTrAT, r);
        tc_barrier();
        if (r == 0) {
            tc_gemm(tm + (L == 3 ? kCG3 : L == 2 ? kCG2 : kCG1), sAT, sDZT, 64, 128, false);
            if (L > 1) tc_gemm(tm + kCS, sDZ, sT + (L == 3 ? kPkT3 : kPkT2), 80, 64, false);
            tc_commit(s.bar);
        }
        tc_wait(s);
    }

    // weight gradients: TMEM lane k holds d loss / d W_L[o][k] for input index k (k == in: bias)
    float *g = gpart + (long long)blockIdx.x * kMlpParams;
    if (s.ok) {
        const uint32_t gc[4] = {kCG1, kCG2, kCG3, kCG4};
        for (int L = 1; L <= 4; L++) {
            int in = L == 1 ? 4 : 64, out = L == 4 ? 8 : 64;
            if (L < 4) {
                tmem_ld64(tm + lane + gc[L - 1], v);
            } else {
                tmem_ld16(tm + lane + gc[3], v);
            }
            if (r <= in)
                for (int o = 0; o < out; o++) g[mlp_index(L, o, r)] = v[o];
        }
    }
    if (!s.ok && r == 0) atomicOr(err, 1u);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tm, 512);
}

// ---- fixed-order sums over the blocks, Adam ---------------------------------------------------
// acc (+)= sum over blocks b = 0 .. nb-1, in that order, of gpart[b]; loss = sum of lpart
__global__ void mlp_sum_kernel(const float *gpart, const float *lpart, int nb, float *acc, float *loss, bool add) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpParams) {
        float g = add ? acc[i] : 0.f;
        for (int b = 0; b < nb; b++) g += gpart[(long long)b * kMlpParams + i];
        acc[i] = g;
    }
    if (i == 0 && loss) {
        float l = add ? *loss : 0.f;
        for (int b = 0; b < nb; b++) l += lpart[b];
        *loss = l;
    }
}

// One Adam step on the gradient summed (in block order) from gpart; loss = the summed loss.
__global__ void mlp_adam_kernel(float *th, float *m, float *v, const float *gpart, const float *lpart, int nb,
                                float *loss, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && loss) {
        float l = 0.f;
        for (int b = 0; b < nb; b++) l += lpart[b];
        *loss = l;
    }
    if (i >= n) return;
    float g = 0.f;
    for (int b = 0; b < nb; b++) g += gpart[(long long)b * kMlpParams + i];
    float mi = b1 * m[i] + (1.f - b1) * g, vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---- launchers -----------------------------------------------------------------------------
int mlp_init_attributes() {
    if (cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem) != cudaSuccess)
        return -1;
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrSmem) != cudaSuccess)
        return -1;
    return 0;
}

void launch_mlp_pack(const float *th, void *wpk, void *tpk, cudaStream_t s) {
    int n = 64 * 16 + 2 * 64 * 80 + 16 * 80;
    mlp_pack_kernel<<<(n + 255) / 256, 256, 0, s>>>(th, (unsigned char *)wpk, (unsigned char *)tpk);
}

void launch_mlp_forward(const float *x, float *y, long long n, const void *wpk, unsigned *err, int grid, cudaStream_t s,
                        const unsigned long long *used, int used_scale) {
    mlp_forward_kernel<<<grid, 128, kFwdSmem, s>>>(reinterpret_cast<const float4 *>(x), y, n,
                                                   reinterpret_cast<const uint4 *>(wpk), err, used, used_scale);
}

void launch_mlp_grad(const float *x, const float *t, long long n, long long ntot, const void *wpk, const void *tpk,
                     float *gpart, float *lpart, unsigned *err, cudaStream_t s) {
    unsigned grid = (unsigned)((n + 127) / 128);
    mlp_grad_kernel<<<grid, 128, kTrSmem, s>>>(reinterpret_cast<const float4 *>(x), t, n, ntot,
                                               reinterpret_cast<const uint4 *>(wpk),
                                               reinterpret_cast<const uint4 *>(tpk), gpart, lpart, err);
}

void launch_mlp_sum(const float *gpart, const float *lpart, int nb, float *acc, float *loss, bool add, cudaStream_t s) {
    mlp_sum_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(gpart, lpart, nb, acc, loss, add);
}

void launch_mlp_adam(float *th, float *m, float *v, const float *gpart, const float *lpart, int nb, float *loss,
                     float lr, float b1, float b2, float eps, float c1, float c2, cudaStream_t s) {
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(th, m, v, gpart, lpart, nb, loss, kMlpParams, lr, b1, b2,
                                                             eps, c1, c2);
}

}  // namespace prt
