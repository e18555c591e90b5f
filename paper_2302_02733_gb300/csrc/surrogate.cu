// Host side of the surrogate (include/polrt.h, rt_mlp_* and rt_surrogate_*): parameters and
// their tensor-core images, the training set made by the quadrature, the Adam training loop
// on the tensor-core gradient kernel, and coefficient evaluation with the quadrature as
// fallback outside the training box.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_util.cuh"
#include "mlp.cuh"
#include "polrt.h"
#include "surrogate.cuh"

using namespace prt;

namespace prt {
int mlp_init_attributes();
void launch_mlp_pack(const float *th, void *wpk, void *tpk, cudaStream_t s);
void launch_mlp_sum(const float *gpart, const float *lpart, int nb, float *acc, float *loss, bool add, cudaStream_t s);
void launch_mlp_grad(const float *x, const float *t, long long n, long long ntot, const void *wpk, const void *tpk,
                     float *grad, float *loss, unsigned *err, cudaStream_t s);
void launch_mlp_adam(float *th, float *m, float *v, const float *gpart, const float *lpart, int nb, float *loss,
                     float lr, float b1, float b2, float eps, float c1, float c2, cudaStream_t s);

__device__ __forceinline__ unsigned long long sm64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct SurBox {
    float lo[4], hi[4];
};

// Training set: features uniform in the box (splitmix64 counters), targets by quadrature with
// n_e = 1 cm^-3 and B = 1 G (the targets do not depend on either).
__global__ void sur_dataset_kernel(KappaTables T, SurBox box, unsigned long long seed, long long n, float *xn,
                                   float *y, int *valid) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        bool ok = false;
        float yy[8];
        // a point whose coefficients underflow is drawn again (a few times at most)
        for (int attempt = 0; attempt < 8 && !ok; attempt++) {
            float f[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                unsigned long long ctr = (unsigned long long)(4 * i + j) + (unsigned long long)attempt * (4ull * n);
                double u = (double)(sm64(seed ^ sm64(ctr)) >> 11) * (1.0 / 9007199254740992.0);
                f[j] = box.lo[j] + (float)u * (box.hi[j] - box.lo[j]);
                xn[4 * i + j] = 2.0f * (float)u - 1.0f;
            }
            double th = f[1], Te = exp((double)f[2]), kap = f[3], B = 1.0;
            double nuB = kQe * B / (2.0 * kPi * kMe * kC);
            double nu = exp((double)f[0]) * 1.5 * nuB * sin(th) * Te * Te;
            double c[8];
            kappa_coeffs_quad(T, 1.0, Te, B, nu, th, kap, c);
            SurPref p = sur_prefactors(1.0, Te, B, nu, th);
            ok = sur_reduce(p, c, yy);
        }
        valid[i] = ok ? 1 : 0;
#pragma unroll
        for (int k = 0; k < 8; k++) y[8 * i + k] = yy[k];
    }
}

// Points -> normalised features (and whether they fall inside the box).
__global__ void sur_features_kernel(const double *in, long long n, SurBox box, float *xn, unsigned char *inside) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double *v = in + 6 * i;
        float f[4];
        sur_features(v[1], v[2], v[3], v[4], v[5], f);
        bool ok = v[0] > 0.0 && v[1] > 0.0 && v[2] > 0.0 && v[3] > 0.0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float u = (f[j] - box.lo[j]) / (box.hi[j] - box.lo[j]);
            ok &= u >= 0.0f && u <= 1.0f;
            xn[4 * i + j] = 2.0f * u - 1.0f;
        }
        inside[i] = ok ? 1 : 0;
    }
}

// network outputs -> coefficients; outside the box the quadrature answers instead
// norm: 8 means, 8 standard deviations, 8 x 35 baseline coefficients
__global__ void sur_expand_kernel(KappaTables T, const double *in, long long n, const float *xn, const float *yhat,
                                  const float *norm, const unsigned char *inside, double *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double *v = in + 6 * i;
        double c[8];
        if (inside[i]) {
            float phi[kSurBasis], y[8];
            float x4[4] = {xn[4 * i], xn[4 * i + 1], xn[4 * i + 2], xn[4 * i + 3]};
            sur_basis(x4, phi);
#pragma unroll
            for (int k = 0; k < 8; k++) {
                float b = 0.f;
                for (int m = 0; m < kSurBasis; m++) b += norm[16 + k * kSurBasis + m] * phi[m];
                y[k] = b + norm[k] + norm[8 + k] * yhat[8 * i + k];
            }
            SurPref p = sur_prefactors(v[0], v[1], v[2], v[3], v[4]);
            sur_expand(p, y, c);
        } else {
            kappa_coeffs_quad(T, v[0], v[1], v[2], v[3], v[4], v[5], c);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) out[8 * i + k] = c[k];
    }
}

// Normal equations of the baseline fit: acc[0..1225) += phi phi^T, acc[1225..1505) += phi y^T,
// acc[1505] += rows (valid rows only). 512 threads, 64 rows staged per pass.
__global__ void __launch_bounds__(512) sur_normal_kernel(const float *x, const float *y, const int *valid, long long n,
                                                          double *acc) {
    __shared__ float ph[64][kSurBasis + 1];
    __shared__ float yy[64][8];
    double part[3] = {0.0, 0.0, 0.0};
    double rows = 0.0;
    const int tid = threadIdx.x;
    for (long long r0 = blockIdx.x * 64ll; r0 < n; r0 += (long long)gridDim.x * 64ll) {
        if (tid < 64) {
            long long r = r0 + tid;
            bool ok = r < n && valid[r];
            float x4[4] = {0.f, 0.f, 0.f, 0.f}, phi[kSurBasis];
            if (ok)
                for (int j = 0; j < 4; j++) x4[j] = x[4 * r + j];
            sur_basis(x4, phi);
            for (int m = 0; m < kSurBasis; m++) ph[tid][m] = ok ? phi[m] : 0.f;
            for (int k = 0; k < 8; k++) yy[tid][k] = ok ? y[8 * r + k] : 0.f;
            rows += ok ? 1.0 : 0.0;
        }
        __syncthreads();
        for (int e = 0; e < 3; e++) {
            int idx = tid + 512 * e;
            if (idx < 1225) {
                int i = idx / kSurBasis, j = idx % kSurBasis;
                double s = 0.0;
                for (int q = 0; q < 64; q++) s += (double)ph[q][i] * ph[q][j];
                part[e] += s;
            } else if (idx < 1505) {
                int i = (idx - 1225) / 8, k = (idx - 1225) % 8;
                double s = 0.0;
                for (int q = 0; q < 64; q++) s += (double)ph[q][i] * yy[q][k];
                part[e] += s;
            }
        }
        __syncthreads();
    }
    for (int e = 0; e < 3; e++) {
        int idx = tid + 512 * e;
        if (idx < 1505) atomicAdd(acc + idx, part[e]);
    }
    if (tid < 64) atomicAdd(acc + 1505, rows);
}

// residuals r = y - base . phi: acc[0..8) += r, acc[8..16) += r^2 (valid rows); with stats
// given (pass 2), t = (r - mean) / std
__global__ void sur_residual_kernel(const float *x, const float *y, const int *valid, long long n, const float *norm,
                                    double *acc, float *t) {
    double s1[8] = {0, 0, 0, 0, 0, 0, 0, 0}, s2[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        if (!valid[r]) {
            if (t)
                for (int k = 0; k < 8; k++) t[8 * r + k] = 0.f;
            continue;
        }
        float x4[4] = {x[4 * r], x[4 * r + 1], x[4 * r + 2], x[4 * r + 3]}, phi[kSurBasis];
        sur_basis(x4, phi);
        for (int k = 0; k < 8; k++) {
            float b = 0.f;
            for (int m = 0; m < kSurBasis; m++) b += norm[16 + k * kSurBasis + m] * phi[m];
            float res = y[8 * r + k] - b;
            if (t) {
                t[8 * r + k] = (res - norm[k]) / norm[8 + k];
            } else {
                s1[k] += res;
                s2[k] += (double)res * res;
            }
        }
    }
    if (!t)
        for (int k = 0; k < 8; k++) {
            atomicAdd(acc + k, s1[k]);
            atomicAdd(acc + 8 + k, s2[k]);
        }
}

}  // namespace prt

namespace {

constexpr size_t kAuxBytes = 2048;            // loss, error flag, then the normalisation
constexpr int kNormFloats = 16 + 8 * kSurBasis;

#define SK(x)                     \
    do {                          \
        if ((x) != cudaSuccess) { \
            cudaGetLastError();   \
            return RT_ERR_CUDA;   \
        }                         \
    } while (0)

int ensure_mlp(rt_ctx *c) {
    if (c->d_theta) return RT_OK;
    if (mlp_init_attributes() != 0) return RT_ERR_CUDA;
    size_t pb = kMlpParams * sizeof(float);
    if (cudaMalloc(&c->d_theta, 4 * pb) != cudaSuccess || cudaMalloc(&c->d_wpk, kPkWBytes) != cudaSuccess ||
        cudaMalloc(&c->d_tpk, kPkTBytes) != cudaSuccess || cudaMalloc(&c->d_mlpaux, kAuxBytes) != cudaSuccess) {
        // all or nothing: d_theta is what later calls test
        cudaFree(c->d_theta);
        cudaFree(c->d_wpk);
        cudaFree(c->d_tpk);
        cudaFree(c->d_mlpaux);
        c->d_theta = nullptr;
        c->d_wpk = nullptr;
        c->d_tpk = nullptr;
        c->d_mlpaux = nullptr;
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    SK(cudaMemsetAsync(c->d_theta, 0, 4 * pb, c->stream));
    SK(cudaMemsetAsync(c->d_mlpaux, 0, kAuxBytes, c->stream));
    return RT_OK;
}

// The per-block gradient partials of up to nb blocks of 128 samples (and their losses after them).
int ensure_gpart(rt_ctx *c, long long nb) {
    if (c->gpart_cap >= nb) return RT_OK;
    cudaFree(c->d_gpart);
    c->d_gpart = nullptr;
    c->gpart_cap = 0;
    if (cudaMalloc(&c->d_gpart, (size_t)nb * (kMlpParams + 1) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    c->gpart_cap = nb;
    return RT_OK;
}
float *gpart_loss(rt_ctx *c) { return c->d_gpart + c->gpart_cap * kMlpParams; }
constexpr long long kGradChunkBlocks = 1024;  // rt_mlp_grad: samples per launch, in blocks of 128

float *mlp_m(rt_ctx *c) { return c->d_theta + kMlpParams; }
float *mlp_v(rt_ctx *c) { return c->d_theta + 2 * kMlpParams; }
float *mlp_g(rt_ctx *c) { return c->d_theta + 3 * kMlpParams; }
float *aux_loss(rt_ctx *c) { return reinterpret_cast<float *>(c->d_mlpaux); }
unsigned *aux_err(rt_ctx *c) { return reinterpret_cast<unsigned *>(c->d_mlpaux) + 1; }
// 8 means, 8 standard deviations, 8 x 35 baseline coefficients (the rt_mlp_norm order)
float *aux_mean(rt_ctx *c) { return reinterpret_cast<float *>(c->d_mlpaux) + 4; }

int copy_in(rt_ctx *c, void *dst, const void *src, size_t bytes) {
    cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SK(cudaMemcpyAsync(dst, src, bytes, k, c->stream));
    return RT_OK;
}

SurBox box_of(const rt_mlp_norm &nm) {
    SurBox b;
    for (int j = 0; j < 4; j++) {
        b.lo[j] = nm.lo[j];
        b.hi[j] = nm.hi[j];
    }
    return b;
}

}  // namespace

extern "C" {

int rt_mlp_set_params(rt_ctx *c, const float *theta, const rt_mlp_norm *norm) {
    if (!c || !theta || !norm) return RT_ERR_INVALID;
    for (int j = 0; j < 4; j++)
        if (!(norm->hi[j] > norm->lo[j])) return RT_ERR_INVALID;
    SK(cudaSetDevice(c->device));
    int rv = ensure_mlp(c);
    if (rv) return rv;
    rv = copy_in(c, c->d_theta, theta, kMlpParams * sizeof(float));
    if (rv) return rv;
    SK(cudaMemcpyAsync(aux_mean(c), norm->y_mean, kNormFloats * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    launch_mlp_pack(c->d_theta, c->d_wpk, c->d_tpk, c->stream);
    SK(cudaGetLastError());
    SK(cudaStreamSynchronize(c->stream));
    c->mlp_norm = *norm;
    c->have_mlp = true;
    return RT_OK;
}

int rt_mlp_get_params(rt_ctx *c, float *theta, rt_mlp_norm *norm) {
    if (!c || !c->have_mlp) return RT_ERR_NOT_READY;
    SK(cudaSetDevice(c->device));
    if (theta) {
        SK(cudaMemcpyAsync(theta, c->d_theta, kMlpParams * sizeof(float), cudaMemcpyDefault, c->stream));
        SK(cudaStreamSynchronize(c->stream));
    }
    if (norm) *norm = c->mlp_norm;
    return RT_OK;
}

int rt_mlp_forward(rt_ctx *c, const float *x, long long n, float *y) {
    if (!c || !x || !y || n < 0) return RT_ERR_INVALID;
    if (!c->have_mlp) return RT_ERR_NOT_READY;
    if (!is_device_ptr(x) || !is_device_ptr(y)) return RT_ERR_INVALID;
    if (n == 0) return RT_OK;
    SK(cudaSetDevice(c->device));
    SK(cudaMemsetAsync(aux_err(c), 0, sizeof(unsigned), c->stream));
    long long tiles = (n + 127) / 128;
    int grid = (int)std::min<long long>(tiles, (long long)c->nsm * 4);
    launch_mlp_forward(x, y, n, c->d_wpk, aux_err(c), grid, c->stream);
    SK(cudaGetLastError());
    unsigned err = 0;
    SK(cudaMemcpyAsync(&err, aux_err(c), sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    SK(cudaStreamSynchronize(c->stream));
    return err ? RT_ERR_STALL : RT_OK;
}

int rt_mlp_grad(rt_ctx *c, const float *x, const float *t, long long n, float *grad, float *loss) {
    if (!c || !x || !t || !grad || n < 1) return RT_ERR_INVALID;
    if (!c->have_mlp) return RT_ERR_NOT_READY;
    if (!is_device_ptr(x) || !is_device_ptr(t)) return RT_ERR_INVALID;
    SK(cudaSetDevice(c->device));
    const long long nb = (n + 127) / 128;
    int rv = ensure_gpart(c, std::min(nb, kGradChunkBlocks));
    if (rv) return rv;
    SK(cudaMemsetAsync(c->d_mlpaux, 0, 2 * sizeof(float), c->stream));
    // chunks of at most kGradChunkBlocks blocks, each summed in block order onto the last
    for (long long b0 = 0; b0 < nb; b0 += kGradChunkBlocks) {
        const long long nbk = std::min(kGradChunkBlocks, nb - b0), off = b0 * 128, nk = std::min(n - off, nbk * 128);
        launch_mlp_grad(x + 4 * off, t + 8 * off, nk, n, c->d_wpk, c->d_tpk, c->d_gpart, gpart_loss(c), aux_err(c),
                        c->stream);
        launch_mlp_sum(c->d_gpart, gpart_loss(c), (int)nbk, mlp_g(c), aux_loss(c), b0 > 0, c->stream);
    }
    SK(cudaGetLastError());
    float h[2];
    SK(cudaMemcpyAsync(grad, mlp_g(c), kMlpParams * sizeof(float), cudaMemcpyDefault, c->stream));
    SK(cudaMemcpyAsync(h, c->d_mlpaux, 2 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    SK(cudaStreamSynchronize(c->stream));
    if (loss) *loss = h[0];
    unsigned err;
    memcpy(&err, &h[1], sizeof(err));
    return err ? RT_ERR_STALL : RT_OK;
}

int rt_mlp_train(rt_ctx *c, const float *x, const float *t, long long n, int steps, int batch, float lr,
                 uint64_t seed, float *loss_curve) {
    if (!c || !x || !t || n < 128 || steps < 1 || batch < 128 || batch % 128 || batch > n || !(lr > 0.f))
        return RT_ERR_INVALID;
    if (!c->have_mlp) return RT_ERR_NOT_READY;
    if (!is_device_ptr(x) || !is_device_ptr(t)) return RT_ERR_INVALID;
    SK(cudaSetDevice(c->device));
    const int nb = batch / 128;
    int rg = ensure_gpart(c, nb);
    if (rg) return rg;
    float *losses = nullptr;
    if (cudaMalloc(&losses, sizeof(float) * steps) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    int rv = RT_OK;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    if (cudaMemsetAsync(mlp_m(c), 0, 3 * kMlpParams * sizeof(float), c->stream) != cudaSuccess ||
        cudaMemsetAsync(losses, 0, sizeof(float) * steps, c->stream) != cudaSuccess ||
        cudaMemsetAsync(aux_err(c), 0, sizeof(unsigned), c->stream) != cudaSuccess)
        rv = RT_ERR_CUDA;
    unsigned long long st = seed;
    double pb1 = 1.0, pb2 = 1.0;
    long long nwin = (n - batch) / 128 + 1;
    for (int s = 0; s < steps && rv == RT_OK; s++) {
        // a random window of the (randomly drawn) training set
        st += 0x9E3779B97F4A7C15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        long long off = (long long)(z % (unsigned long long)nwin) * 128;
        pb1 *= b1;
        pb2 *= b2;
        float lrs = lr * 0.5f * (1.0f + cosf(3.14159265f * s / steps));  // cosine decay
        launch_mlp_grad(x + 4 * off, t + 8 * off, batch, batch, c->d_wpk, c->d_tpk, c->d_gpart, gpart_loss(c),
                        aux_err(c), c->stream);
        launch_mlp_adam(c->d_theta, mlp_m(c), mlp_v(c), c->d_gpart, gpart_loss(c), nb, losses + s, lrs, b1, b2, eps,
                        (float)(1.0 - pb1), (float)(1.0 - pb2), c->stream);
        launch_mlp_pack(c->d_theta, c->d_wpk, c->d_tpk, c->stream);
        if (cudaGetLastError() != cudaSuccess) rv = RT_ERR_CUDA;
    }
    unsigned err = 0;
    if (rv == RT_OK && loss_curve &&
        cudaMemcpyAsync(loss_curve, losses, sizeof(float) * steps, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rv = RT_ERR_CUDA;
    if (rv == RT_OK && cudaMemcpyAsync(&err, aux_err(c), sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rv = RT_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rv = RT_ERR_CUDA;
    cudaFree(losses);
    cudaGetLastError();
    if (rv == RT_OK && err) rv = RT_ERR_STALL;
    return rv;
}

int rt_surrogate_dataset(rt_ctx *c, const float box[8], long long n, uint64_t seed, float *x, float *y, int *valid) {
    if (!c || !box || n < 1 || !x || !y || !valid) return RT_ERR_INVALID;
    for (int j = 0; j < 4; j++)
        if (!(box[4 + j] > box[j])) return RT_ERR_INVALID;
    if (!(box[1] > 0.f) || box[5] > 1.5707964f || !(box[3] > 3.0f)) return RT_ERR_INVALID;
    if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(valid)) return RT_ERR_INVALID;
    SK(cudaSetDevice(c->device));
    SurBox b;
    for (int j = 0; j < 4; j++) {
        b.lo[j] = box[j];
        b.hi[j] = box[4 + j];
    }
    KappaTables T{c->d_syn, c->d_gl, c->d_gl + 8};
    sur_dataset_kernel<<<c->nsm * 8, 128, 0, c->stream>>>(T, b, seed, n, x, y, valid);
    SK(cudaGetLastError());
    SK(cudaStreamSynchronize(c->stream));
    return RT_OK;
}

int rt_surrogate_fit(rt_ctx *c, const float *x, const float *y, const int *valid, long long n, float *t,
                     rt_mlp_norm *norm) {
    if (!c || !x || !y || !valid || !t || !norm || n < kSurBasis) return RT_ERR_INVALID;
    if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(valid) || !is_device_ptr(t)) return RT_ERR_INVALID;
    SK(cudaSetDevice(c->device));
    double *acc = nullptr;
    float *dnorm = nullptr;
    if (cudaMalloc(&acc, 1520 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dnorm, kNormFloats * sizeof(float)) != cudaSuccess) {
        cudaFree(acc);
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    const int B = kSurBasis;
    std::vector<double> h(1520, 0.0);
    auto run = [&]() -> int {
        // 1. normal equations of the baseline over the valid rows
        SK(cudaMemsetAsync(acc, 0, 1520 * sizeof(double), c->stream));
        sur_normal_kernel<<<c->nsm * 2, 512, 0, c->stream>>>(x, y, valid, n, acc);
        SK(cudaGetLastError());
        SK(cudaMemcpyAsync(h.data(), acc, 1506 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SK(cudaStreamSynchronize(c->stream));
        const double rows = h[1505];
        if (rows < 2.0 * B) return RT_ERR_INVALID;
        // 2. Cholesky factor of phi^T phi (with a tiny ridge) and the 8 solutions
        std::vector<double> A(h.begin(), h.begin() + B * B), L(B * B, 0.0);
        double tr = 0.0;
        for (int i = 0; i < B; i++) tr += A[i * B + i];
        for (int i = 0; i < B; i++) A[i * B + i] += 1e-10 * tr / B;
        for (int i = 0; i < B; i++)
            for (int j = 0; j <= i; j++) {
                double sum = A[i * B + j];
                for (int k = 0; k < j; k++) sum -= L[i * B + k] * L[j * B + k];
                if (i == j) {
                    if (!(sum > 0.0)) return RT_ERR_INVALID;
                    L[i * B + i] = std::sqrt(sum);
                } else {
                    L[i * B + j] = sum / L[j * B + j];
                }
            }
        for (int k = 0; k < 8; k++) {
            std::vector<double> z(B), b(B);
            for (int i = 0; i < B; i++) {
                double sum = h[1225 + i * 8 + k];
                for (int j = 0; j < i; j++) sum -= L[i * B + j] * z[j];
                z[i] = sum / L[i * B + i];
            }
            for (int i = B - 1; i >= 0; i--) {
                double sum = z[i];
                for (int j = i + 1; j < B; j++) sum -= L[j * B + i] * b[j];
                b[i] = sum / L[i * B + i];
            }
            for (int i = 0; i < B; i++) norm->base[k][i] = (float)b[i];
            norm->y_mean[k] = 0.f;
            norm->y_std[k] = 1.f;
        }
        // 3. residual mean and standard deviation
        SK(cudaMemcpyAsync(dnorm, norm->y_mean, kNormFloats * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        SK(cudaMemsetAsync(acc, 0, 16 * sizeof(double), c->stream));
        sur_residual_kernel<<<c->nsm * 4, 256, 0, c->stream>>>(x, y, valid, n, dnorm, acc, nullptr);
        SK(cudaGetLastError());
        SK(cudaMemcpyAsync(h.data(), acc, 16 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SK(cudaStreamSynchronize(c->stream));
        for (int k = 0; k < 8; k++) {
            double m = h[k] / rows, var = h[8 + k] / rows - m * m;
            norm->y_mean[k] = (float)m;
            norm->y_std[k] = (float)std::sqrt(std::max(var, 1e-30));
        }
        // 4. standardised residual targets
        SK(cudaMemcpyAsync(dnorm, norm->y_mean, kNormFloats * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        sur_residual_kernel<<<c->nsm * 4, 256, 0, c->stream>>>(x, y, valid, n, dnorm, acc, t);
        SK(cudaGetLastError());
        SK(cudaStreamSynchronize(c->stream));
        return RT_OK;
    };
    int rv = run();
    cudaFree(acc);
    cudaFree(dnorm);
    cudaGetLastError();
    return rv;
}

int rt_surrogate_coeffs(rt_ctx *c, const double *in, long long n, double *out, uint8_t *inside) {
    if (!c || !in || !out || n < 0) return RT_ERR_INVALID;
    if (!c->have_mlp) return RT_ERR_NOT_READY;
    if (!is_device_ptr(in) || !is_device_ptr(out) || (inside && !is_device_ptr(inside))) return RT_ERR_INVALID;
    if (n == 0) return RT_OK;
    SK(cudaSetDevice(c->device));
    float *xn = nullptr;
    if (cudaMalloc(&xn, (size_t)n * 12 * sizeof(float) + (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    float *yh = xn + 4 * n;
    unsigned char *ins = reinterpret_cast<unsigned char *>(yh + 8 * n);
    SurBox b = box_of(c->mlp_norm);
    KappaTables T{c->d_syn, c->d_gl, c->d_gl + 8};
    int rv = RT_OK;
    sur_features_kernel<<<c->nsm * 8, 128, 0, c->stream>>>(in, n, b, xn, ins);
    if (cudaMemsetAsync(aux_err(c), 0, sizeof(unsigned), c->stream) != cudaSuccess) rv = RT_ERR_CUDA;
    long long tiles = (n + 127) / 128;
    launch_mlp_forward(xn, yh, n, c->d_wpk, aux_err(c), (int)std::min<long long>(tiles, (long long)c->nsm * 4),
                       c->stream);
    sur_expand_kernel<<<c->nsm * 8, 128, 0, c->stream>>>(T, in, n, xn, yh, aux_mean(c), ins, out);
    if (inside && cudaMemcpyAsync(inside, ins, (size_t)n, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        rv = RT_ERR_CUDA;
    unsigned err = 0;
    if (cudaGetLastError() != cudaSuccess) rv = RT_ERR_CUDA;
    if (cudaMemcpyAsync(&err, aux_err(c), sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        rv = RT_ERR_CUDA;
    cudaFree(xn);
    cudaGetLastError();
    if (rv == RT_OK && err) rv = RT_ERR_STALL;
    return rv;
}

}  // extern "C"
