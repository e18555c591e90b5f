// Set-up and reduction kernels: the FMKS inverse table and the image statistics.
#include "transfer.cuh"

namespace prt {

// Table of X2(w, theta) for the FMKS map theta = theta_G(X2) + w (theta_J(X2) - theta_G(X2)),
// w in [0, 1] (64 rows), theta in [0, pi] (1024 columns), by bisection to the last bit. The
// transfer kernels start Newton's method from a bilinear read of this table.
__global__ void x2_table_kernel(GridModel g, double *tab) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kX2TabW * kX2TabT) return;
    int iw = idx / kX2TabT, it = idx % kX2TabT;
    double w = (double)iw / (kX2TabW - 1);
    double th = kPi * (double)it / (kX2TabT - 1);
    double lo = 0.0, hi = 1.0;
    for (int k = 0; k < 70; k++) {
        double mid = 0.5 * (lo + hi);
        if (fmks_theta_w<double>(g, w, mid, nullptr, nullptr) < th)
            lo = mid;
        else
            hi = mid;
    }
    tab[idx] = 0.5 * (lo + hi);
}

void launch_x2_table(const GridModel &g, double *table, cudaStream_t s) {
    int n = kX2TabW * kX2TabT;
    x2_table_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, table);
}

// Image statistics: compensated (Kahan) per-thread sums over a strided subset of pixels, then
// a pairwise tree in shared memory; one block, deterministic order. The epilogue forms the
// flux sum(I) dOmega 1e23 [Jy] and the net polarization fractions.
constexpr int kStatThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kStatThreads) image_sums_kernel(const T *img, long long npix, double domega,
                                                                   double *out) {
    __shared__ double sh[4][kStatThreads];
    double s[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
    for (long long p = threadIdx.x; p < npix; p += kStatThreads) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            double y = (double)img[4 * p + k] - cmp[k];
            double t = s[k] + y;
            cmp[k] = (t - s[k]) - y;
            s[k] = t;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kStatThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 4; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double I = sh[0][0], Q = sh[1][0], U = sh[2][0], V = sh[3][0];
        out[0] = I;
        out[1] = Q;
        out[2] = U;
        out[3] = V;
        out[4] = I * domega * 1e23;
        out[5] = sqrt(Q * Q + U * U) / I;
        out[6] = V / I;
    }
}

void launch_image_sums(const void *img, int form, long long npix, double domega, double *out, cudaStream_t s) {
    if (form == 0)
        image_sums_kernel<double><<<1, kStatThreads, 0, s>>>((const double *)img, npix, domega, out);
    else
        image_sums_kernel<float><<<1, kStatThreads, 0, s>>>((const float *)img, npix, domega, out);
}

}  // namespace prt
