// Set-up and reduction kernels: the FMKS inverse table and the image statistics.
#include "transfer.cuh"

namespace prt {

// Table of X2(w, theta) for the FMKS map theta = theta_G(X2) + w (theta_J(X2) - theta_G(X2)),
// w in [0, 1] (64 rows), theta in [0, pi] (1024 columns), by bisection to the last bit. The
// transfer kernels start Newton's method from a bilinear read of this table.
__global__ void x2_table_kernel(GridModel g, double *tab, float *tabf) {
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
    tabf[idx] = (float)(0.5 * (lo + hi));
}

void launch_x2_table(const GridModel &g, double *table, float *table_f, cudaStream_t s) {
    int n = kX2TabW * kX2TabT;
    x2_table_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, table, table_f);
}

// Image statistics in two deterministic passes: each block takes a fixed contiguous range of
// pixels, sums it with Kahan compensation per thread and a pairwise tree in shared memory, and
// writes its partial sums; one block then adds the partials in block order. The epilogue forms
// the flux sum(I) dOmega 1e23 [Jy] and the net polarization fractions.
constexpr int kStatThreads = 256;

template <typename T, int NC>  // NC components per pixel: 4 (IQUV) or 1 (I)
__global__ void __launch_bounds__(kStatThreads) image_partial_kernel(const T *img, long long npix, double *part) {
    __shared__ double sh[4][kStatThreads];
    long long per = (npix + gridDim.x - 1) / gridDim.x;
    long long p0 = (long long)blockIdx.x * per, p1 = min(npix, p0 + per);
    double s[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
    for (long long p = p0 + threadIdx.x; p < p1; p += kStatThreads) {
#pragma unroll
        for (int k = 0; k < NC; k++) {
            double y = (double)img[NC * p + k] - cmp[k];
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
    if (threadIdx.x < 4) part[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void image_final_kernel(const double *part, int nblocks, double domega, double *out) {
    if (threadIdx.x != 0) return;
    double s[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
    for (int b = 0; b < nblocks; b++)
        for (int k = 0; k < 4; k++) {
            double y = part[4 * b + k] - cmp[k];
            double t = s[k] + y;
            cmp[k] = (t - s[k]) - y;
            s[k] = t;
        }
    double I = s[0], Q = s[1], U = s[2], V = s[3];
    out[0] = I;
    out[1] = Q;
    out[2] = U;
    out[3] = V;
    out[4] = I * domega * 1e23;
    out[5] = sqrt(Q * Q + U * U) / I;
    out[6] = V / I;
}

// out must hold 8 + 4 * kStatBlocks doubles (the partials live after the 7 results).
void launch_image_sums(const void *img, int form, long long npix, double domega, double *out, cudaStream_t s) {
    double *part = out + 8;
    if (form == 0)
        image_partial_kernel<double, 4><<<kStatBlocks, kStatThreads, 0, s>>>((const double *)img, npix, part);
    else if (form == 1)
        image_partial_kernel<float, 4><<<kStatBlocks, kStatThreads, 0, s>>>((const float *)img, npix, part);
    else
        image_partial_kernel<float, 1><<<kStatBlocks, kStatThreads, 0, s>>>((const float *)img, npix, part);
    image_final_kernel<<<1, 32, 0, s>>>(part, kStatBlocks, domega, out);
}

}  // namespace prt
