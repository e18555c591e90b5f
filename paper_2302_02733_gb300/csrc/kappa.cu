// Kappa-distribution coefficients by quadrature: the synchrotron-kernel tables and the batch
// kernel behind rt_kappa_coeffs (one thread per point).
#include <cmath>
#include <vector>

#include "kappa.cuh"
#include "rt_kernels.cuh"

namespace prt {

// ln F, ln G, ln H at node i: trapezoid rule (step 1/100) on
// F/x = int_0^inf e^{-x cosh t} cosh(5t/3)/cosh t dt, G/x = int e^{-x cosh t} cosh(2t/3) dt,
// H = x int e^{-x cosh t} cosh(t/3) dt + int e^{-x cosh t} cosh(t/3)/cosh t dt.
__global__ void synch_table_kernel(double *lnk) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kSynTab) return;
    double x = exp(kSynLo + i * (kSynHi - kSynLo) / (kSynTab - 1));
    const double h = 0.01;
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int k = 0; k < 1000000; k++) {
        double t = k * h, ch = cosh(t);
        if (x * ch > 745.0) break;
        double e = exp(-x * ch) * (k == 0 ? 0.5 : 1.0);
        double c13 = cosh(t / 3.0);
        a += e * cosh(5.0 * t / 3.0) / ch;
        b += e * cosh(2.0 * t / 3.0);
        c += e * c13;
        d += e * c13 / ch;
    }
    lnk[i] = log(x * h * a);
    lnk[kSynTab + i] = log(x * h * b);
    lnk[2 * kSynTab + i] = log(x * h * c + h * d);
}

__global__ void kappa_quad_kernel(KappaTables T, const double *in, double *out, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double *v = in + 6 * q;
        double o[8];
        kappa_coeffs_quad(T, v[0], v[1], v[2], v[3], v[4], v[5], o);
#pragma unroll
        for (int k = 0; k < 8; k++) out[8 * q + k] = o[k];
    }
}

int launch_kappa_tables(double *lnk, double *gl, cudaStream_t s) {
    // 8-point Gauss-Legendre rule on [-1, 1] (Newton iteration on P_8 from Chebyshev guesses)
    const int n = 8;
    double hb[16];
    for (int i = 0; i < n; i++) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; j++) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        hb[i] = z;
        hb[8 + i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (cudaMemcpyAsync(gl, hb, sizeof(hb), cudaMemcpyHostToDevice, s) != cudaSuccess) return -1;
    synch_table_kernel<<<(kSynTab + 127) / 128, 128, 0, s>>>(lnk);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_kappa_quad(const KappaTables &T, const double *in, double *out, long long n, int grid, cudaStream_t s) {
    kappa_quad_kernel<<<grid, 128, 0, s>>>(T, in, out, n);
}

}  // namespace prt
