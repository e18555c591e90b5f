// Visibilities of an image (the paper's Section 2.1: power-of-two images go straight to the
// interferometer's Fourier plane, with no regridding): V(u, v) = sum over pixels of
// S(x, y) dOmega e^{-2 pi i (u x + v y)} [Jy], x, y the pixel-centre angles from the image
// centre, on the image's own grid u_k = k / FOV, k = -nx/2 .. nx/2 - 1 (and v likewise).
// One Stokes plane is scaled into a complex buffer, transformed with cuFFT, and a kernel
// applies the half-pixel phase and the centring shift.
#include <cufft.h>

#include <cmath>

#include "host_util.cuh"
#include "polrt.h"

using namespace prt;

namespace {

template <typename T, typename C>
__global__ void vis_gather_kernel(const T *img, int ncomp, int comp, long long npix, double scale, C *buf) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
        buf[p].x = (decltype(buf[p].x))(scale * (double)img[ncomp * p + comp]);
        buf[p].y = 0;
    }
}

// out[l + ny/2][k + nx/2] = F[l mod ny][k mod nx] e^{-2 pi i (k (1/2 - nx/2) / nx + l (1/2 - ny/2) / ny)}
template <typename C>
__global__ void vis_phase_kernel(const C *F, int nx, int ny, C *out) {
    long long n = (long long)nx * ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int r = (int)(q / nx), c = (int)(q % nx);
        int k = c - nx / 2, l = r - ny / 2;
        int sk = ((k % nx) + nx) % nx, sl = ((l % ny) + ny) % ny;
        C f = F[(long long)sl * nx + sk];
        double ph = -2.0 * kPi * ((double)k * (0.5 - 0.5 * nx) / nx + (double)l * (0.5 - 0.5 * ny) / ny);
        double s, co;
        sincos(ph, &s, &co);
        out[q].x = (decltype(out[q].x))(co * f.x - s * f.y);
        out[q].y = (decltype(out[q].y))(s * f.x + co * f.y);
    }
}

}  // namespace

extern "C" {

int rt_image_visibilities(rt_ctx *c, const void *img, int form, int stokes, void *vis) {
    if (!c || !img || !vis || form < RT_FP64 || form > RT_UNPOL || stokes < 0 || stokes > 3) return RT_ERR_INVALID;
    if (form == RT_UNPOL && stokes != 0) return RT_ERR_INVALID;
    if (!c->have_cam) return RT_ERR_NOT_READY;
    if (cudaSetDevice(c->device) != cudaSuccess) return RT_ERR_CUDA;
    const int nx = c->cam.nx, ny = c->cam.ny;
    const long long npix = (long long)nx * ny;
    const bool dbl = form == RT_FP64;
    const int ncomp = form == RT_UNPOL ? 1 : 4;
    const size_t esz = dbl ? sizeof(double) : sizeof(float), csz = dbl ? sizeof(cufftDoubleComplex) : sizeof(cufftComplex);
    double L = kG * c->cam.M_bh_g / (kC * kC);
    double pixang = c->cam.fov_M * L / (nx * c->cam.dist_cm);
    double scale = pixang * pixang * 1e23;  // I dOmega in Jy
    // buffers: the image (if on the host), the transform, the result (if on the host)
    bool img_dev = is_device_ptr(img), vis_dev = is_device_ptr(vis);
    size_t need = (size_t)npix * (csz * (vis_dev ? 1 : 2) + (img_dev ? 0 : ncomp * esz));
    void *buf = nullptr;
    if (cudaMalloc(&buf, need) != cudaSuccess) {
        cudaGetLastError();
        return RT_ERR_NOMEM;
    }
    char *b = (char *)buf;
    void *F = b;
    b += npix * csz;
    void *out = vis_dev ? vis : (void *)b;
    if (!vis_dev) b += npix * csz;
    const void *d_img = img;
    int rv = RT_OK;
    cufftHandle plan = 0;
    bool have_plan = false;
    if (!img_dev) {
        d_img = b;
        if (cudaMemcpyAsync((void *)d_img, img, (size_t)npix * ncomp * esz, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            rv = RT_ERR_CUDA;
    }
    int grid = c->nsm * 4;
    if (rv == RT_OK) {
        if (dbl)
            vis_gather_kernel<<<grid, 256, 0, c->stream>>>((const double *)d_img, ncomp, stokes, npix, scale,
                                                          (cufftDoubleComplex *)F);
        else
            vis_gather_kernel<<<grid, 256, 0, c->stream>>>((const float *)d_img, ncomp, stokes, npix, scale,
                                                          (cufftComplex *)F);
        if (cufftPlan2d(&plan, ny, nx, dbl ? CUFFT_Z2Z : CUFFT_C2C) != CUFFT_SUCCESS) rv = RT_ERR_CUDA;
        else have_plan = true;
    }
    if (rv == RT_OK && cufftSetStream(plan, c->stream) != CUFFT_SUCCESS) rv = RT_ERR_CUDA;
    if (rv == RT_OK) {
        cufftResult r = dbl ? cufftExecZ2Z(plan, (cufftDoubleComplex *)F, (cufftDoubleComplex *)F, CUFFT_FORWARD)
                            : cufftExecC2C(plan, (cufftComplex *)F, (cufftComplex *)F, CUFFT_FORWARD);
        if (r != CUFFT_SUCCESS) rv = RT_ERR_CUDA;
    }
    if (rv == RT_OK) {
        if (dbl)
            vis_phase_kernel<<<grid, 256, 0, c->stream>>>((const cufftDoubleComplex *)F, nx, ny, (cufftDoubleComplex *)out);
        else
            vis_phase_kernel<<<grid, 256, 0, c->stream>>>((const cufftComplex *)F, nx, ny, (cufftComplex *)out);
        if (cudaGetLastError() != cudaSuccess) rv = RT_ERR_CUDA;
    }
    if (rv == RT_OK && !vis_dev &&
        cudaMemcpyAsync(vis, out, (size_t)npix * csz, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rv = RT_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rv = RT_ERR_CUDA;
    if (have_plan) cufftDestroy(plan);
    cudaFree(buf);
    cudaGetLastError();
    return rv;
}

}  // extern "C"
