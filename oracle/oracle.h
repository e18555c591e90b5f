/*
 * Plain FP64 CPU oracle for polarized general-relativistic ray tracing.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library. The CUDA library shares no code, header, table or constant
 * with it.
 *
 * What it computes (the paper, Section 2.1): one photon per camera pixel. A null geodesic
 * is integrated backward in time from the camera and saved. Then the covariant, fully
 * polarized transfer equations (coherency matrix in the coordinate frame; synchrotron
 * emission, absorption, Faraday rotation and conversion) are integrated along the saved
 * path toward the observer. Section 2.2 states that the CPU code saves the path, and this
 * oracle does too.
 *
 * The paper leaves every formula to its method paper, which is not available here. Each
 * function states the reading it implements. Every reading is listed in the design notes.
 *
 * Parity unpinned (the values below follow from published model constants or from a reading,
 * and nothing independent fixes them; every other function has a pin in tests/):
 *  - the middle range of the Shcherbakov correction functions of the rotativities: the fit is
 *    pinned at X -> 0 (cold-plasma rates) and at large X (its closed-form X^(-8/3) asymptote),
 *    and between them it is the transcription of a published fit;
 *  - the kappa rotativities (kappa.c) as a reading: their distribution averages are pinned by an
 *    independent quadrature, but the reading itself is exact for Maxwell-Juttner electrons only;
 *  - the absolute flux scale of the ADAF and grid models, which follows from the model constants.
 * The emissivities, j_V included, are pinned by the exact sum over cyclotron harmonics; the
 * camera-to-flux chain and the depth maps by the closed-form image of a static sphere.
 */
#ifndef PR_ORACLE_H
#define PR_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_HORIZON = 1, ORA_ESCAPE = 2, ORA_NMAX = 3, ORA_NAN = 4 };
enum { ORA_MODEL_ADAF = 1, ORA_MODEL_GRID = 2, ORA_MODEL_SPHERE = 3 };
enum { ORA_EDF_THERMAL = 0, ORA_EDF_KAPPA = 1 };

typedef struct {
    double a, incl_deg, r_cam, freq_hz, fov_M;
    int nx, ny;
    double M_bh_g, dist_cm;
    double eps;
    int nmax;
} ora_camera;

typedef struct {
    int kind;
    /* ADAF */
    double n0, T0, beta, f_kep, Ti_over_Te, r_out_emit;
    /* FMKS grid */
    int n1, n2, n3;
    double r_in, r_out, hslope, poly_xt, poly_alpha, mks_smooth;
    const float *prims; /* [n1][n2][n3][8]: rho,u,U1,U2,U3,B1,B2,B3 */
    double M_unit, R_high, R_low, sigma_cut, gamma_ad;
    /* electron distribution */
    int edf;
    double kappa;
    /* test switch: keep only j_I and a_I in the polarized transfer (for the unpolarized pin) */
    int unpol_test;
    /* static sphere (a pin with a closed-form image, not a model of the paper): Theta_e and B
     * constant for r < sph_R, n_e constant (sph_smooth 0) or sph_ne (1 - r^2/R^2)^2
     * (sph_smooth 1), fluid at rest (u along d_t), field along d_phi */
    double sph_R, sph_ne, sph_Te, sph_B;
    int sph_smooth;
} ora_model;

/* geometry */
void ora_metric_ks(double a, double r, double th, double g[16]);
int ora_invert4(const double g[16], double ginv[16]);
void ora_metric_derivs(double a, double r, double th, double dgr[16], double dgth[16]);
void ora_connection(double a, double r, double th, double G[64]); /* G[mu*16+al*4+be] */

/* camera + geodesic */
void ora_camera_ray(const ora_camera *cam, double px, double py, double x[4], double K[4]);
/* states[n*9]: t r th ph Kt Kr Kth Kph h (h<0 marks a pole reflection on that step) */
int ora_trace_geodesic(const ora_camera *cam, double px, double py, int maxstates,
                       double *states, int *status);
/* the transfer's transport of one index of N: a vector f at saved point M carried back to
 * points M-1..0; out[(M+1)*4], row n at point n */
void ora_transport_vector(double a, const double *states, int M, const double f[4], double *out);
/* the transfer's camera reading of N^{mu nu} (Nre + i Nim, row-major) for pixel (px, py):
 * S = (I, Q, U, V) on the image basis x ~ e_phi, y ~ -e_theta */
void ora_camera_stokes(const ora_camera *cam, double px, double py, const double Nre[16], const double Nim[16],
                       double S[4]);

/* plasma */
double ora_fmks_theta(const ora_model *m, double X1, double X2, double *dth1, double *dth2);
double ora_fmks_x2(const ora_model *m, double X1, double th);
void ora_grid_interp(const ora_model *m, double X1, double X2, double X3, double out[8]);
/* out: ne, Thetae, B_gauss, valid, ucon[4], bcon[4]  (12 doubles) */
void ora_plasma(const ora_camera *cam, const ora_model *m, const double x[4], double out[12]);
/* fluid tetrad e[0..3][4] at x for past-directed K; returns theta_B */
double ora_fluid_tetrad(double a, const double x[4], const double K[4], const double u[4], const double b[4],
                        double e[16]);

/* coefficients + transfer */
double ora_bessel_k_scaled(int n, double z); /* e^z K_n(z) */
/* out: jI jQ jV aI aQ aV rQ rV (cgs) */
void ora_thermal_coeffs(double ne, double Thetae, double B, double nu, double thetaB, double out[8]);
/* kappa.c: synchrotron kernels (F, G, H)(x) and coefficients by quadrature over a kappa
 * distribution (kappa > 3) or, for kappa <= 0, over the Maxwell-Juttner distribution */
void ora_synch_kernels(double x, double out[3]);
void ora_kappa_coeffs(double ne, double Thetae, double B, double nu, double thetaB, double kappa, double out[8]);
/* coef: jI jQ jU jV aI aQ aU aV rQ rU rV ; exact constant-coefficient solution over ds */
void ora_substep(const double coef[11], double ds, const double S0[4], double S1[4]);

/* full pixels: image-plane pixel (ix, iy) of the camera grid; pert 0 none, 1 px+ulp, 2 py+ulp.
 * depth (optional, 2 per pixel): tau = sum alpha_I ds and phi = sum rho_V ds over the emitting
 * points, the exponents of the isotropic absorption and of the Faraday rotation along the ray. */
int ora_render_pixels(const ora_camera *cam, const ora_model *m, int npix, const int *ix,
                      const int *iy, int pert, double *iquv, int *nsteps, int *status,
                      double *minpol, double *depth, int nthreads);
/* Stokes I alone with j_I and a_I only (the unpolarized transfer), per listed pixel */
int ora_render_unpol(const ora_camera *cam, const ora_model *m, int npix, const int *ix, const int *iy,
                     double *Iout, int nthreads);
void ora_image_stats(const ora_camera *cam, const double *iquv, long npix, double *flux_jy,
                     double *lp, double *cp);

#ifdef __cplusplus
}
#endif
#endif
