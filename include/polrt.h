/*
 * polrt: polarized general-relativistic ray tracing on one GB300 (sm_103a).
 *
 * C ABI of the CUDA library. The method follows the paper's Section 2.1. One photon is
 * launched per camera pixel, and its null geodesic in the Kerr metric is integrated
 * backward in time and saved. The covariant, fully polarized transfer of Stokes I, Q, U, V
 * (synchrotron emission, self-absorption, Faraday rotation and conversion; the coherency
 * matrix is carried in the coordinate frame) is then integrated along the saved path
 * toward the observer. Plasma comes from a semi-analytic ADAF or from gridded GRMHD
 * primitives (Sections 2.1 and 3). Section 2.2 states that the CPU code saves the path. This
 * library does the same in a device-memory arena, so the transfer follows exactly the
 * states of the backward pass.
 *
 * Conventions for every call:
 *   - Return RT_OK (0) on success or a negative RT_ERR_* code; rt_error_string names it.
 *     Nothing throws across this boundary.
 *   - Work is enqueued on the context's CUDA stream and is asynchronous, unless a call
 *     says it synchronizes.
 *   - Pointers marked "host or device" are classified with cudaPointerGetAttributes.
 *   - The library never frees memory it did not allocate. The caller may hand it a
 *     device workspace (rt_set_workspace). Otherwise it allocates one and frees it in
 *     rt_destroy.
 *   - Units: geometry in M = GM/c^2 (G = c = 1); intensities in cgs
 *     (erg s^-1 cm^-2 Hz^-1 sr^-1); flux in Jy.
 *   - A context is not thread safe: it holds the camera, the model, the workspace and the
 *     pinned counters of its last call. Threads that share one must serialize their calls.
 *     Separate contexts, on one device or several, are independent, except for
 *     rt_render_static's shared array.
 *   - A rejected call (RT_ERR_INVALID, RT_ERR_NOT_READY, RT_ERR_SIZE) leaves the context as
 *     it was.
 */
#ifndef POLRT_H
#define POLRT_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RT_OK = 0,
    RT_ERR_INVALID = -1,    /* a bad argument; nothing was enqueued */
    RT_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    RT_ERR_NOMEM = -3,      /* an allocation failed */
    RT_ERR_NOT_READY = -4,  /* no model or no camera set */
    RT_ERR_WORKSPACE = -5,  /* the path arena ran out; rays carry RT_RAY_OVERFLOW */
    RT_ERR_SIZE = -6,       /* a size beyond a fixed limit of the call */
    RT_ERR_STALL = -7       /* a bounded wait ran out (inside a kernel, or rt_render's host wait of
                               600 s for a streamed render's chunks); results invalid */
};

enum { RT_MODEL_ADAF = 1, RT_MODEL_GRID = 2 };

/* Forms of the hot path. */
enum {
    RT_FP64 = 0,  /* geodesic, plasma, coefficients and transfer all in FP64; output double */
    RT_MIXED = 1, /* FP64 geodesic and path; FP32 plasma fetch, coefficients and transfer.
                     The Stokes vector is carried as a compensated pair (value + error term):
                     every step forms its change (screen re-projection, radiative step) as an
                     increment and adds it by an error-free sum, and the optical and Faraday
                     depths are Kahan sums. Output float. */
    RT_SURROGATE = 2, /* the mixed form with kappa electrons whose coefficients come from the
                        trained surrogate network (rt_mlp_*), evaluated on the tensor cores for
                        every saved state before the transfer; the quadrature answers outside
                        the network's box. Needs model edf RT_EDF_KAPPA and loaded
                        parameters. Output float. */
    RT_UNPOL = 3      /* Stokes I alone with j_I and a_I only (the unpolarized transfer, for
                        fitting loops): the FP64 geodesic, then an FP32 scalar transfer with a
                        compensated sum and no coherency transport. Thermal electrons. Output
                        nx*ny floats [iy][ix]; rt_image_stats gives the flux (LP = CP = 0). */
};

/* Per-pixel status codes written to the optional status buffer. */
enum {
    RT_RAY_HORIZON = 1,  /* reached r < 1.05 r_h */
    RT_RAY_ESCAPE = 2,   /* left r > r_cam moving outward */
    RT_RAY_NMAX = 3,     /* hit the step limit; the image keeps what was integrated */
    RT_RAY_NAN = 4,      /* a non-finite state; the pixel is zero */
    RT_RAY_OVERFLOW = 5  /* the path arena was full; the pixel is zero */
};

typedef struct rt_ctx rt_ctx;

/* Semi-analytic ADAF: n_e = n0 r^-3/2 [cm^-3], T_e = T0/r [K], B^2/8pi = n_e k T_e
 * (1 + Ti/Te)/beta, sub-Keplerian rotation f_kep l_K sin^2(theta) with infall from the
 * normalisation, field direction along KS components (1, 0, 1/r); emission for r <= r_out. */
typedef struct {
    double n0, T0, beta, f_kep, Ti_over_Te, r_out;
} rt_adaf_params;

/* Gridded GRMHD primitives on a cell-centred FMKS grid (X1 = ln r in [ln r_in, ln r_out],
 * X2 in [0, 1], X3 = phi in [0, 2 pi)). prims: n1*n2*n3*8 floats, layout
 * [n1][n2][n3][8] = rho, u, U1, U2, U3, B1, B2, B3 (HARM conventions: U the velocity relative
 * to the normal observer, B the field, both in FMKS components). The pointer may be host or
 * device memory; it is copied during rt_load_model and the caller keeps ownership. */
typedef struct {
    int n1, n2, n3;
    double r_in, r_out;
    double hslope, poly_xt, poly_alpha, mks_smooth;
    const float *prims;
    double M_unit;       /* mass unit [g]: rho_unit = M_unit / L^3 */
    double R_high, R_low;/* T_i/T_e = R_high b^2/(1+b^2) + R_low/(1+b^2), b = plasma beta */
    double sigma_cut;    /* no emission where b^2/rho exceeds this */
    double gamma_ad;     /* adiabatic index of the fluid */
} rt_grid_params;

enum { RT_EDF_THERMAL = 0, RT_EDF_KAPPA = 1 };

typedef struct {
    int kind; /* RT_MODEL_ADAF or RT_MODEL_GRID */
    rt_adaf_params adaf;
    rt_grid_params grid;
    /* electron distribution (Section 2.1: thermal or nonthermal): RT_EDF_THERMAL uses the
     * Maxwell-Juttner fits; RT_EDF_KAPPA the kappa distribution of index kappa (> 3) with
     * width w = (kappa - 3) Theta_e / kappa, by quadrature (RT_FP64, RT_MIXED) or by the
     * surrogate (RT_SURROGATE) */
    int edf;
    double kappa;
} rt_model_params;

/* Camera and image: a static observer at radius r_cam, inclination incl_deg, azimuth 0,
 * looking at the hole through a pinhole image plane fov_M wide (square pixels). freq_hz is
 * the observing frequency; M_bh_g and dist_cm set the length unit and the pixel solid angle. */
typedef struct {
    double a;         /* spin, |a| < 1 */
    double incl_deg;  /* in (0, 180) */
    double r_cam;
    double freq_hz;
    double fov_M;
    int nx, ny;
    double M_bh_g, dist_cm;
} rt_camera;

/* Counters of the last render, filled by rt_last_counters (which synchronizes). */
typedef struct {
    uint64_t rays, steps, points, emitting_points;
    uint64_t arena_blocks_used, arena_blocks_total;
    uint32_t n_horizon, n_escape, n_nmax, n_nan, n_overflow;
    float ms_geodesic, ms_transfer; /* device time of the two kernels (CUDA events); in an
                                     * overlapped render the span from the first launch's start
                                     * to the last one's end; 0 after a batch */
    float ms_total;                 /* device time of the whole render or batch */
    uint32_t chunks;                /* ray chunks of the last rt_render; 0 after a batch */
    uint32_t shape;                 /* launch shape of the last rt_render: 0 one pass (of each
                                     * kernel per chunk), 1 overlapped in two workspace halves,
                                     * 2 streamed (rt_render_config); 0 after a batch */
    uint32_t geodesic_launches;     /* geodesic kernels the last rt_render launched (one per
                                     * chunk, or one per streamed piece); 0 after a batch */
    uint32_t transfer_launches;     /* transfer kernels it launched (streamed: one per run of
                                     * complete chunks); 0 after a batch */
} rt_counters;

/* Create a context on CUDA device `device`, enqueueing on `stream` (a cudaStream_t, or
 * NULL for the legacy default stream). *out is owned by the caller and released with
 * rt_destroy. */
int rt_create(rt_ctx **out, int device, void *stream);
int rt_destroy(rt_ctx *ctx);
/* Change the stream later calls enqueue on. */
int rt_set_stream(rt_ctx *ctx, void *stream);

/* Load the plasma model (Section 2.1: semi-analytic prescription or GRMHD arrays).
 * Grid primitives are copied to a context-owned device buffer. Synchronizes on the copy. */
int rt_load_model(rt_ctx *ctx, const rt_model_params *p);

/* Camera: spin, inclination, distance, frequency, field of view and resolution. Copied.
 * RT_ERR_INVALID for |a| >= 1, an inclination outside (0, 180) degrees, a size, frequency,
 * field of view, mass or distance that is not positive, or r_cam <= 2 r_h; RT_ERR_SIZE for
 * more than 2^31 - 1 pixels. */
int rt_set_camera(rt_ctx *ctx, const rt_camera *cam);
/* The current camera, copied to *cam (which the caller owns); RT_ERR_NOT_READY before the
 * first rt_set_camera. Callers size their image buffers from it. */
int rt_get_camera(const rt_ctx *ctx, rt_camera *cam);

/* Geodesic step control: h = eps / (|K^r|/r + |K^th|/max(min(th, pi - th), 0.01) + |K^ph|),
 * classic RK4, at most nmax steps per ray. Defaults: eps = 0.05, nmax = 20000. */
int rt_set_integrator(rt_ctx *ctx, double eps, int nmax);

/* Device workspace for the path arena and counters (bytes >= rt_workspace_min_bytes). The
 * caller owns it; it must stay valid until the next rt_set_workspace or rt_destroy. Pass
 * NULL to go back to a library-owned workspace. */
int rt_set_workspace(rt_ctx *ctx, void *dev_ptr, size_t bytes);
size_t rt_workspace_min_bytes(void);
/* Workspace size the library would use for the current camera: every ray's path at once, as
 * the streamed overlapped shape needs (a sizing hint; smaller workspaces render in chunks). */
int rt_workspace_hint(const rt_ctx *ctx, size_t *bytes);

/* Render the IQUV image: out_iquv holds nx*ny*4 values, row-major [iy][ix][I,Q,U,V]
 * (double for RT_FP64, float for RT_MIXED and RT_SURROGATE; RT_UNPOL writes nx*ny floats of
 * I alone), host or device. Row iy = 0 is the bottom
 * (image y = -FOV/2); x runs along +e_phi and y along -e_theta of the camera. Stokes Q is
 * positive for E along x, and V > 0 for right-handed light in the IEEE/IAU sense. status:
 * optional nx*ny uint8 per-pixel codes (host or device), or NULL. The rays are processed in
 * chunks that fit the workspace. The call synchronizes the context's stream before it
 * returns (it reads the ray counters). It returns RT_ERR_WORKSPACE if any ray overflowed the
 * path arena; those pixels are zero with status RT_RAY_OVERFLOW. */
int rt_render(rt_ctx *ctx, int form, void *out_iquv, uint8_t *status);

/* rt_render that also writes, per pixel, the optical depth tau = sum alpha_I ds and the
 * Faraday depth phi = sum rho_V ds accumulated along the ray over its emitting points (the
 * exponents of the isotropic absorption and of the Faraday rotation that the constant-
 * coefficient steps of Section 2.1's transfer apply; alpha and rho in the fluid frame, ds the
 * fluid-frame path length). out_depth: nx*ny*2 values [iy][ix][tau, phi] of the form's type,
 * host or device; it must not be NULL. Both sums are compensated (Kahan) in either form. */
int rt_render_depths(rt_ctx *ctx, int form, void *out_iquv, uint8_t *status, void *out_depth);

/* Total flux [Jy] = sum(I) dOmega 1e23, dOmega = (fov_M L / (nx D))^2, and the net linear
 * and circular polarization fractions sqrt(sum Q^2 + sum U^2)/sum I, sum V / sum I, from an
 * image in `form` layout (host or device). A compensated device reduction; synchronizes. */
int rt_image_stats(rt_ctx *ctx, const void *iquv, int form, double *flux_jy, double *lp_frac,
                   double *cp_frac);

/* Synchrotron coefficients of n plasma points by quadrature over the electron distribution
 * (the nonthermal models of Section 2.1, integrated numerically as Section 4 proposes).
 * in: n x 6 doubles per point (n_e [cm^-3], Theta_e, B [G], nu [Hz] in the fluid frame,
 * theta_B [rad], kappa): kappa > 3 selects the kappa distribution with width
 * w = (kappa - 3) Theta_e / kappa, kappa <= 0 the Maxwell-Juttner distribution; other kappa
 * give zeros. out: n x 8 doubles (j_I, j_Q, j_V [erg s^-1 cm^-3 Hz^-1 sr^-1], a_I, a_Q, a_V,
 * r_Q, r_V [cm^-1]) in the polarization basis of rt_render (Q across the projected field).
 * Host or device pointers; synchronizes. */
int rt_kappa_coeffs(rt_ctx *ctx, const double *in, long long n, double *out);

/* ---- The nonthermal coefficient surrogate ---------------------------------------------------
 * A 4 -> 64 -> 64 -> 64 -> 8 perceptron with SiLU hidden units stands in for rt_kappa_coeffs. It
 * runs on the tensor cores (BF16 operands, FP32 accumulation), and is trained there.
 *
 * Inputs: f = (ln(nu / nu_c), theta_B folded into (0, pi/2], ln Theta_e, kappa) with
 * nu_c = (3/2) nu_B sin(theta_B) Theta_e^2, each mapped linearly from the box [lo, hi] to
 * [-1, 1] (x). Targets: the logarithms of the coefficients over known prefactors (the thermal
 * fits' prefactors; Shcherbakov's corrections for the rotativities), which depend on f only.
 * Each target k is base[k] . phi(x) + y_mean[k] + y_std[k] y_k with phi the 35 monomials of
 * degree <= 3 in x (order: 1; x_i; x_i x_j, i <= j; x_i x_j x_k, i <= j <= k) and y the
 * network's output: the polynomial carries the large trends, the network the standardised
 * residual. Parameters: RT_MLP_PARAMS floats,
 * layer after layer (4 -> 64, 64 -> 64, 64 -> 64, 64 -> 8), each as [out][in + 1] with the bias
 * in the last column. */
#define RT_MLP_PARAMS 9160
typedef struct {
    float lo[4], hi[4];          /* the training box of the inputs */
    float y_mean[8], y_std[8];   /* residual standardisation */
    float base[8][35];           /* polynomial baseline of each target */
} rt_mlp_norm;

/* Load parameters (host or device) and normalisation; builds the tensor-core images. */
int rt_mlp_set_params(rt_ctx *ctx, const float *theta, const rt_mlp_norm *norm);
/* Copy the current parameters (theta may be host or device, or NULL) and normalisation out. */
int rt_mlp_get_params(rt_ctx *ctx, float *theta, rt_mlp_norm *norm);
/* y[n][8] = network(x[n][4]) on normalised inputs (device pointers). RT_ERR_STALL if a bounded
 * wait for the tensor core ran out. */
int rt_mlp_forward(rt_ctx *ctx, const float *x, long long n, float *y);
/* Gradient of the mean squared error sum_(samples, outputs) (y - t)^2 / (8 n) with respect to
 * the parameters, and the loss (x, t device; grad host or device, RT_MLP_PARAMS floats). */
int rt_mlp_grad(rt_ctx *ctx, const float *x, const float *t, long long n, float *grad, float *loss);
/* Adam (beta 0.9, 0.999; cosine-decayed learning rate from lr) for `steps` steps on batches of
 * `batch` samples (a multiple of 128) taken as random windows of the n samples (device x, t:
 * standardised targets). Starts from the loaded parameters; loss_curve (host, steps floats)
 * may be NULL. */
int rt_mlp_train(rt_ctx *ctx, const float *x, const float *t, long long n, int steps, int batch, float lr,
                 uint64_t seed, float *loss_curve);
/* Training set of n points drawn uniformly (counter-based splitmix64 from seed) in the box
 * {lo[4], hi[4]} of the inputs (theta_B inside (0, pi/2], kappa > 3): x[n][4] normalised inputs,
 * y[n][8] unstandardised targets computed by the quadrature, valid[n] whether every target is
 * finite. Device pointers; synchronizes. */
int rt_surrogate_dataset(rt_ctx *ctx, const float box[8], long long n, uint64_t seed, float *x, float *y, int *valid);
/* Prepare training targets from a rt_surrogate_dataset set: fit the polynomial baseline by least
 * squares over the valid rows, and standardise the residuals. norm: lo and hi set by the caller
 * (the box); base, y_mean and y_std are filled. t[n][8] receives the standardised residuals
 * (zeros on invalid rows). Device x, y, valid, t. */
int rt_surrogate_fit(rt_ctx *ctx, const float *x, const float *y, const int *valid, long long n, float *t,
                     rt_mlp_norm *norm);
/* The surrogate's inputs f = (ln(nu/nu_c), theta_B folded into (0, pi/2], ln Theta_e, kappa) at
 * every emitting point of the current camera's rays (the points the transfer will visit), as
 * float4 rows written to feat (device) in no particular order, at most cap of them; *count
 * receives the number of emitting points (which may exceed cap). For choosing a training box
 * from an image. Synchronizes. */
int rt_render_features(rt_ctx *ctx, float *feat, long long cap, long long *count);
/* rt_kappa_coeffs through the surrogate: points inside the training box from the network,
 * others from the quadrature (inside[n], optional, tells which). Device pointers. */
int rt_surrogate_coeffs(rt_ctx *ctx, const double *in, long long n, double *out, uint8_t *inside);

/* Adaptive ray tracing (the paper's outlook: dense rays only near image features). Rays are
 * traced on a lattice of every base_step-th pixel (a power of two >= 2; last row and column
 * included); then, halving the side each level, the centre of each block between traced corners
 * is traced, and the block is refined (edge midpoints traced, children examined) when a Stokes
 * parameter at the centre differs from the corners' bilinear prediction by more than tol times
 * the lattice's largest intensity, or when the corner and centre rays ended differently;
 * otherwise its untraced pixels are filled by bilinear interpolation. Features smaller than
 * base_step that no lattice or centre ray touches are missed: choose base_step below the
 * smallest feature of interest. out (and
 * status, optional) are device buffers in rt_render's layout for form RT_FP64, RT_MIXED or
 * RT_UNPOL; every pixel is written. *rays_traced (optional) receives the number of rays
 * traced. Rays that overflow the path arena are marked RT_RAY_OVERFLOW as in rt_render; the
 * refinement still completes and the call then returns RT_ERR_WORKSPACE. Synchronizes. */
int rt_render_adaptive(rt_ctx *ctx, int form, void *out, uint8_t *status, int base_step, double tol,
                       long long *rays_traced);

/* Visibilities of one Stokes plane of an image (Section 2.1: power-of-two images are Fourier
 * transformed to the interferometer's visibilities without regridding):
 *   V(u, v) = sum over pixels of S(x, y) dOmega e^{-2 pi i (u x + v y)}   [Jy],
 * x, y the pixel-centre angles [rad] from the image centre (x along +e_phi, y along -e_theta),
 * dOmega the pixel solid angle, on the grid u = k / FOV, v = l / FOV (FOV in radians),
 * k = -nx/2 .. nx/2 - 1, l = -ny/2 .. ny/2 - 1. img: an image of the current camera in
 * `form` layout (host or device); stokes: 0..3 for I, Q, U, V (0 only for RT_UNPOL). vis:
 * nx*ny complex values [l + ny/2][k + nx/2] as (re, im) pairs of double (RT_FP64) or float,
 * host or device. A cuFFT transform of any size; synchronizes. */
int rt_image_visibilities(rt_ctx *ctx, const void *img, int form, int stokes, void *vis);

/* Launch shape of rt_render and rt_render_depths (forms RT_FP64, RT_MIXED, RT_UNPOL).
 * geo_blocks_per_sm and xfer_blocks_per_sm are the resident blocks per SM the geodesic and
 * transfer kernels are launched with (the grid is that times the SM count; 0 = automatic).
 * chunks >= 2 overlaps the two phases, so that the FP64 geodesic and the FP32 transfer share
 * the SMs, in one of two shapes:
 *   - streamed, in pieces of the rays that the workspace holds at once (1 when it holds every
 *     ray's path; up to 64; a library-owned workspace first grows to what 60% of the free
 *     device memory allows). The longest-first order is dealt to the pieces, and each piece's
 *     order is cut into `chunks` contiguous chunks. One geodesic launch traces a piece; each
 *     ray that stops counts toward its chunk, and the lane that completes a chunk raises a flag
 *     in mapped host memory. rt_render waits on the host for the flags and launches one
 *     transfer for each run of complete chunks on a second internal stream, beside the
 *     geodesic still running (after the geodesic has ended, at the transfer's full occupancy);
 *     a piece starts when the previous one has ended. The call occupies its host thread until
 *     the render ends.
 *   - in two halves of the workspace, when a piece would hold under 1/64 of the rays: the
 *     rays are dealt to the chunks, each chunk uses one half in turn, and
 *     the geodesic kernel of chunk i + 1 runs on one internal stream beside the transfer
 *     kernel of chunk i on another. last_chunk_div >= 2 shrinks the last chunk to
 *     1/last_chunk_div of a regular one (1 to 16; 0 = 1).
 * In both, the transfer runs with no more blocks per SM than fit in the register file beside
 * the geodesic's. chunks 1 runs the phases one after the other on the context's stream.
 * chunks 0 (the default, with {0, 0, 0, 0}) is automatic: RT_MIXED and RT_UNPOL images of 2^19
 * rays or more are overlapped, streamed in chunks of about 2^15 rays (at least 16 per piece)
 * with the geodesic at 2 blocks per SM, or in halves of 4 to 16 chunks of about 2^17 rays with
 * the geodesic at 1 block per SM; smaller images, and the RT_FP64 and RT_SURROGATE forms, run
 * one pass of each kernel. RT_SURROGATE overlaps when chunks >= 2 is set: streamed, each
 * transfer launch's rays go through the features pass, the network (over compact rows) and
 * the transfer in turn; in halves, per chunk (both measured slower than one pass on GB300).
 * Independently of the shape, a full render records each pixel's step count, and the next
 * render of the same camera and integrator takes its rays longest first, so that no launch ends
 * waiting for a few long photon-ring rays. The first render of a new camera of 2^18 rays or more
 * predicts the counts from a probe of one ray per 8 x 8 block; the next render rebuilds the
 * order from the counts the first one recorded. The image is the same in every shape and order
 * (every ray takes the same arithmetic); only the time differs. Shapes that exceed the
 * kernels' occupancy, chunks above 256 or last_chunk_div outside 0..16 return RT_ERR_INVALID. */
typedef struct {
    int geo_blocks_per_sm;
    int xfer_blocks_per_sm;
    int chunks;
    int last_chunk_div;
} rt_render_config;
int rt_set_render_config(rt_ctx *ctx, const rt_render_config *cfg);
int rt_get_render_config(rt_ctx *ctx, rt_render_config *cfg);

/* The grid fetch of the FP32 transfer (Section 2.1: the grid's primitives are interpolated at
 * every point of the geodesic): form RT_MIXED with thermal electrons on a grid model, in
 * rt_render, rt_render_depths and rt_render_adaptive. RT_FETCH_GATHER: each point reads the
 * eight cells of its trilinear stencil with plain loads. RT_FETCH_STAGED: while a lane works on
 * one saved state, the stencil of its next state is copied into the lane's slot of shared
 * memory by one TMA tensor load, completing on an mbarrier (every wait is bounded; one that
 * runs out makes the render return RT_ERR_STALL). The image is the same bit for bit either way;
 * only the time differs. RT_FETCH_AUTO (the default) takes the one measured faster on GB300 for
 * the benchmark image. Other forms and models always gather. Unknown modes: RT_ERR_INVALID. */
enum { RT_FETCH_AUTO = 0, RT_FETCH_GATHER = 1, RT_FETCH_STAGED = 2 };
int rt_set_grid_fetch(rt_ctx *ctx, int mode);
int rt_get_grid_fetch(rt_ctx *ctx, int *mode);

/* Counters of the last rt_render (synchronizes). */
int rt_last_counters(rt_ctx *ctx, rt_counters *out);

/* Timeline of the last overlapped render (synchronizes): for each of its chunks, four device
 * times in ms from the first geodesic launch's start, in out[4 * k .. 4 * k + 3]: geodesic
 * start, geodesic end, transfer start, transfer end (CUDA events on the two launching
 * streams). In the streamed shape (one geodesic launch for all the chunks of a piece) every
 * chunk reports its piece's launch's start and end, and the chunks that one transfer launch
 * covered report the same transfer start and end. out (host) holds `cap` chunks; *n receives the chunk count, of which
 * min(*n, cap) are written. An overlapped rt_render_batch (RT_BATCH_CHUNKS) has one too.
 * *n = 0 when the last render was not overlapped (one pass, a persistent batch, or
 * rt_render_static). For choosing a chunk count and launch shape. */
int rt_last_timeline(rt_ctx *ctx, float *out, int cap, int *n);

const char *rt_error_string(int code);

/* The device's measured FP64 FMA rate [TFLOP/s, an FMA counting 2]: independent FMA chains on
 * every SM, timed with CUDA events over five launches after a warm-up. A measurement helper
 * (the paper has no counterpart): the benchmark reports the geodesic's FP64 fraction against it
 * beside the nominal peak. Synchronizes the device. */
int rt_fp64_fma_peak(int device, double *tflops);

/* ---- Batched rendering (image libraries, MCMC fitting) -------------------------------------
 * Many images of different cameras and model parameters in one persistent launch, replayed
 * from a CUDA graph. All images share the loaded model (the GRMHD grid or the ADAF). A grid
 * image may override the mass unit and R_high. */
typedef struct {
    rt_camera cam;     /* resolution, inclination, frequency, ... of this image */
    double M_unit;     /* grid models: this image's mass unit [g]; <= 0 keeps the loaded value */
    double R_high;     /* grid models: this image's R_high; <= 0 keeps the loaded value */
    void *out_iquv;    /* device buffer, nx*ny*4 values of the form's type, layout as rt_render
                        * (RT_UNPOL: nx*ny floats of I) */
    uint8_t *status;   /* optional device nx*ny codes, or NULL */
    void *out_depth;   /* optional device nx*ny*2 depths (see rt_render_depths), or NULL */
} rt_job;

/* Launch shape of the batched form. mode 0 (RT_BATCH_PERSISTENT) is one persistent launch,
 * captured in a CUDA graph: each block has 8 warps, geo_warps of them integrate geodesics and
 * the rest run the transfer (odd-numbered blocks take geo_warps_odd instead when it is not 0,
 * so that the two roles can be balanced in steps of half a warp per block); step_tile is the number of RK4 steps a lane takes between its
 * queue and pool checks; blocks_per_sm is the number of resident blocks per SM (the grid is
 * that times the SM count). mode 1 (RT_BATCH_CHUNKS) treats the rays of all images as one ray
 * space and runs it like one large image in the automatic overlapped shape of
 * rt_set_render_config: streamed, in pieces of the ray space that the workspace holds (up to
 * 64), or, beyond that, in two workspace halves (chunks of about 2^17 rays, 2 to 64 of them, up
 * to 256 when the workspace is short; a batch that needs more runs in mode 0); on the
 * context's streams and without a graph; geo_warps, step_tile and blocks_per_sm are then
 * ignored. ms is the time the autotuner measured for this shape (0 when set by hand). */
typedef struct {
    int geo_warps;      /* 1..7 (mode 0) */
    int step_tile;      /* 1..16 (mode 0) */
    int blocks_per_sm;  /* 1..(the kernel's occupancy limit) (mode 0) */
    float ms;
    int mode;           /* RT_BATCH_PERSISTENT or RT_BATCH_CHUNKS */
    int geo_warps_odd;  /* 0 (as geo_warps) or 1..7: geodesic warps of odd-numbered blocks (mode 0) */
} rt_batch_config;
enum { RT_BATCH_PERSISTENT = 0, RT_BATCH_CHUNKS = 1 };

/* Render njobs images (form RT_FP64, RT_MIXED or RT_UNPOL; RT_UNPOL always in mode 1, with
 * out_iquv holding nx*ny floats of I and out_depth NULL): mode 0 in one persistent launch, where rays of all images share one work
 * queue and path blocks come from a bounded pool that the transfer frees as it walks, so memory
 * does not grow with the batch; the launch (with its set-up) is captured once into a CUDA graph
 * and replayed while the form, the image count and the total ray count stay the same. Mode 1
 * as described above. The first call for a form runs the autotuner (rt_batch_autotune, which
 * times both modes) on this batch unless a shape was set by hand, and so does a call whose
 * batch has over 4x more or 4x fewer rays than the tuned one. Results equal rt_render's for
 * each image. Synchronizes; RT_ERR_WORKSPACE if a ray had to be given up for lack of path
 * blocks (its pixel is zero, status RT_RAY_OVERFLOW); RT_ERR_STALL if a bounded wait ran out.
 * At most 2^31 - 1 rays in total. */
int rt_render_batch(rt_ctx *ctx, int form, const rt_job *jobs, int njobs);

/* Time the candidate launch shapes on a calibration batch (the leading images of `jobs`,
 * about 2^20 rays, rendered into their own buffers). Keep the fastest for `form`; return it in
 * *best (may be NULL). Synchronizes. */
int rt_batch_autotune(rt_ctx *ctx, int form, const rt_job *jobs, int njobs, rt_batch_config *best);
int rt_set_batch_config(rt_ctx *ctx, int form, const rt_batch_config *cfg);
int rt_get_batch_config(rt_ctx *ctx, int form, rt_batch_config *cfg);
/* Flow statistics of the last batch rendered as one persistent launch (mode 0): lane
 * iterations of the geodesic and the transfer warps' loops and, of those, the ones in which the
 * whole warp slept (no lane could step: waiting for path blocks, or for rays to be published);
 * polls of a ticket's ring slot that found no block yet, polls of a ready slot that found no
 * ray yet, polls of a busy slot when returning a block, and tickets taken. A measurement of the
 * persistent kernel's flow control (the paper has no counterpart). RT_ERR_NOT_READY before a
 * mode-0 batch. */
typedef struct {
    uint64_t geo_iters, geo_sleeps, xfer_iters, xfer_sleeps;
    uint64_t ticket_polls, ready_polls, free_spins, tickets;
} rt_batch_stats;
int rt_get_batch_stats(rt_ctx *ctx, rt_batch_stats *out);

/* rt_render without any device allocation, for callers that cannot allocate (their device
 * memory is budgeted by someone else, or allocation is forbidden on their code path). The
 * paper has no counterpart; it is a service of this library. The scratch (counters, ray
 * records, path arena) lives in one static 512 MiB device array that every GPU loading this
 * library holds until the process exits. The whole image is one chunk, so nx*ny must not
 * exceed rt_render_static_max_pixels() (13076 pixels, e.g. 114x114): larger images return
 * RT_ERR_SIZE. out_iquv (and status, if given) must be device memory, else RT_ERR_INVALID.
 * It renders the forms RT_FP64 and RT_MIXED (thermal or kappa electrons by quadrature); the
 * other forms (RT_UNPOL, RT_SURROGATE, whose network scratch it does not hold) return
 * RT_ERR_INVALID. It runs one pass of each kernel, at the blocks per SM that
 * rt_set_render_config sets (its chunk count does not apply). The first call on a device looks up the array's device address (cudaGetSymbolAddress),
 * so make that first call before any stream capture. Every call shares the one array and
 * clears its counters first; calls that overlap on the GPU (on different streams or from
 * several threads) race on it and must be serialized by the caller. Synchronizes the
 * context's stream like rt_render and fills the same counters (rt_last_counters). */
int rt_render_static(rt_ctx *ctx, int form, void *out_iquv, uint8_t *status);
long long rt_render_static_max_pixels(void);

#ifdef __cplusplus
}
#endif
#endif
