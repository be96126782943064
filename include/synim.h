/*
 * synim.h -- C ABI of the B300 (sm_103a) synthetic interaction-matrix library.
 *
 * The library computes Shack-Hartmann interaction matrices (IMs) from
 * deformable-mirror influence functions (IFs), following the method of the
 * paper's Sec. 2:
 *   - Sec. 2.1: the DM misregistration (shift, rotation, magnification), the
 *     sensor transform (rotation, anamorphic magnification, shift), the LGS
 *     cone factor (1 - h/H) and the off-axis footprint shift h * theta are
 *     folded into one composite affine map, and each IF is resampled exactly
 *     once (bilinear) onto the sensor grid;
 *   - Sec. 2.2: the sensor grid is M = k * n_sub pixels so that every
 *     subaperture is an exact k x k block; slopes are central differences
 *     averaged over the lit pixels of each subaperture, or, with the
 *     telescoping-sum engine (synim_opts.slope_engine), phase sums at the
 *     ends of the lit pixel runs;
 *   - Sec. 2.3: edge repair (strict core of the interpolated DM mask at
 *     0.999999, ring = cross dilation minus core, ring value = mean over the
 *     valid cardinal directions of 2 P1 - P2 or P1);
 *   - Sec. 4.2: many DMs x many sensors in one pass, each IF fetched once.
 *
 * Conventions (all calls):
 *   - Images are row-major, row = y, column = x; pixel centres sit at integer
 *     indices and each grid is centred at (n - 1) / 2.
 *   - The IM of pair (dm, wfs) is FP32, column-major: column a (actuator a of
 *     the DM, cube order) is contiguous and holds 2 * nv rows: the x slopes of
 *     the nv valid subapertures (row-major subaperture order), then their y
 *     slopes.  Memory size = n_act * 2 * nv * 4 bytes.
 *   - Slopes are in IF units per metre of the sensor's pupil-plane frame,
 *     times slope_scale.
 *   - Positive DM shift moves the DM pattern towards +x / +y on the sensor;
 *     positive rotation turns it from +x towards +y; mag > 1 enlarges it.
 *   - Every call returns a synim_status; nothing aborts or throws across the
 *     ABI.  Device work is ordered on the caller's CUDA stream (cudaStream_t
 *     passed as void*; NULL = legacy default stream).  A context belongs to
 *     the device that was current at create and is not thread-safe.
 *   - Output buffers are allocated by the caller (sizes from synim_im_query)
 *     and must stay valid until the stream has executed the call.
 */
#ifndef SYNIM_H
#define SYNIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SYNIM_OK = 0,
    SYNIM_ERR_INVALID_ARG = 1, /* NULL pointer, negative size, bad enum */
    SYNIM_ERR_SHAPE = 2,       /* inconsistent sizes (e.g. grid_m % n_sub != 0, k < 2) */
    SYNIM_ERR_OOM = 3,         /* a device allocation failed */
    SYNIM_ERR_CUDA = 4,        /* a CUDA runtime call failed (see synim_last_error) */
    SYNIM_ERR_TIMEOUT = 5,     /* a bounded device wait gave up (kernel returned early) */
    SYNIM_ERR_NOT_CONVERGED = 6,
    SYNIM_ERR_NOT_TRAINED = 7,
    SYNIM_ERR_BOUNDS = 8       /* bounds-checked build only: an IM kernel index left its buffer;
                                  the access was skipped (see synim_debug_bounds) */
} synim_status;

typedef struct synim_ctx synim_ctx;

/* One deformable mirror (or virtual layer).  Sec. 2.1, Sec. 4.1. */
typedef struct {
    int32_t n_act;          /* number of IFs = IM columns, >= 1 */
    int32_t grid_n;         /* N: every IF is N x N FP32, N >= 4 */
    double pixel_pitch_m;   /* DM-plane pixel size in metres, > 0 */
    double altitude_m;      /* conjugation altitude h, >= 0 */
    const float *ifs;       /* [n_act][N][N]; borrowed for the duration of create only */
    int32_t ifs_on_device;  /* 1: ifs is a device pointer on the current device; 0: host */
    const uint8_t *mask;    /* host [N][N] 0/1 DM mask (IFs are assumed already masked);
                               NULL = all ones */
    float support_eps;      /* |IF| <= support_eps * (largest |IF| of this DM) is treated as
                               zero outside each actuator's support window; 0 = keep the
                               whole grid */
} synim_dm_desc;

/* One Shack-Hartmann sensor.  Sec. 2.1 (sensor transform), Sec. 2.2 (grid). */
typedef struct {
    int32_t n_sub;              /* subapertures per side, >= 1 */
    int32_t grid_m;             /* M = k * n_sub with k >= 2 */
    double pupil_diam_m;        /* D: the M x M grid spans D (pixel = D / M) */
    double src_height_m;        /* guide-star height H; 0 (or inf) = natural guide star */
    double field_rad[2];        /* guide-star direction (x, y) in radians */
    double rot_deg;             /* sensor rotation */
    double mag[2];              /* sensor magnification (x, y): anamorphosis */
    double shift_m[2];          /* sensor shift in the pupil plane, metres */
    const uint8_t *pupil_mask;  /* host [M][M] 0/1; NULL = annulus of inner radius
                                   obstruction * M / 2 and outer radius M / 2 (pixel units) */
    const uint8_t *subap_valid; /* host [n_sub][n_sub] 0/1; NULL = valid when at least half
                                   of the k x k pixels are lit */
    double obstruction;         /* used only when pupil_mask is NULL */
    double slope_scale;         /* multiplies every slope (1 = IF units per metre) */
} synim_wfs_desc;

/* DM misregistration relative to one sensor (Sec. 5: the SPRINT parameters). */
typedef struct {
    double shift_x_px; /* DM pixels */
    double shift_y_px; /* DM pixels */
    double rot_deg;    /* degrees */
    double mag;        /* dimensionless, 1 = nominal */
} synim_misreg;

/* Creation options; pass NULL for defaults. */
typedef struct {
    int32_t threads_per_cta; /* 0 = default (256); a multiple of 32 in 64..256 */
    int32_t ctas_per_sm;     /* reserved, 0 (every column is one warp of one launch) */
    int32_t use_graph;       /* 1 = replay a CUDA graph per stream (interaction matrices) and
                                per small estimator batch; 0 = plain launches */
    int32_t autotune;        /* 1 = at the first call of each mode, time the candidate launch
                                shapes (128 or 256 threads x 2, 4 or 8 lanes per boundary
                                segment; telescoping engine: x 1/2, 1, 2 or 4 times the
                                default lanes per subaperture) on that call's inputs and
                                keep the fastest */
    int32_t profile;         /* 1 = record CUDA events around every IM-kernel launch
                                (read back with synim_im_kernel_ms) */
    int64_t device_mem_cap;  /* bytes of device memory create may take (the context's
                                holdings plus the temporary cube staging); 0 = no cap.
                                Exceeding it fails create with SYNIM_ERR_OOM */
    int32_t slope_engine;    /* SYNIM_ENGINE_NUMERICAL (0, default): central-difference slopes
                                with edge repair (Sec. 2.2-2.3).  SYNIM_ENGINE_TELESCOPING (1):
                                the telescoping sum of Sec. 2.2, read as the gradient tilt over
                                each valid subaperture's lit area,
                                  s_x = slope_scale * sum_edges sign * phi(edge) / (dw * n_lit),
                                over the half-pixel ends of every lit pixel run along x
                                (sign -1 at the start, +1 at the end; y likewise along
                                pixel columns), phi resampled at the edge point with no edge
                                repair.  Sensor grids up to 8191 pixels.  With engine 1 only
                                synim_im_compute is available (sensitivity and vjp return
                                SYNIM_ERR_INVALID_ARG) */
} synim_opts;

#define SYNIM_ENGINE_NUMERICAL 0
#define SYNIM_ENGINE_TELESCOPING 1

/*
 * Create a context: uploads the IF cubes once, scans each IF's support
 * window (|IF| > support_eps * the DM's largest |IF|), packs the windows into device memory,
 * and builds the per-sensor subaperture tables (Sec. 2.2) and derivative
 * stencils.  The caller may free every input as soon as create returns.
 * dms[n_dm], wfs[n_wfs]: 1 <= n_dm <= 16, 1 <= n_wfs <= 16.
 * On success *out owns device memory until synim_im_destroy.
 */
synim_status synim_im_create(const synim_dm_desc *dms, int32_t n_dm, const synim_wfs_desc *wfs,
                             int32_t n_wfs, const synim_opts *opts, synim_ctx **out);

/* IM shape of pair (dm, wfs): n_rows = 2 * nv, n_cols = n_act. */
synim_status synim_im_query(const synim_ctx *ctx, int32_t dm, int32_t wfs, int64_t *n_rows,
                            int64_t *n_cols);

/* Side W of the square support window of DM dm's influence functions, in DM
 * pixels (every window of that DM has this size; Sec. 4.2 staging unit). */
synim_status synim_dm_window(const synim_ctx *ctx, int32_t dm, int32_t *W);

/*
 * The composite affine of pair (dm, wfs) under misregistration mis (Sec. 2.1):
 * DM pixel (x, y) sampled by sensor pixel (row i, column j) is
 *   x = A[0] j + A[1] i + b[0],  y = A[2] j + A[3] i + b[1].
 * Host-only; A[4], b[2] are host buffers.
 */
synim_status synim_pair_affine(const synim_ctx *ctx, int32_t dm, int32_t wfs,
                               const synim_misreg *mis, double *A, double *b);

/*
 * Compute every IM of the context in one launch (Sec. 2.1-2.3, Sec. 4.2):
 * one warp per (actuator, sensor) column over a grid-stride loop.  mis[n_dm * n_wfs] (host) holds one misregistration per pair,
 * pair index = dm * n_wfs + wfs; im[n_dm * n_wfs] (host array) holds device
 * pointers to the caller's FP32 output buffers (layout above); a NULL entry
 * skips that pair.  Asynchronous on cuda_stream.  With the numerical slope
 * engine, the call's per-pair pixel classes and weight boxes are built on a
 * stream the context owns, ordered before the IM launch on cuda_stream; the
 * context alternates two sets of these tables, so the next call's tables are
 * built while this call's IM kernel runs.  One host thread at a time per
 * context.
 */
synim_status synim_im_compute(synim_ctx *ctx, const synim_misreg *mis, float *const *im,
                              void *cuda_stream);

/*
 * IM and its tangents with respect to the four misregistration parameters
 * p = (shift_x_px, shift_y_px, rot_deg, mag) of every pair, in one pass
 * (forward-mode derivative of Sec. 2.1-2.3 with the edge-repair core set held
 * fixed; the bilinear derivative is that of the floor cell).
 * im[n_pairs] (may be NULL, or hold NULL entries) receives the IMs;
 * d_im[4 * n_pairs] holds device pointers, d_im[4 p + k] = dIM_p / dp_k
 * (same layout as the IM; NULL entries are skipped).  Asynchronous.
 */
synim_status synim_im_sensitivity(synim_ctx *ctx, const synim_misreg *mis, float *const *im,
                                  float *const *d_im, void *cuda_stream);

/*
 * Vector-Jacobian product of the IMs: grad_p[4 p + k] = sum over the IM of
 * pair p of grad_im[p] * dIM_p / dp_k, without forming the tangents (the
 * adjoint of synim_im_sensitivity).  grad_im[n_pairs]: device pointers (NULL
 * = zero cotangent); grad_p: host [4 * n_pairs] doubles, written when the call
 * returns (it synchronises cuda_stream).
 */
synim_status synim_im_vjp(synim_ctx *ctx, const synim_misreg *mis, const float *const *grad_im,
                          double *grad_p, void *cuda_stream);

/* 1 if the library was built with -DSYNIM_DEBUG_BOUNDS: every global and
 * shared-memory index of the IM kernels (k_im, k_tele) is tested against
 * its buffer; an index outside skips the access and makes the next
 * synim_im_check (or the no-allocation entry point) return
 * SYNIM_ERR_BOUNDS.  0 for the release build. */
int32_t synim_debug_bounds(void);

/*
 * Synchronise cuda_stream and report whether any kernel of this context has
 * flagged an error since the last check (SYNIM_ERR_TIMEOUT if a bounded wait
 * gave up).  Clears the flag.
 */
synim_status synim_im_check(synim_ctx *ctx, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Tomographic projection (Sec. 2.5, tomographic projection matrices).
 *
 * The components of a context (its DMs and virtual layers) are seen from
 * n_dir optimisation directions dirs_rad[j] = (theta_x, theta_y) by a
 * source at infinity, on the pupil grid of sensor `wfs` (M x M, its pupil
 * mask) binned bin x bin (M % bin == 0).  Entry (row, column) of a
 * projection matrix P_X is the mean over the bin x bin fine pixels of the
 * binned pixel of P(p) * bilinear(IF_a; A_j (p_col, p_row) + b_j), where:
 *   - the columns are the actuators of the listed components, in order;
 *   - the rows are direction-major, row = j (M / bin)^2 + binned pixel
 *     (row-major);
 *   - (A_j, b_j) is the composite affine with the direction's field angle,
 *     no cone, no sensor rotation, magnification or shift, and no
 *     misregistration (footprint shift h theta_j);
 *   - there is no edge repair.
 * ---------------------------------------------------------------------- */

/* Rows of the projection matrices: n_dir (M / bin)^2. */
synim_status synim_projection_rows(const synim_ctx *ctx, int32_t wfs, int32_t n_dir, int32_t bin, int64_t *rows);

/* P_X of components comps[n_comp] into P (device, FP32, column-major
 * [n_cols][rows]: each actuator's column contiguous).  Synchronises the
 * stream before returning. */
synim_status synim_projection_matrix(synim_ctx *ctx, int32_t wfs, int32_t n_dir, const double *dirs_rad, int32_t bin,
                                     int32_t n_comp, const int32_t *comps, float *P, void *cuda_stream);

/* P_opt = (P_DM^T P_DM + lambda I)^{-1} P_DM^T P_Layer for DM components
 * dms[n_dm] and layer components layers[n_layer] (lambda >= 0, absolute):
 * p_opt (device, FP32, column-major [n_layer_cols][n_dm_cols], i.e. column l
 * holds the DM commands of layer mode l).  Stores both projection matrices
 * box by box in device scratch (each column is non-zero only on its footprint
 * box per direction), forms P_DM^T P_DM and P_DM^T P_Layer from the box
 * intersections (FP32), factors by a blocked Cholesky and solves with two
 * block triangular sweeps, every block update a tensor-core GEMM with
 * FP32-level accuracy (synim_linalg_gemm).
 * Synchronises the stream before returning.  SYNIM_ERR_NOT_CONVERGED if the
 * normal matrix is not positive definite. */
synim_status synim_projection_opt(synim_ctx *ctx, int32_t wfs, int32_t n_dir, const double *dirs_rad, int32_t bin,
                                  int32_t n_dm, const int32_t *dms, int32_t n_layer, const int32_t *layers,
                                  double lambda, float *p_opt, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Dense linear algebra of the tomographic operators (Sec. 2.4, Sec. 2.5)
 *
 * The projection P_opt and the MMSE reconstructor are dense contractions and
 * symmetric positive definite solves.  The library runs them on the tensor
 * cores (tcgen05, TF32 inputs) with every operand split into a TF32 part and
 * its FP32 remainder and three products accumulated in FP32 (hi.hi + hi.lo +
 * lo.hi), about 2^-21 relative error per product: FP32-level accuracy.
 * Matrices are row-major FP32 device arrays with a leading dimension (in
 * elements).  These calls need no context; errors are reported through
 * synim_last_error(NULL).  They enqueue on cuda_stream and synchronise it
 * before returning.
 * ---------------------------------------------------------------------- */

/* C = beta C + alpha A B.  A is M x K (lda); B is N x K (b_kn = 0: element
 * (k, n) at B[n ldb + k]) or K x N (b_kn = 1: B[k ldb + n]); C is M x N (ldc).
 * M, N, K >= 0.  SYNIM_ERR_TIMEOUT if a bounded tensor-core wait gave up. */
synim_status synim_linalg_gemm(int32_t M, int32_t N, int32_t K, float alpha, const float *A, int64_t lda,
                               const float *B, int64_t ldb, int32_t b_kn, float beta, float *C, int64_t ldc,
                               void *cuda_stream);

/* Y <- Y S^-1 for a symmetric positive definite S (n x n, lds): S is
 * overwritten by its Cholesky factor L (lower triangle, S = L L^T, blocked
 * right-looking, 128-row blocks); Y is m x n (ldy).  Allocates its scratch
 * (the factor's diagonal-block inverses and one panel).  SYNIM_ERR_NOT_CONVERGED
 * if S is not positive definite. */
synim_status synim_linalg_spd_solve(float *S, int32_t n, int64_t lds, float *Y, int32_t m, int64_t ldy,
                                    void *cuda_stream);

/* ------------------------------------------------------------------------
 * Tomographic covariances and the MMSE reconstructor (Sec. 2.4)
 *
 * The paper names the models without formulas; the readings are:
 *   - von Karman phase covariance of a layer (phase in radians at the
 *     wavelength r0 refers to), x = 2 pi r / L0:
 *       B(r) = c (L0 / r0)^(5/3) x^(5/6) K_5/6(x),
 *       c = Gamma(11/6) / (2^(5/6) pi^(8/3)) (24/5 Gamma(6/5))^(5/6);
 *     a layer holding the fraction f of the C_n^2 profile has r0 f^(-3/5);
 *   - projected onto the DM's basis: F = the influence functions averaged
 *     over bin x bin pixel blocks, C_atm = G^-1 F^T C_phi F G^-1 with
 *     G = F^T F (covariance of the least-squares coefficients);
 *   - Shack-Hartmann centroid noise (photon and read-out terms) per valid
 *     subaperture, with the LGS spot elongated along the direction from the
 *     launch telescope;
 *   - R = C_atm D^T (D C_atm D^T + C_n)^-1, D^T being the IM.
 * Outputs are row-major FP32 device matrices; the calls synchronise the
 * stream before returning.
 * ---------------------------------------------------------------------- */

/* Detector and guide-star parameters of one sensor's noise covariance. */
typedef struct {
    double n_photons;       /* photons per subaperture per frame, > 0 */
    double ron_e;           /* read-out noise, electrons rms per pixel, >= 0 */
    double pixel_scale_rad; /* detector pixel, radians on the sky, > 0 */
    int32_t n_pix;          /* centroiding window width, pixels, >= 1 */
    int32_t lgs;            /* 1 = laser guide star (spot elongation), 0 = natural */
    double fwhm_rad;        /* spot FWHM without elongation, radians, > 0 */
    double wavelength_m;    /* sensing wavelength, > 0 */
    double llt_xy_m[2];     /* launch telescope position in the pupil plane (LGS) */
    double na_altitude_m;   /* sodium layer altitude above the telescope (LGS), > 0 */
    double na_thickness_m;  /* sodium layer thickness (LGS), >= 0 */
    double zenith_rad;      /* zenith angle (LGS): both lengths scale by 1 / cos */
} synim_noise_desc;

/* C_atm [n_act][n_act] of DM dm's basis for a von Karman layer of Fried
 * parameter r0_m and outer scale L0_m, on the DM grid binned by bin (grid_n
 * a multiple of bin, at most 46340 binned pixels).  The FP32 result carries
 * about cond(G)^2 2^-24 relative error: choose bin so that each influence
 * function spans at least two binned pixels (cond(G) grows fast as the
 * binned basis functions shrink below that; SYNIM_ERR_NOT_CONVERGED if G is
 * singular, as it is whenever some influence function vanishes on the grid,
 * e.g. actuators masked out by the DM mask: leave those out of the basis).
 * Allocates scratch of (grid_n / bin)^4 floats plus a few n_act^2. */
synim_status synim_atm_covariance(synim_ctx *ctx, int32_t dm, int32_t bin, double r0_m, double L0_m,
                                  float *c_atm, void *cuda_stream);

/* C_n [2 nv][2 nv] of sensor wfs (rows as the IM's: x slopes then y slopes of
 * the valid subapertures), in the IM's slope units (radians of phase per
 * metre times slope_scale). */
synim_status synim_noise_covariance(synim_ctx *ctx, int32_t wfs, const synim_noise_desc *nd, float *c_noise,
                                    void *cuda_stream);

/* R [n_modes][n_slopes] = C_atm D^T (D C_atm D^T + C_n)^-1 for im = D^T
 * [n_modes][n_slopes], c_atm [n_modes][n_modes], c_noise [n_slopes][n_slopes].
 * Context-free (errors through synim_last_error(NULL)). */
synim_status synim_mmse_reconstructor(int32_t n_modes, int32_t n_slopes, const float *im, const float *c_atm,
                                      const float *c_noise, float *R, void *cuda_stream);

/*
 * Self-test of the bounded device waits (the mbarrier waits of the
 * tensor-core kernels use the same helper): one thread waits on an mbarrier
 * that nothing arrives at, gives up after limit_clocks SM clocks (clamped to
 * 1 .. 2^31), raises the context's error flag and returns; the call then
 * synchronises `cuda_stream` and reports the flag like synim_im_check.
 * Expected result: SYNIM_ERR_TIMEOUT, with the context still usable.
 */
synim_status synim_wait_selftest(synim_ctx *ctx, int64_t limit_clocks, void *cuda_stream);

/*
 * With opts.profile = 1: wait for the IM-kernel launches recorded since the
 * previous call and return their summed device time (ms) and count.  Up to
 * 256 launches are kept between two calls (older ones are dropped from the
 * sum and the count).  Returns SYNIM_ERR_INVALID_ARG without profiling.
 */
synim_status synim_im_kernel_ms(synim_ctx *ctx, double *total_ms, int32_t *n_launches);

/* ------------------------------------------------------------------------
 * Probe responses.  The paper's Sec. 5 drives the IM generator from online
 * estimates of slowly drifting misregistrations; the estimators of this
 * library (below) read the misregistration of one (DM, sensor) pair from the
 * sensor's response to a few probe commands.  A probe mode m is the DM shape
 * S_m = sum_a cmd[m][a] IF_a; its response is the slope vector that the
 * method of Sec. 2.1-2.3 gives for S_m.  For a fixed edge-repair core set
 * every step is linear, so the response equals cmd[m] . IM.
 *
 * Slope maps: [n_sub][n_sub][C] FP32 (or bfloat16), C = 2 n_modes, channel
 * 2 m = x slope of mode m, 2 m + 1 = its y slope; invalid subapertures hold 0.
 * A sample's parameters are a synim_misreg as 4 doubles
 * (shift_x_px, shift_y_px, rot_deg, mag) and replace the pair's
 * misregistration.
 * ---------------------------------------------------------------------- */

/*
 * Attach probe modes to pair (dm, wfs): cmd is host [n_modes][n_act] doubles
 * (mode m's command on actuator a, cube order), 1 <= n_modes <= 32.  Forms
 * the modal screens once on the device from the packed supports (FP64 sums,
 * stored FP32 [N + 2][N + 2][modes rounded up to 4], zero border).  The
 * per-row working tile needs 4 (k + 2)(k + 2) (n_modes rounded up to 4) bytes
 * of shared memory for tangents x 5; sensors whose k makes even one
 * subaperture too large are refused (SYNIM_ERR_SHAPE).  Replaces a previous
 * attachment; synchronous.
 */
synim_status synim_probe_attach(synim_ctx *ctx, int32_t dm, int32_t wfs, const double *cmd,
                                int32_t n_modes);

/* Map shape of the attached probes; valid (host [n_sub][n_sub], may be NULL)
 * receives 1 for valid subapertures. */
synim_status synim_probe_query(const synim_ctx *ctx, int32_t *n_sub, int32_t *n_channels,
                               uint8_t *valid);

/*
 * Clean probe responses of n samples.  params: device [n][4] doubles.
 * maps: device [n][n_sub][n_sub][C] FP32.  d_maps: NULL, or device
 * [4][n][n_sub][n_sub][C] FP32 tangents with respect to the four parameters
 * (core set held fixed, floor-cell bilinear derivative, as
 * synim_im_sensitivity).  Asynchronous on cuda_stream.
 */
synim_status synim_probe_response(synim_ctx *ctx, const double *params, int64_t n, float *maps,
                                  float *d_maps, void *cuda_stream);

/*
 * Noisy bfloat16 probe inputs (training data of the learned estimator).
 * Sample q gets its clean maps plus Gaussian noise of standard deviation
 * noise_rel x (largest |slope| of its maps) on valid subapertures (invalid
 * ones stay 0), rounded to the nearest bfloat16 (ties to even).  Noise of
 * element e of the sample's maps: Philox4x32-10 (Salmon et al., SC 2011)
 * under key (seed low, seed high) at counter (e / 4, s low, s high, 0),
 * s = sample0 + q; words (2t, 2t + 1), t = (e mod 4) / 2, give
 * u1 = (w + 1) 2^-32 and u2 = w' 2^-32, and the Box-Muller transform gives
 * sqrt(-2 ln u1) cos(2 pi u2) for even e, sqrt(-2 ln u1) sin(2 pi u2) for
 * odd e.  params: device [n][4]; out: device [n][n_sub][n_sub][C] bfloat16
 * bits.  Asynchronous; works in batches with context-owned scratch.
 */
synim_status synim_probe_generate(synim_ctx *ctx, const double *params, int64_t n, uint64_t seed,
                                  uint64_t sample0, float noise_rel, uint16_t *out,
                                  void *cuda_stream);

/*
 * Misregistration of the probed pair from measured probe responses.
 *   probe_slopes: device [n][n_sub][n_sub][C] FP32 slope maps (layout above).
 *   method: 0 = Gauss-Newton fit from the initial guesses in inout;
 *           1 = the network alone (synim_cnn_init, then synim_cnn_train or
 *               trained parameters);
 *           2 = the network's estimate refined by the fit.
 *   inout: host [n]: initial guesses (method 0; ignored otherwise), then the
 *          estimates.
 *   residual_out: host [n] or NULL: ||y - s(p)|| / ||y|| at the estimate, with
 *          s regenerated by Sec. 2.1-2.3 (the check on the estimate).
 * Fit: r = y - s(p) over all map entries, Jacobian J from the probe tangents,
 * step (J^T J + mu diag(J^T J)) dp = J^T r solved in FP64 (Cholesky); mu = 0
 * at first, x10 when the cost rises (the step is rejected), /10 after an
 * accepted step; stops when an accepted step, divided component-wise by
 * the scale (default 8 px, 8 px, 2 deg, 0.02), has norm below tol (default
 * 1e-4), or after max_iter steps (default 30).  The cost is only piecewise
 * smooth (bilinear cells, core changes), so the step test stops at a step
 * size well below the estimate's noise rather than at rounding level.  An
 * initial guess should not put the sensor grid exactly on the DM grid (the
 * identity when N = M): there every sample lies on a cell line and the
 * floor-cell Jacobian is one-sided.  SYNIM_ERR_NOT_TRAINED for methods 1-2
 * without a network.  Synchronous.
 * Small batches (n <= 32) of method 1, and of method 2 with max_iter <= 4,
 * run as one CUDA graph per (method, n, max_iter, residual wanted), captured
 * at the first such call (unless the context was created with use_graph =
 * 0): the network, the residual or the max_iter + 1 fit passes, and the
 * readback, with one synchronisation per call.  The results are those of the
 * plain launches with the same batch size.  A later probe attach, network
 * init or fit setting recaptures.
 */
synim_status synim_misreg_estimate(synim_ctx *ctx, const float *probe_slopes, int64_t n, int32_t method,
                                   synim_misreg *inout, double *residual_out, void *cuda_stream);

/* Fit settings: max_iter in 1..1000, tol > 0, scale (4 positive doubles) or NULL to keep. */
synim_status synim_gn_config(synim_ctx *ctx, int32_t max_iter, double tol, const double *scale);

/* Steps taken and convergence flag (1 = stopped on the step test) of each
 * sample of the last synim_misreg_estimate; host [n] each, either may be NULL. */
synim_status synim_misreg_estimate_stats(const synim_ctx *ctx, int32_t *iters, int32_t *converged);

/* ------------------------------------------------------------------------
 * The learned estimator: a small BF16 convolutional network (tensor cores,
 * FP32 accumulation) on the probe slope maps, trained on the GPU on probe
 * responses the library generates.  Layers: conv 3x3 stride 1 (C -> 64),
 * conv 3x3 stride 2 (64 -> 64), conv 3x3 stride 2 (64 -> 64), each with
 * bias and ReLU, then a dense layer from the flattened H3 x H3 x 64 map
 * (H3 = side after the two stride-2 layers, 10 for 40x40 maps) to 4 outputs.  Output: the
 * misregistration normalised as (p - center) / range per component.
 * Parameters (FP32, this order): W1 [64][3][3][C], b1 [64], W2 [64][3][3][64],
 * b2, W3 [64][3][3][64], b3, Wfc [4][H3][H3][64], bfc [4]; C = 2 n_modes must be a
 * multiple of 32.
 * ---------------------------------------------------------------------- */

/* Number of parameters for n_sub x n_sub maps with n_channels channels. */
int32_t synim_cnn_n_params(int32_t n_sub, int32_t n_channels);

/* Create the network of the attached probes with initial parameters (host
 * [n_params]) and normalisation norm = {center[4], range[4]} (host). */
synim_status synim_cnn_init(synim_ctx *ctx, const float *params, const double *norm);

/* Copy the current parameters (host [n_params]) and normalisation (host [8]); either may be NULL. */
synim_status synim_cnn_get(const synim_ctx *ctx, float *params, double *norm);

/* Normalised outputs (device [n][4] FP32) for bfloat16 maps x (device [n][n_sub][n_sub][C],
 * 16-byte aligned: the first layer reads it through a TMA tensor map; SYNIM_ERR_INVALID_ARG
 * otherwise). */
synim_status synim_cnn_forward(synim_ctx *ctx, const uint16_t *x, int64_t n, float *out, void *cuda_stream);

/* One forward and backward pass without an update, 1 <= n <= 256 (x 16-byte aligned, as
 * for synim_cnn_forward): loss_out
 * (host, may be NULL) = mean squared error over the n x 4 outputs against
 * target (device [n][4], normalised); grad_out (host [n_params], may be
 * NULL) = its gradient.  Synchronous. */
synim_status synim_cnn_grad(synim_ctx *ctx, const uint16_t *x, const float *target, int64_t n,
                            double *loss_out, float *grad_out, void *cuda_stream);

typedef struct {
    int32_t epochs, batch;   /* batch <= 256 */
    float lr, lr_final;      /* Adam step, decayed geometrically to lr_final (0 = constant) */
    float beta1, beta2, eps; /* 0 = defaults 0.9, 0.999, 1e-8 */
    float noise_rel;         /* probe noise, as synim_probe_generate */
    uint64_t seed, sample0;  /* noise stream and shuffling seed, first sample index */
} synim_train_opts;

/* Train on n samples with misregistrations params (device [n][4]): the
 * library generates one noisy bfloat16 probe response per sample
 * (synim_probe_generate), then runs opts->epochs epochs of shuffled
 * minibatches (std::mt19937_64 permutation seeded from opts->seed) with Adam
 * on the mean squared error of the normalised outputs.  loss_out (host
 * [epochs], may be NULL): the loss of the last batch of each epoch.  Keeps
 * the generated inputs (n x n_sub^2 x C x 2 bytes of device memory).
 * Synchronous. */
synim_status synim_cnn_train(synim_ctx *ctx, const double *params, int64_t n, const synim_train_opts *opts,
                             double *loss_out, void *cuda_stream);

/*
 * Checkpoint / resume of the network and its optimiser.  Layout (little-
 * endian): a 128-byte header {char magic[8] = "SYNIMCNN"; uint32 version =
 * 1; int32 n_sub, channels, step (Adam steps taken); int64 n_params; double
 * center[4], range[4]; zero padding}, then FP32 parameters, Adam first
 * moments and Adam second moments, [n_params] each.
 * save: *bytes = the checkpoint's size; with buf (host, cap bytes) also
 * writes it there (SYNIM_ERR_INVALID_ARG if cap is smaller).  Synchronous.
 * load: replaces the context's network with the checkpoint's (as
 * synim_cnn_init, then the moments and the step count), so that a training
 * run resumed from a checkpoint continues exactly as the uninterrupted one.
 * SYNIM_ERR_INVALID_ARG for a foreign or truncated buffer; SYNIM_ERR_SHAPE
 * if its map shape differs from the attached probes'.  Synchronous.
 */
synim_status synim_cnn_save(const synim_ctx *ctx, void *buf, int64_t cap, int64_t *bytes);
synim_status synim_cnn_load(synim_ctx *ctx, const void *buf, int64_t bytes);

/* Launch shape chosen by the autotuner for mode 0 (IM), 1 (tangents) or 2
 * (adjoint): threads per CTA, lanes per boundary segment (telescoping
 * engine: lanes per subaperture on sensor 0), and the mean kernel time of
 * the winner (ms).  SYNIM_ERR_NOT_CONVERGED (outputs hold the defaults)
 * while that mode has not been tuned. */
synim_status synim_im_tuning(const synim_ctx *ctx, int32_t mode, int32_t *threads, int32_t *seg_lanes,
                             double *ms);

/* Free all device memory of the context (waits for its streams). NULL is a no-op. */
void synim_im_destroy(synim_ctx *ctx);

/*
 * IM of one (DM, sensor) pair without allocating any memory.  The paper has
 * no counterpart: this entry point exists for callers that must not allocate
 * device memory while they run -- a real-time controller whose GPU memory is
 * reserved once at start-up, or a host framework whose pooled allocator owns
 * all device memory so that a direct cudaMalloc would fail or fragment it.
 * It calls no cudaMalloc / cudaFree (nor any allocating library routine) and
 * uses no host heap; all intermediates live in one fixed device array of
 * SYNIM_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits.
 *   dm:     dm->ifs must be a DEVICE pointer (ifs_on_device = 1), cube
 *           [n_act][N][N] FP32; dm->mask is a host pointer or NULL.
 *   wfs:    as for synim_im_create (host mask pointers).
 *   mis:    the pair's misregistration (host).
 *   im:     device output [n_act][2 nv] FP32 (column-major IM, layout above),
 *           or NULL to only return the row count.
 *   n_rows: if not NULL, receives 2 nv.
 * Same results as synim_im_compute for the same pair.  The call synchronises
 * cuda_stream and returns when the IM is written.  Inputs whose support
 * windows, sensor tables and pixel maps do not fit the fixed array are
 * rejected with SYNIM_ERR_SHAPE (message in synim_last_error(NULL)); the
 * tables alone take about 8 M^2 + 30 n_act bytes, the windows
 * 4 n_act (W + 3)^2 bytes for support side W.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * Every call shares the array and it keeps the previous call's contents:
 * the call clears what must start at zero, but calls whose GPU work overlaps
 * (other host threads or streams) race on it and must be serialised.
 */
#define SYNIM_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)
synim_status synim_im_compute_noalloc(const synim_dm_desc *dm, const synim_wfs_desc *wfs,
                                      const synim_misreg *mis, float *im, int64_t *n_rows,
                                      void *cuda_stream);

/* Static description of a status code. */
const char *synim_status_string(synim_status s);

/* Last error message recorded on ctx ("" if none); valid until the next call on ctx.
 * With ctx == NULL: the last error of a failed synim_im_create or
 * synim_im_compute_noalloc on this thread. */
const char *synim_last_error(const synim_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SYNIM_H */
