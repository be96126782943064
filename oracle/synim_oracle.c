/*
 * synim_oracle.c -- plain FP64 CPU oracle for synthetic interaction matrices.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only through the
 * seeded inputs of the workload generator.
 *
 * Everything is computed in double precision, one WFS pixel at a time, over
 * the whole M x M sensor grid for every actuator (no support windows, no
 * tiling, no fusion).  Each step follows the paper:
 *   - composite affine transform (Sec. 2.1): DM and WFS shifts, rotations,
 *     magnifications, the LGS cone and the off-axis footprint shift are
 *     multiplied into one matrix and the influence function is resampled
 *     exactly once by bilinear interpolation;
 *   - absolute sub-pixel grid alignment (Sec. 2.2): the sensor grid is
 *     M = k * n_sub pixels, so each subaperture is an exact k x k block;
 *   - edge repair (Sec. 2.3, three steps): strict binarisation of the
 *     interpolated mask at 0.999999, identification of the dilated ring,
 *     omnidirectional extrapolation 2 P1 - P2 (or P1) averaged over the
 *     valid cardinal directions;
 *   - numerical derivative (Sec. 2.2): central differences at every pixel,
 *     masked by the sensor pupil and averaged over each subaperture.
 *
 * Readings where the paper is silent (listed in the design notes):
 *   - pixel centres at integer indices, both grids centred at (n-1)/2;
 *   - bilinear samples outside [0, N-1] are zero; the cell is floor(x);
 *   - the dilation is the 4-connected cross; P1 is the adjacent pixel;
 *   - the derivative is (phi[j+1] - phi[j-1]) / (2 dw) with phi = 0 outside
 *     the sensor grid; the slope is the mean over illuminated pixels;
 *   - a subaperture is valid when at least half of its pixels are lit.
 *
 * Parity: every public function here is pinned by tests against closed forms
 * (tilt, quadratic), invariants (90-degree rotation, magnification,
 * linearity), the exact telescoping identity of summed central differences,
 * the continuous gradient at low spatial frequency, hand-worked edge-repair
 * cases and central finite differences for the tangents.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNOR_CORE_THRESHOLD 0.999999 /* Sec. 2.3, step 1 */

/* ---------------------------------------------------------------------------
 * 3x3 homogeneous helpers (row-major).
 * ------------------------------------------------------------------------- */
static void mat3_mul(const double a[9], const double b[9], double out[9]) {
    double t[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += a[r * 3 + k] * b[k * 3 + c];
            t[r * 3 + c] = s;
        }
    memcpy(out, t, sizeof(t));
}

/*
 * The individual transforms of Sec. 2.1, each as a 3x3 homogeneous matrix.
 *
 * g = { N, dd, h_dm, M, D, H_src, theta_x, theta_y, wfs_rot_deg,
 *       wfs_mag_x, wfs_mag_y, wfs_shift_x_m, wfs_shift_y_m }
 * p = { dm_shift_x_px, dm_shift_y_px, dm_rot_deg, dm_mag }
 *
 * T1: sensor pixel (j, i) -> pupil-plane metres (u, v), centre (M-1)/2.
 * T2: sensor rotation, anamorphic magnification and shift.
 * T3: LGS cone factor (1 - h/H) and footprint shift h * theta.
 * T4: DM misregistration, inverted: r = R(-rot) (q - s) / mag.
 * T5: DM metres -> DM pixel, centre (N-1)/2.
 */
static void transforms(const double g[13], const double p[4], double T1[9], double T2[9],
                       double T3[9], double T4[9], double T5[9]) {
    const double N = g[0], dd = g[1], h = g[2], M = g[3], D = g[4], H = g[5];
    const double dw = D / M, cM = (M - 1.0) / 2.0, cN = (N - 1.0) / 2.0;
    const double tw = g[8] * M_PI / 180.0;
    const double cone = (H > 0.0 && isfinite(H)) ? 1.0 - h / H : 1.0;
    const double td = p[2] * M_PI / 180.0, md = p[3];
    const double sx = p[0] * dd, sy = p[1] * dd;

    double t1[9] = {dw, 0, -cM * dw, 0, dw, -cM * dw, 0, 0, 1};
    double t2[9] = {cos(tw) * g[9], -sin(tw) * g[10], g[11],
                    sin(tw) * g[9], cos(tw) * g[10], g[12],
                    0, 0, 1};
    double t3[9] = {cone, 0, h * g[6], 0, cone, h * g[7], 0, 0, 1};
    /* R(-td) = [[cos, sin], [-sin, cos]] */
    const double c = cos(td), s = sin(td);
    double t4[9] = {c / md, s / md, -(c * sx + s * sy) / md,
                    -s / md, c / md, -(-s * sx + c * sy) / md,
                    0, 0, 1};
    double t5[9] = {1.0 / dd, 0, cN, 0, 1.0 / dd, cN, 0, 0, 1};
    memcpy(T1, t1, sizeof(t1));
    memcpy(T2, t2, sizeof(t2));
    memcpy(T3, t3, sizeof(t3));
    memcpy(T4, t4, sizeof(t4));
    memcpy(T5, t5, sizeof(t5));
}

/*
 * Composite affine (Sec. 2.1): the product T5 T4 T3 T2 T1, so that the DM
 * pixel sampled by sensor pixel (row i, column j) is
 *   x = A[0] j + A[1] i + b[0],   y = A[2] j + A[3] i + b[1].
 */
void synor_composite(const double g[13], const double p[4], double A[4], double b[2]) {
    double T1[9], T2[9], T3[9], T4[9], T5[9], C[9];
    transforms(g, p, T1, T2, T3, T4, T5);
    mat3_mul(T2, T1, C);
    mat3_mul(T3, C, C);
    mat3_mul(T4, C, C);
    mat3_mul(T5, C, C);
    A[0] = C[0]; A[1] = C[1]; b[0] = C[2];
    A[2] = C[3]; A[3] = C[4]; b[1] = C[5];
}

/*
 * Derivative of the composite affine with respect to the four DM
 * misregistration parameters p_k (shift x [px], shift y [px], rotation [deg],
 * magnification).  Only T4 depends on p, so d(C)/dp_k = T5 (dT4/dp_k) T3 T2 T1.
 * dA[4k..4k+3], db[2k..2k+1] follow the layout of synor_composite.
 */
void synor_composite_jac(const double g[13], const double p[4], double dA[16], double db[8]) {
    double T1[9], T2[9], T3[9], T4[9], T5[9], R[9];
    transforms(g, p, T1, T2, T3, T4, T5);
    mat3_mul(T2, T1, R);
    mat3_mul(T3, R, R); /* R = T3 T2 T1 */
    const double dd = g[1];
    const double td = p[2] * M_PI / 180.0, md = p[3];
    const double sx = p[0] * dd, sy = p[1] * dd;
    const double c = cos(td), s = sin(td);
    double dT4[4][9];
    /* d/dsx_px: translation column -R(-td) (dd, 0) / md */
    double a0[9] = {0, 0, -(c * dd) / md, 0, 0, -(-s * dd) / md, 0, 0, 0};
    /* d/dsy_px */
    double a1[9] = {0, 0, -(s * dd) / md, 0, 0, -(c * dd) / md, 0, 0, 0};
    /* d/drot_deg: dR(-td)/dtd = [[-s, c], [-c, -s]], times pi/180 */
    const double k = M_PI / 180.0;
    double a2[9] = {k * (-s) / md, k * c / md, -k * ((-s) * sx + c * sy) / md,
                    k * (-c) / md, k * (-s) / md, -k * ((-c) * sx + (-s) * sy) / md,
                    0, 0, 0};
    /* d/dmd: -(1/md) times the non-homogeneous part of T4 */
    double a3[9] = {-T4[0] / md, -T4[1] / md, -T4[2] / md,
                    -T4[3] / md, -T4[4] / md, -T4[5] / md, 0, 0, 0};
    memcpy(dT4[0], a0, sizeof(a0));
    memcpy(dT4[1], a1, sizeof(a1));
    memcpy(dT4[2], a2, sizeof(a2));
    memcpy(dT4[3], a3, sizeof(a3));
    for (int q = 0; q < 4; ++q) {
        double C[9];
        mat3_mul(dT4[q], R, C);
        mat3_mul(T5, C, C);
        dA[4 * q + 0] = C[0]; dA[4 * q + 1] = C[1]; db[2 * q + 0] = C[2];
        dA[4 * q + 2] = C[3]; dA[4 * q + 3] = C[4]; db[2 * q + 1] = C[5];
    }
}

/*
 * Valid subapertures (Sec. 2.2 grid alignment; validity rule: at least half of
 * the k x k pixels lit, unless an explicit list is given).  Fills
 * row_of_sub[si * n_sub + sj] with the subaperture's rank among valid ones in
 * row-major order (-1 if invalid) and lit[] with its lit-pixel count.
 * Returns the number of valid subapertures, or -1 if M is not k * n_sub.
 */
int synor_valid_subaps(int M, int n_sub, const uint8_t *P, const uint8_t *valid_in,
                       int32_t *row_of_sub, int32_t *lit) {
    if (n_sub <= 0 || M % n_sub != 0) return -1;
    const int k = M / n_sub;
    int nv = 0;
    for (int si = 0; si < n_sub; ++si)
        for (int sj = 0; sj < n_sub; ++sj) {
            int c = 0;
            for (int i = si * k; i < (si + 1) * k; ++i)
                for (int j = sj * k; j < (sj + 1) * k; ++j) c += P[(long)i * M + j] ? 1 : 0;
            lit[si * n_sub + sj] = c;
            int ok = valid_in ? (valid_in[si * n_sub + sj] != 0) : (2 * c >= k * k);
            if (c == 0) ok = 0; /* a subaperture with no light has no slope */
            row_of_sub[si * n_sub + sj] = ok ? nv++ : -1;
        }
    return nv;
}

/* ---------------------------------------------------------------------------
 * Bilinear interpolation (Sec. 2.1), zero outside the N x N grid.
 * ------------------------------------------------------------------------- */
static inline double tap_f(const float *img, int N, long x, long y) {
    if (x < 0 || y < 0 || x >= N || y >= N) return 0.0;
    return (double)img[y * (long)N + x];
}
static inline double tap_u8(const uint8_t *img, int N, long x, long y) {
    if (x < 0 || y < 0 || x >= N || y >= N) return 0.0;
    return img ? (double)img[y * (long)N + x] : 1.0;
}

static double bilinear(const float *img, int N, double x, double y, double *dx, double *dy) {
    const double x0 = floor(x), y0 = floor(y);
    const double fx = x - x0, fy = y - y0;
    const long ix = (long)x0, iy = (long)y0;
    const double v00 = tap_f(img, N, ix, iy), v10 = tap_f(img, N, ix + 1, iy);
    const double v01 = tap_f(img, N, ix, iy + 1), v11 = tap_f(img, N, ix + 1, iy + 1);
    if (dx) *dx = (1.0 - fy) * (v10 - v00) + fy * (v11 - v01);
    if (dy) *dy = (1.0 - fx) * (v01 - v00) + fx * (v11 - v10);
    return (1.0 - fx) * (1.0 - fy) * v00 + fx * (1.0 - fy) * v10 + (1.0 - fx) * fy * v01 +
           fx * fy * v11;
}

static double bilinear_mask(const uint8_t *mask, int N, double x, double y) {
    const double x0 = floor(x), y0 = floor(y);
    const double fx = x - x0, fy = y - y0;
    const long ix = (long)x0, iy = (long)y0;
    return (1.0 - fx) * (1.0 - fy) * tap_u8(mask, N, ix, iy) +
           fx * (1.0 - fy) * tap_u8(mask, N, ix + 1, iy) +
           (1.0 - fx) * fy * tap_u8(mask, N, ix, iy + 1) + fx * fy * tap_u8(mask, N, ix + 1, iy + 1);
}

/*
 * Edge repair step 1 (Sec. 2.3): the DM mask carried by the same composite
 * transform, binarised at 0.999999.  core[i*M + j] = 1 for the pure core.
 * min_margin (optional) receives min |m - 0.999999| over all pixels, so a test
 * can tell how close any pixel came to the threshold.
 */
void synor_core(int N, const uint8_t *dm_mask, int M, const double A[4], const double b[2],
                uint8_t *core, double *min_margin) {
    double mm = INFINITY;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            const double x = A[0] * j + A[1] * i + b[0];
            const double y = A[2] * j + A[3] * i + b[1];
            const double m = bilinear_mask(dm_mask, N, x, y);
            core[(long)i * M + j] = (m >= SYNOR_CORE_THRESHOLD) ? 1 : 0;
            const double d = fabs(m - SYNOR_CORE_THRESHOLD);
            if (d < mm) mm = d;
        }
    if (min_margin) *min_margin = mm;
}

static inline int is_core(const uint8_t *core, int M, long i, long j) {
    if (i < 0 || j < 0 || i >= M || j >= M) return 0;
    return core[i * M + j] != 0;
}

/*
 * Edge repair steps 2 and 3 (Sec. 2.3), applied to a field that is already
 * zero outside the core: ring = 4-connected dilation of the core minus the
 * core; each ring pixel becomes the mean over the valid cardinal directions
 * of 2 P1 - P2 (both in the core) or P1 (only the adjacent pixel in the core).
 * Writes the repaired field to phi and the pixel class (0 zero, 1 core,
 * 2 ring) to cls when cls is not NULL.
 */
static void edge_repair(const double *phic, const uint8_t *core, int M, double *phi, uint8_t *cls) {
    static const int di[4] = {0, 0, 1, -1}, dj[4] = {1, -1, 0, 0};
    for (long i = 0; i < M; ++i)
        for (long j = 0; j < M; ++j) {
            const long p = i * M + j;
            if (core[p]) {
                phi[p] = phic[p];
                if (cls) cls[p] = 1;
                continue;
            }
            double sum = 0.0;
            int n = 0;
            for (int d = 0; d < 4; ++d) {
                const long i1 = i + di[d], j1 = j + dj[d];
                if (!is_core(core, M, i1, j1)) continue;
                const long i2 = i + 2 * di[d], j2 = j + 2 * dj[d];
                if (is_core(core, M, i2, j2))
                    sum += 2.0 * phic[i1 * M + j1] - phic[i2 * M + j2];
                else
                    sum += phic[i1 * M + j1];
                ++n;
            }
            phi[p] = n ? sum / n : 0.0;
            if (cls) cls[p] = n ? 2 : 0;
        }
}

/*
 * Numerical derivative and subaperture average (Sec. 2.2): central
 * differences of the repaired phase at every pixel, weighted by the sensor
 * pupil P, summed over each subaperture and divided by its lit-pixel count.
 * Writes rows [x slopes of valid subaps ; y slopes] of one IM column.
 */
static void slopes_from_phase(const double *phi, int M, int n_sub, const uint8_t *P,
                              const int32_t *row_of_sub, const int32_t *lit, int nv, double dw,
                              double slope_scale, double *col, double *sx, double *sy) {
    const int k = M / n_sub;
    const int ns = n_sub * n_sub;
    for (int s = 0; s < ns; ++s) sx[s] = sy[s] = 0.0;
    for (long i = 0; i < M; ++i)
        for (long j = 0; j < M; ++j) {
            if (!P[i * M + j]) continue;
            const double e = (j + 1 < M) ? phi[i * M + j + 1] : 0.0;
            const double w = (j - 1 >= 0) ? phi[i * M + j - 1] : 0.0;
            const double n = (i + 1 < M) ? phi[(i + 1) * M + j] : 0.0;
            const double s = (i - 1 >= 0) ? phi[(i - 1) * M + j] : 0.0;
            const int sub = (int)(i / k) * n_sub + (int)(j / k);
            sx[sub] += (e - w) / (2.0 * dw);
            sy[sub] += (n - s) / (2.0 * dw);
        }
    for (int s = 0; s < ns; ++s) {
        const int r = row_of_sub[s];
        if (r < 0) continue;
        col[r] = slope_scale * sx[s] / lit[s];
        col[nv + r] = slope_scale * sy[s] / lit[s];
    }
}

/*
 * Repaired phase of one influence function on the sensor grid (Sec. 2.1 +
 * Sec. 2.3), for tests that check the later stages independently.
 */
void synor_phase(const float *ifs_a, int N, const uint8_t *dm_mask, int M, const double A[4],
                 const double b[2], double *phi, uint8_t *cls) {
    uint8_t *core = (uint8_t *)malloc((size_t)M * M);
    double *phic = (double *)malloc(sizeof(double) * (size_t)M * M);
    synor_core(N, dm_mask, M, A, b, core, NULL);
    for (long i = 0; i < M; ++i)
        for (long j = 0; j < M; ++j) {
            const long p = i * M + j;
            phic[p] = core[p] ? bilinear(ifs_a, N, A[0] * j + A[1] * i + b[0],
                                         A[2] * j + A[3] * i + b[1], NULL, NULL)
                              : 0.0;
        }
    edge_repair(phic, core, M, phi, cls);
    free(core);
    free(phic);
}

/*
 * IM columns (the whole method, Sec. 2.1-2.3) for the actuators listed in
 * cols[0..ncols).  out is [ncols][2 nv] (column-major IM).  Returns nv, or
 * -1 on a shape error.  Columns are independent; nthreads > 1 splits them
 * over OpenMP threads without changing any arithmetic.
 */
int synor_im(const float *ifs, int n_act, int N, const uint8_t *dm_mask, int M, int n_sub,
             const uint8_t *P, const uint8_t *valid_in, const double A[4], const double b[2],
             double dw, double slope_scale, const int32_t *cols, int ncols, double *out,
             int nthreads) {
    if (n_sub <= 0 || M % n_sub != 0) return -1;
    const int ns = n_sub * n_sub;
    int32_t *row_of_sub = (int32_t *)malloc(sizeof(int32_t) * ns);
    int32_t *lit = (int32_t *)malloc(sizeof(int32_t) * ns);
    const int nv = synor_valid_subaps(M, n_sub, P, valid_in, row_of_sub, lit);
    uint8_t *core = (uint8_t *)malloc((size_t)M * M);
    synor_core(N, dm_mask, M, A, b, core, NULL);
    const long MM = (long)M * M;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *phic = (double *)malloc(sizeof(double) * MM);
        double *phi = (double *)malloc(sizeof(double) * MM);
        double *sx = (double *)malloc(sizeof(double) * ns);
        double *sy = (double *)malloc(sizeof(double) * ns);
#pragma omp for schedule(dynamic, 1)
        for (int c = 0; c < ncols; ++c) {
            const int a = cols[c];
            double *col = out + (long)c * 2 * nv;
            if (a < 0 || a >= n_act) {
                for (int r = 0; r < 2 * nv; ++r) col[r] = NAN;
                continue;
            }
            const float *img = ifs + (long)a * N * N;
            for (long i = 0; i < M; ++i)
                for (long j = 0; j < M; ++j) {
                    const long p = i * M + j;
                    phic[p] = core[p] ? bilinear(img, N, A[0] * j + A[1] * i + b[0],
                                                 A[2] * j + A[3] * i + b[1], NULL, NULL)
                                      : 0.0;
                }
            edge_repair(phic, core, M, phi, NULL);
            slopes_from_phase(phi, M, n_sub, P, row_of_sub, lit, nv, dw, slope_scale, col, sx, sy);
        }
        free(phic);
        free(phi);
        free(sx);
        free(sy);
    }
    free(core);
    free(row_of_sub);
    free(lit);
    return nv;
}

/*
 * Tangents of the IM columns with respect to the four misregistration
 * parameters, with the core set held fixed: the chain rule through the
 * bilinear interpolation (derivative of the floor cell), the linear edge
 * repair, the derivative and the average.  dA/db come from
 * synor_composite_jac.  out is [4][ncols][2 nv].
 */
int synor_im_tangent(const float *ifs, int n_act, int N, const uint8_t *dm_mask, int M, int n_sub,
                     const uint8_t *P, const uint8_t *valid_in, const double A[4],
                     const double b[2], const double dA[16], const double db[8], double dw,
                     double slope_scale, const int32_t *cols, int ncols, double *out,
                     int nthreads) {
    if (n_sub <= 0 || M % n_sub != 0) return -1;
    const int ns = n_sub * n_sub;
    int32_t *row_of_sub = (int32_t *)malloc(sizeof(int32_t) * ns);
    int32_t *lit = (int32_t *)malloc(sizeof(int32_t) * ns);
    const int nv = synor_valid_subaps(M, n_sub, P, valid_in, row_of_sub, lit);
    uint8_t *core = (uint8_t *)malloc((size_t)M * M);
    synor_core(N, dm_mask, M, A, b, core, NULL);
    const long MM = (long)M * M;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *dphic = (double *)malloc(sizeof(double) * MM * 4);
        double *phi = (double *)malloc(sizeof(double) * MM);
        double *sx = (double *)malloc(sizeof(double) * ns);
        double *sy = (double *)malloc(sizeof(double) * ns);
#pragma omp for schedule(dynamic, 1)
        for (int c = 0; c < ncols; ++c) {
            const int a = cols[c];
            if (a < 0 || a >= n_act) continue;
            const float *img = ifs + (long)a * N * N;
            for (long i = 0; i < M; ++i)
                for (long j = 0; j < M; ++j) {
                    const long p = i * M + j;
                    if (!core[p]) {
                        for (int q = 0; q < 4; ++q) dphic[q * MM + p] = 0.0;
                        continue;
                    }
                    double gx, gy;
                    bilinear(img, N, A[0] * j + A[1] * i + b[0], A[2] * j + A[3] * i + b[1], &gx,
                             &gy);
                    for (int q = 0; q < 4; ++q) {
                        const double ddx = dA[4 * q + 0] * j + dA[4 * q + 1] * i + db[2 * q + 0];
                        const double ddy = dA[4 * q + 2] * j + dA[4 * q + 3] * i + db[2 * q + 1];
                        dphic[q * MM + p] = gx * ddx + gy * ddy;
                    }
                }
            for (int q = 0; q < 4; ++q) {
                double *col = out + ((long)q * ncols + c) * 2 * nv;
                edge_repair(dphic + q * MM, core, M, phi, NULL);
                slopes_from_phase(phi, M, n_sub, P, row_of_sub, lit, nv, dw, slope_scale, col, sx,
                                  sy);
            }
        }
        free(dphic);
        free(phi);
        free(sx);
        free(sy);
    }
    free(core);
    free(row_of_sub);
    free(lit);
    return nv;
}

/* ---------------------------------------------------------------------------
 * Probe responses (training data of the learned misregistration estimator).
 *
 * A probe mode m is the DM shape S_m = sum_a cmd[m][a] IF_a (a "modal
 * screen", formed by the caller in double precision).  Its response at
 * misregistration p is the slope vector the method (Sec. 2.1-2.3) gives for
 * S_m: one bilinear resample through the composite transform, edge repair
 * with the core set of the DM mask, central differences, pupil-weighted
 * subaperture mean.  Every step is linear in the phase for a fixed core set,
 * so the response equals cmd[m] . IM(p); the tests pin this function to the
 * already pinned IM oracle that way.
 * ------------------------------------------------------------------------- */
static inline double tap_d(const double *img, int N, long x, long y) {
    if (x < 0 || y < 0 || x >= N || y >= N) return 0.0;
    return img[y * (long)N + x];
}

static double bilinear_d(const double *img, int N, double x, double y, double *dx, double *dy) {
    const double x0 = floor(x), y0 = floor(y);
    const double fx = x - x0, fy = y - y0;
    const long ix = (long)x0, iy = (long)y0;
    const double v00 = tap_d(img, N, ix, iy), v10 = tap_d(img, N, ix + 1, iy);
    const double v01 = tap_d(img, N, ix, iy + 1), v11 = tap_d(img, N, ix + 1, iy + 1);
    if (dx) *dx = (1.0 - fy) * (v10 - v00) + fy * (v11 - v01);
    if (dy) *dy = (1.0 - fx) * (v01 - v00) + fx * (v11 - v10);
    return (1.0 - fx) * (1.0 - fy) * v00 + fx * (1.0 - fy) * v10 + (1.0 - fx) * fy * v01 +
           fx * fy * v11;
}

/*
 * Responses of n_modes screens [n_modes][N][N] (double) at one composite
 * transform.  out is [n_modes][2 nv]; when dA/db are given, dout receives the
 * tangents [4][n_modes][2 nv] (core set held fixed, floor-cell derivative, as
 * synor_im_tangent).  Returns nv, or -1 on a shape error.
 */
int synor_probe(const double *screens, int n_modes, int N, const uint8_t *dm_mask, int M,
                int n_sub, const uint8_t *P, const uint8_t *valid_in, const double A[4],
                const double b[2], const double *dA, const double *db, double dw,
                double slope_scale, double *out, double *dout) {
    if (n_sub <= 0 || M % n_sub != 0) return -1;
    const int ns = n_sub * n_sub;
    const long MM = (long)M * M;
    int32_t *row_of_sub = (int32_t *)malloc(sizeof(int32_t) * ns);
    int32_t *lit = (int32_t *)malloc(sizeof(int32_t) * ns);
    const int nv = synor_valid_subaps(M, n_sub, P, valid_in, row_of_sub, lit);
    uint8_t *core = (uint8_t *)malloc((size_t)MM);
    double *phic = (double *)malloc(sizeof(double) * MM * 5);
    double *phi = (double *)malloc(sizeof(double) * MM);
    double *sx = (double *)malloc(sizeof(double) * ns);
    double *sy = (double *)malloc(sizeof(double) * ns);
    synor_core(N, dm_mask, M, A, b, core, NULL);
    const int nq = (dA && db && dout) ? 5 : 1;
    for (int m = 0; m < n_modes; ++m) {
        const double *img = screens + (long)m * N * N;
        for (long i = 0; i < M; ++i)
            for (long j = 0; j < M; ++j) {
                const long p = i * M + j;
                if (!core[p]) {
                    for (int q = 0; q < nq; ++q) phic[q * MM + p] = 0.0;
                    continue;
                }
                double gx, gy;
                phic[p] = bilinear_d(img, N, A[0] * j + A[1] * i + b[0],
                                     A[2] * j + A[3] * i + b[1], &gx, &gy);
                for (int q = 1; q < nq; ++q) {
                    const int k = q - 1;
                    const double ddx = dA[4 * k + 0] * j + dA[4 * k + 1] * i + db[2 * k + 0];
                    const double ddy = dA[4 * k + 2] * j + dA[4 * k + 3] * i + db[2 * k + 1];
                    phic[q * MM + p] = gx * ddx + gy * ddy;
                }
            }
        for (int q = 0; q < nq; ++q) {
            double *col = (q == 0) ? out + (long)m * 2 * nv
                                   : dout + ((long)(q - 1) * n_modes + m) * 2 * nv;
            edge_repair(phic + q * MM, core, M, phi, NULL);
            slopes_from_phase(phi, M, n_sub, P, row_of_sub, lit, nv, dw, slope_scale, col, sx,
                              sy);
        }
    }
    free(core);
    free(phic);
    free(phi);
    free(sx);
    free(sy);
    free(row_of_sub);
    free(lit);
    return nv;
}

/* ---------------------------------------------------------------------------
 * Counter-based random numbers for the probe noise: Philox4x32 with 10
 * rounds (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC 2011), written from its published definition.  Each round
 * multiplies counter words 0 and 2 by the two round constants, takes the
 * 64-bit products apart and mixes the high halves with the other counter
 * words and the key; the key is bumped by the two Weyl constants between
 * rounds.
 * ------------------------------------------------------------------------- */
void synor_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    memcpy(out, c, sizeof(c));
}

/*
 * Standard normal deviates of probe-noise element e[0..n) of one sample.
 * Element e takes Philox block ctr = (e / 4, sample low, sample high, 0)
 * under key (seed low, seed high); its lane pair (words 2t, 2t+1, t = (e % 4)
 * / 2) gives u1 = (w0 + 1) 2^-32 and u2 = w1 2^-32, and the Box-Muller
 * transform (Box and Muller 1958) turns them into sqrt(-2 ln u1) times
 * cos(2 pi u2) for even e, sin(2 pi u2) for odd e.
 */
void synor_gauss(uint64_t seed, uint64_t sample, const int64_t *e, long n, double *z) {
    const double two32 = 4294967296.0;
    const double pi = 3.14159265358979323846;
    for (long q = 0; q < n; ++q) {
        const uint64_t blk = (uint64_t)e[q] / 4;
        const int lane = (int)(e[q] % 4);
        const uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)sample, (uint32_t)(sample >> 32), 0u};
        const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t w[4];
        synor_philox4x32_10(ctr, key, w);
        const int t = lane / 2;
        const double u1 = ((double)w[2 * t] + 1.0) / two32;
        const double u2 = (double)w[2 * t + 1] / two32;
        const double r = sqrt(-2.0 * log(u1));
        z[q] = (lane % 2 == 0) ? r * cos(2.0 * pi * u2) : r * sin(2.0 * pi * u2);
    }
}
