// synim_projection.cu -- tomographic projection matrices and P_opt (Sec. 3,
// tomographic projection matrices).
//
// P_X[(j, q), a] is the mean over the bin x bin fine pixels p of binned pupil
// pixel q of P(p) * bilinear(IF_a; A_j (p_col, p_row) + b_j).  Here (A_j, b_j)
// is the composite affine (Sec. 2.1) of the component seen from direction j
// by a source at infinity on the chosen sensor's grid: no cone, no sensor
// rotation, magnification or shift, no misregistration, so the footprint
// moves by h theta_j.  P is the sensor's pupil mask.  There is no edge
// repair (a phase projection, not a slope).  Rows are direction-major,
// row = j (M / bin)^2 + q.
//
//   k_proj             one CTA per (actuator, direction) writes that column
//                      segment: the binned pixels of the actuator's footprint
//                      box from its packed window (zero border = zero outside),
//                      zeros elsewhere;
//   P_DM^T P_DM, P_DM^T P_Layer
//                      FP32 products (cuBLAS SSYRK for the symmetric normal
//                      matrix, SGEMM for the right-hand side); TF32 would
//                      lose ~1e-3 relative per product, which the solve
//                      multiplies by the condition number;
//   + lambda I, Cholesky factor (cuSOLVER SPOTRF) and two triangular solves
//                      (cuBLAS STRSM) for all layer columns.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <cublas_v2.h>
#include <cusolverDn.h>

#include "synim.h"
#include "synim_device.cuh"
#include "synim_geom.h"
#include "synim_internal.h"

namespace synim {

struct ProjDir {
    double A[4], b[2];   // composite affine of (component, direction), DM pixels
};

constexpr int kProjThreads = 256;

// Column segment of actuator a (blockIdx.x) and direction j (blockIdx.y) of
// one component: out[col0 + a][j * Mb^2 + q].
__global__ void __launch_bounds__(kProjThreads)
k_proj(const DevDM D, const ProjDir *__restrict__ dirs, const uint8_t *__restrict__ pupil, int M, int bin,
       long long K, long long col0, float *__restrict__ out) {
    const int a = blockIdx.x, j = blockIdx.y;
    const int Mb = M / bin;
    const ProjDir pd = dirs[j];
    const int wx0 = D.org[2 * a], wy0 = D.org[2 * a + 1];
    // footprint box: the sensor pixels whose image falls in the window's cells
    __shared__ int box[4];
    __shared__ float ref[2];
    if (threadIdx.x == 0) {
        const double det = pd.A[0] * pd.A[3] - pd.A[1] * pd.A[2];
        const double i00 = pd.A[3] / det, i01 = -pd.A[1] / det, i10 = -pd.A[2] / det, i11 = pd.A[0] / det;
        double jmin = 1e300, jmax = -1e300, imin = 1e300, imax = -1e300;
        for (int c = 0; c < 4; ++c) {
            const double dx = ((c & 1) ? wx0 + D.W : wx0 - 1) - pd.b[0];
            const double dy = ((c & 2) ? wy0 + D.W : wy0 - 1) - pd.b[1];
            const double jj = i00 * dx + i01 * dy, ii = i10 * dx + i11 * dy;
            jmin = fmin(jmin, jj); jmax = fmax(jmax, jj);
            imin = fmin(imin, ii); imax = fmax(imax, ii);
        }
        const double lo = -2.0, hi = (double)M + 2.0;
        jmin = fmax(jmin, lo); imin = fmax(imin, lo); jmax = fmin(jmax, hi); imax = fmin(imax, hi);
        const int j0 = max(0, (int)floor(jmin) - 1), j1 = min(M - 1, (int)ceil(jmax) + 1);
        const int i0 = max(0, (int)floor(imin) - 1), i1 = min(M - 1, (int)ceil(imax) + 1);
        box[0] = i0 / bin; box[1] = i1 / bin; box[2] = j0 / bin; box[3] = j1 / bin;
        if (j0 > j1 || i0 > i1) box[1] = box[0] - 1;   // empty
        // window-local coordinates of fine pixel (row box[0] bin, col box[2] bin), FP64
        const double jr = (double)(box[2] * bin), ir = (double)(box[0] * bin);
        ref[0] = (float)(pd.A[0] * jr + pd.A[1] * ir + pd.b[0] - (wx0 - 1));
        ref[1] = (float)(pd.A[2] * jr + pd.A[3] * ir + pd.b[1] - (wy0 - 1));
    }
    __syncthreads();
    const int qi0 = box[0], qi1 = box[1], qj0 = box[2], qj1 = box[3];
    const float a00 = (float)pd.A[0], a01 = (float)pd.A[1], a10 = (float)pd.A[2], a11 = (float)pd.A[3];
    const float xr = ref[0], yr = ref[1];
    const float *win = D.win + (size_t)a * D.win_stride;
    const float Wf1 = (float)(D.W + 1);
    const float inv = 1.f / (float)(bin * bin);
    float *dst = out + (size_t)(col0 + a) * K + (size_t)j * Mb * Mb;
    for (int q = threadIdx.x; q < Mb * Mb; q += kProjThreads) {
        const int qi = q / Mb, qj = q - qi * Mb;
        float v = 0.f;
        if (qi >= qi0 && qi <= qi1 && qj >= qj0 && qj <= qj1) {
            for (int u = 0; u < bin; ++u)
                for (int w = 0; w < bin; ++w) {
                    const int i = qi * bin + u, jj = qj * bin + w;
                    if (!pupil[(size_t)i * M + jj]) continue;
                    const float di = (float)(i - qi0 * bin), dj = (float)(jj - qj0 * bin);
                    const float x = fmaf(a00, dj, fmaf(a01, di, xr));
                    const float y = fmaf(a10, dj, fmaf(a11, di, yr));
                    if (!(x > 0.f && x < Wf1 && y > 0.f && y < Wf1)) continue;
                    const float fx0 = floorf(x), fy0 = floorf(y);
                    const float fx = x - fx0, fy = y - fy0;
                    const float *t = win + (int)fy0 * D.Wp + (int)fx0;
                    const float top = fmaf(fx, t[1] - t[0], t[0]);
                    const float bot = fmaf(fx, t[D.Wp + 1] - t[D.Wp], t[D.Wp]);
                    v += fmaf(fy, bot - top, top);
                }
            v *= inv;
        }
        dst[q] = v;
    }
}

__global__ void k_add_diag(float *__restrict__ G, long long n, float lam) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) G[i * n + i] += lam;
}

void projection_destroy(synim_ctx *c) {
    if (c->cublas) cublasDestroy(static_cast<cublasHandle_t>(c->cublas));
    if (c->cusolver) cusolverDnDestroy(static_cast<cusolverDnHandle_t>(c->cusolver));
    c->cublas = nullptr;
    c->cusolver = nullptr;
}

}  // namespace synim

using namespace synim;

namespace {

synim_status pfail(synim_ctx *c, synim_status s, const std::string &m) {
    if (c) c->err = m;
    return s;
}

// Projection matrices of the listed components into P [n_cols][K].
synim_status build_p(synim_ctx *ctx, int w, int n_dir, const double *dirs, int bin, int n_comp, const int *comps,
                     float *P, long long K, const uint8_t *d_pupil, ProjDir *d_dirs, cudaStream_t st) {
    long long col = 0;
    std::vector<ProjDir> hd((size_t)n_dir);
    for (int c = 0; c < n_comp; ++c) {
        const int d = comps[c];
        const DmHost &Dh = ctx->dmh[d];
        WfsHost view = ctx->wh[w];
        view.H = 0.0;
        view.rot = 0.0;
        view.mag[0] = view.mag[1] = 1.0;
        view.shift[0] = view.shift[1] = 0.0;
        for (int j = 0; j < n_dir; ++j) {
            view.th[0] = dirs[2 * j];
            view.th[1] = dirs[2 * j + 1];
            const synim_misreg m{0.0, 0.0, 0.0, 1.0};
            composite(Dh, view, m, hd[j].A, hd[j].b);
        }
        cudaError_t e = cudaMemcpyAsync(d_dirs + (size_t)c * n_dir, hd.data(), sizeof(ProjDir) * n_dir,
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_CUDA, std::string("projection upload: ") + cudaGetErrorString(e));
        dim3 grid((unsigned)Dh.n_act, (unsigned)n_dir);
        k_proj<<<grid, kProjThreads, 0, st>>>(ctx->geo.dm[d], d_dirs + (size_t)c * n_dir, d_pupil, ctx->wh[w].M, bin,
                                              K, col, P);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return pfail(ctx, SYNIM_ERR_CUDA, std::string("k_proj: ") + cudaGetErrorString(e));
        col += Dh.n_act;
    }
    return SYNIM_OK;
}

synim_status check_args(synim_ctx *ctx, int w, int n_dir, const double *dirs, int bin, int n_comp, const int *comps) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    if (w < 0 || w >= ctx->n_wfs || n_dir < 1 || !dirs || bin < 1 || n_comp < 1 || !comps)
        return pfail(ctx, SYNIM_ERR_INVALID_ARG, "projection: bad sensor, directions, binning or components");
    if (ctx->wh[w].M % bin != 0)
        return pfail(ctx, SYNIM_ERR_SHAPE, "projection: the sensor grid must be a multiple of the binning");
    for (int c = 0; c < n_comp; ++c)
        if (comps[c] < 0 || comps[c] >= ctx->n_dm) return pfail(ctx, SYNIM_ERR_INVALID_ARG, "projection: bad component");
    return SYNIM_OK;
}

long long n_cols(const synim_ctx *ctx, int n_comp, const int *comps) {
    long long n = 0;
    for (int c = 0; c < n_comp; ++c) n += ctx->dmh[comps[c]].n_act;
    return n;
}

// Scratch of one call, freed on every return path.
struct ProjScratch {
    std::vector<void *> p;
    ~ProjScratch() {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    cudaError_t alloc(T **q, size_t n) {
        void *v = nullptr;
        cudaError_t e = cudaMalloc(&v, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) {
            p.push_back(v);
            *q = static_cast<T *>(v);
        }
        return e;
    }
};

}  // namespace

extern "C" {

synim_status synim_projection_rows(const synim_ctx *ctx, int32_t wfs, int32_t n_dir, int32_t bin, int64_t *rows) {
    if (!ctx || !rows || wfs < 0 || wfs >= ctx->n_wfs || n_dir < 1 || bin < 1 || ctx->wh[wfs].M % bin != 0)
        return SYNIM_ERR_INVALID_ARG;
    const long long Mb = ctx->wh[wfs].M / bin;
    *rows = (int64_t)n_dir * Mb * Mb;
    return SYNIM_OK;
}

synim_status synim_projection_matrix(synim_ctx *ctx, int32_t wfs, int32_t n_dir, const double *dirs_rad, int32_t bin,
                                     int32_t n_comp, const int32_t *comps, float *P, void *cuda_stream) {
    synim_status s = check_args(ctx, wfs, n_dir, dirs_rad, bin, n_comp, comps);
    if (s != SYNIM_OK) return s;
    if (!P) return pfail(ctx, SYNIM_ERR_INVALID_ARG, "projection: P is required");
    ctx->err.clear();
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int64_t K = 0;
    synim_projection_rows(ctx, wfs, n_dir, bin, &K);
    ProjScratch sc;
    uint8_t *d_pupil = nullptr;
    ProjDir *d_dirs = nullptr;
    const int M = ctx->wh[wfs].M;
    cudaError_t e = sc.alloc(&d_pupil, (size_t)M * M);
    if (e == cudaSuccess) e = sc.alloc(&d_dirs, (size_t)n_comp * n_dir);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pupil, ctx->pupil[wfs].data(), (size_t)M * M, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_OOM, std::string("projection scratch: ") + cudaGetErrorString(e));
    s = build_p(ctx, wfs, n_dir, dirs_rad, bin, n_comp, comps, P, K, d_pupil, d_dirs, st);
    if (s != SYNIM_OK) return s;
    // the scratch is freed on return: wait for the kernels that read it
    e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? SYNIM_OK : pfail(ctx, SYNIM_ERR_CUDA, cudaGetErrorString(e));
}

synim_status synim_projection_opt(synim_ctx *ctx, int32_t wfs, int32_t n_dir, const double *dirs_rad, int32_t bin,
                                  int32_t n_dm, const int32_t *dms, int32_t n_layer, const int32_t *layers,
                                  double lambda, float *p_opt, void *cuda_stream) {
    synim_status s = check_args(ctx, wfs, n_dir, dirs_rad, bin, n_dm, dms);
    if (s == SYNIM_OK) s = check_args(ctx, wfs, n_dir, dirs_rad, bin, n_layer, layers);
    if (s != SYNIM_OK) return s;
    if (!p_opt || !(lambda >= 0.0)) return pfail(ctx, SYNIM_ERR_INVALID_ARG, "projection: p_opt and lambda >= 0 required");
    ctx->err.clear();
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int64_t K = 0;
    synim_projection_rows(ctx, wfs, n_dir, bin, &K);
    const long long nd = n_cols(ctx, n_dm, dms), nl = n_cols(ctx, n_layer, layers);
    const int M = ctx->wh[wfs].M;
    ProjScratch sc;
    uint8_t *d_pupil = nullptr;
    ProjDir *d_dirs = nullptr;
    float *Pd = nullptr, *Pl = nullptr, *G = nullptr, *work = nullptr;
    int *info = nullptr;
    cudaError_t e = sc.alloc(&d_pupil, (size_t)M * M);
    if (e == cudaSuccess) e = sc.alloc(&d_dirs, (size_t)(n_dm + n_layer) * n_dir);
    if (e == cudaSuccess) e = sc.alloc(&Pd, (size_t)nd * K);
    if (e == cudaSuccess) e = sc.alloc(&Pl, (size_t)nl * K);
    if (e == cudaSuccess) e = sc.alloc(&G, (size_t)nd * nd);
    if (e == cudaSuccess) e = sc.alloc(&info, 2);
    if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pupil, ctx->pupil[wfs].data(), (size_t)M * M, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_OOM, std::string("projection scratch: ") + cudaGetErrorString(e));
    if ((s = build_p(ctx, wfs, n_dir, dirs_rad, bin, n_dm, dms, Pd, K, d_pupil, d_dirs, st)) != SYNIM_OK) return s;
    if ((s = build_p(ctx, wfs, n_dir, dirs_rad, bin, n_layer, layers, Pl, K, d_pupil, d_dirs + (size_t)n_dm * n_dir,
                     st)) != SYNIM_OK)
        return s;
    // normal matrix (lower triangle) and right-hand side, FP32
    if (!ctx->cublas) {
        cublasHandle_t h = nullptr;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return pfail(ctx, SYNIM_ERR_CUDA, "cublasCreate failed");
        ctx->cublas = h;
    }
    if (!ctx->cusolver) {
        cusolverDnHandle_t h = nullptr;
        if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return pfail(ctx, SYNIM_ERR_CUDA, "cusolverDnCreate failed");
        ctx->cusolver = h;
    }
    cublasHandle_t hb = static_cast<cublasHandle_t>(ctx->cublas);
    cusolverDnHandle_t hs = static_cast<cusolverDnHandle_t>(ctx->cusolver);
    cublasSetStream(hb, st);
    cusolverDnSetStream(hs, st);
    cublasSetMathMode(hb, CUBLAS_PEDANTIC_MATH);   // no TF32 anywhere
    const float one = 1.f, zero = 0.f;
    cublasStatus_t bs = cublasSsyrk(hb, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, (int)nd, (int)K, &one, Pd, (int)K, &zero,
                                    G, (int)nd);
    if (bs == CUBLAS_STATUS_SUCCESS)
        bs = cublasSgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, (int)nd, (int)nl, (int)K, &one, Pd, (int)K, Pl, (int)K, &zero,
                         p_opt, (int)nd);
    if (bs != CUBLAS_STATUS_SUCCESS)
        return pfail(ctx, SYNIM_ERR_CUDA, "projection products failed (cuBLAS status " + std::to_string((int)bs) + ")");
    k_add_diag<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(G, nd, (float)lambda);
    // G + lambda I = L L^T, then P_opt = L^-T (L^-1 R) for all layer columns
    int lwork = 0;
    if (cusolverDnSpotrf_bufferSize(hs, CUBLAS_FILL_MODE_LOWER, (int)nd, G, (int)nd, &lwork) != CUSOLVER_STATUS_SUCCESS)
        return pfail(ctx, SYNIM_ERR_CUDA, "cusolverDnSpotrf_bufferSize failed");
    if ((e = sc.alloc(&work, (size_t)std::max(lwork, 1))) != cudaSuccess)
        return pfail(ctx, SYNIM_ERR_OOM, "projection solver workspace");
    if (cusolverDnSpotrf(hs, CUBLAS_FILL_MODE_LOWER, (int)nd, G, (int)nd, work, lwork, info) != CUSOLVER_STATUS_SUCCESS)
        return pfail(ctx, SYNIM_ERR_CUDA, "cusolverDnSpotrf failed");
    bs = cublasStrsm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, (int)nd, (int)nl,
                     &one, G, (int)nd, p_opt, (int)nd);
    if (bs == CUBLAS_STATUS_SUCCESS)
        bs = cublasStrsm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, (int)nd,
                         (int)nl, &one, G, (int)nd, p_opt, (int)nd);
    if (bs != CUBLAS_STATUS_SUCCESS)
        return pfail(ctx, SYNIM_ERR_CUDA, "projection triangular solves failed (cuBLAS status " +
                                              std::to_string((int)bs) + ")");
    int h_info[2] = {0, 0};
    if ((e = cudaMemcpyAsync(h_info, info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return pfail(ctx, SYNIM_ERR_CUDA, std::string("projection: ") + cudaGetErrorString(e));
    if (h_info[0] != 0)
        return pfail(ctx, SYNIM_ERR_NOT_CONVERGED,
                     "projection: P_DM^T P_DM + lambda I is not positive definite (raise lambda)");
    return SYNIM_OK;
}

}  // extern "C"
