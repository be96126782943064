// synim_projection.cu -- tomographic projection matrices and P_opt (Sec. 2.5,
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
//   k_proj             (synim_projection_matrix) one CTA per (actuator,
//                      direction) writes that dense column segment: the binned
//                      pixels of the actuator's footprint box from its packed
//                      window (zero border = zero outside), zeros elsewhere;
//   k_proj_boxes, k_proj_vals
//                      (P_opt) the same values, stored box by box: a column
//                      is non-zero only on its footprint box in each direction
//                      (about 1 % of the rows at the bench size);
//   k_box_dot          P_DM^T P_DM and P_DM^T P_Layer from the boxes: one CTA
//                      per DM actuator; the candidates are the actuators whose
//                      union box (over the directions) meets its own, found
//                      through a bucket grid; each candidate's entry is the sum
//                      over directions of the dot product over the two boxes'
//                      intersection (FP32), everything else stays zero;
//   + lambda I, then the blocked Cholesky factor and the two block triangular
//                      sweeps for all layer columns (synim_dense.cu: every
//                      block update a 3xTF32 tcgen05 GEMM, FP32 accuracy).
#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

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

// Footprint box (binned pixels, inclusive; qi1 < qi0 when empty) of actuator
// a seen from one direction, and the window-local coordinates (xr, yr) of fine
// pixel (qi0 bin, qj0 bin), both from the FP64 affine.
__device__ __forceinline__ int4 proj_box(const DevDM &D, const ProjDir &pd, int a, int M, int bin, float &xr,
                                         float &yr) {
    const int wx0 = D.org[2 * a], wy0 = D.org[2 * a + 1];
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
    int4 box = make_int4(i0 / bin, i1 / bin, j0 / bin, j1 / bin);
    if (j0 > j1 || i0 > i1) box = make_int4(0, -1, 0, -1);
    const double jr = (double)(box.z * bin), ir = (double)(box.x * bin);
    xr = (float)(pd.A[0] * jr + pd.A[1] * ir + pd.b[0] - (wx0 - 1));
    yr = (float)(pd.A[2] * jr + pd.A[3] * ir + pd.b[1] - (wy0 - 1));
    return box;
}

// Value of binned pixel (qi, qj) of a box whose first fine pixel has window
// coordinates (xr, yr).
__device__ __forceinline__ float proj_value(const DevDM &D, const float *__restrict__ win, const ProjDir &pd,
                                            const uint8_t *__restrict__ pupil, int M, int bin, int4 box, float xr,
                                            float yr, int qi, int qj) {
    const float a00 = (float)pd.A[0], a01 = (float)pd.A[1], a10 = (float)pd.A[2], a11 = (float)pd.A[3];
    const float Wf1 = (float)(D.W + 1);
    float v = 0.f;
    for (int u = 0; u < bin; ++u)
        for (int w = 0; w < bin; ++w) {
            const int i = qi * bin + u, jj = qj * bin + w;
            if (!pupil[(size_t)i * M + jj]) continue;
            const float di = (float)(i - box.x * bin), dj = (float)(jj - box.z * bin);
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
    return v * (1.f / (float)(bin * bin));
}

// Boxes of every (actuator, direction) of one component: boxes[(col0 + a) n_dir + j].
__global__ void k_proj_boxes(const DevDM D, const ProjDir *__restrict__ dirs, int M, int bin, int n_act, int n_dir,
                             long long col0, int4 *__restrict__ boxes) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_act * n_dir) return;
    const int a = (int)(t / n_dir), j = (int)(t - (long long)a * n_dir);
    float xr, yr;
    boxes[(col0 + a) * n_dir + j] = proj_box(D, dirs[j], a, M, bin, xr, yr);
}

// Box values of actuator a (blockIdx.x), direction j (blockIdx.y), row-major
// within the box, at vals[offs[(col0 + a) n_dir + j]].
__global__ void __launch_bounds__(kProjThreads)
k_proj_vals(const DevDM D, const ProjDir *__restrict__ dirs, const uint8_t *__restrict__ pupil, int M, int bin,
            int n_dir, long long col0, const long long *__restrict__ offs, float *__restrict__ vals) {
    const int a = blockIdx.x, j = blockIdx.y;
    __shared__ int4 sbox;
    __shared__ float sref[2];
    if (threadIdx.x == 0) {
        float xr, yr;
        sbox = proj_box(D, dirs[j], a, M, bin, xr, yr);
        sref[0] = xr;
        sref[1] = yr;
    }
    __syncthreads();
    const int4 box = sbox;
    const int w = box.w - box.z + 1, area = (box.y - box.x + 1) * w;
    if (box.y < box.x || area <= 0) return;
    const ProjDir pd = dirs[j];
    const float *win = D.win + (size_t)a * D.win_stride;
    float *dst = vals + offs[(col0 + a) * n_dir + j];
    for (int q = threadIdx.x; q < area; q += kProjThreads) {
        const int qi = box.x + q / w, qj = box.z + q % w;
        dst[q] = proj_value(D, win, pd, pupil, M, bin, box, sref[0], sref[1], qi, qj);
    }
}

// Products of the box-stored columns: out[l ld + a] = sum_j <col a, col l>
// over the intersection of their direction-j boxes, for every right column l
// whose union box meets left column a's (the others stay zero).  Right
// columns are bucketed by the top-left cell (cell x cell binned pixels) of
// their union box; every candidate is visited once.
struct BoxSet {
    const int4 *box;        // [cols][n_dir]
    const long long *off;   // [cols][n_dir] value offsets
    const float *val;
    const int4 *uni;        // [cols] union box over the directions (qi1 < qi0: empty)
};

__global__ void __launch_bounds__(kProjThreads)
k_box_dot(const BoxSet L, const BoxSet R, int n_dir, const int *__restrict__ cell_start,
          const int *__restrict__ cell_item, int cell, int n_cr, int n_cc, int max_h, int max_w, long long ld,
          float *__restrict__ out) {
    const int a = blockIdx.x;
    const int4 ua = L.uni[a];
    if (ua.y < ua.x) return;
    const int r0 = max(0, (ua.x - max_h + 1) / cell), r1 = min(n_cr - 1, ua.y / cell);
    const int c0 = max(0, (ua.z - max_w + 1) / cell), c1 = min(n_cc - 1, ua.w / cell);
    for (int r = r0; r <= r1; ++r)
        for (int c = c0; c <= c1; ++c) {
            const int cid = r * n_cc + c;
            for (int it = cell_start[cid] + threadIdx.x; it < cell_start[cid + 1]; it += kProjThreads) {
                const int l = cell_item[it];
                const int4 ul = R.uni[l];
                if (ul.x > ua.y || ul.y < ua.x || ul.z > ua.w || ul.w < ua.z) continue;
                float acc = 0.f;
                bool any = false;
                for (int j = 0; j < n_dir; ++j) {
                    const int4 A = L.box[(size_t)a * n_dir + j], B = R.box[(size_t)l * n_dir + j];
                    const int i0 = max(A.x, B.x), i1 = min(A.y, B.y), j0 = max(A.z, B.z), j1 = min(A.w, B.w);
                    if (i0 > i1 || j0 > j1 || A.y < A.x || B.y < B.x) continue;
                    any = true;
                    const int wa = A.w - A.z + 1, wb = B.w - B.z + 1;
                    const float *pa = L.val + L.off[(size_t)a * n_dir + j];
                    const float *pb = R.val + R.off[(size_t)l * n_dir + j];
                    for (int qi = i0; qi <= i1; ++qi) {
                        const float *ra = pa + (size_t)(qi - A.x) * wa, *rb = pb + (size_t)(qi - B.x) * wb;
                        for (int qj = j0; qj <= j1; ++qj) acc = fmaf(ra[qj - A.z], rb[qj - B.z], acc);
                    }
                }
                if (any) out[(size_t)l * ld + a] = acc;
            }
        }
}

__global__ void k_add_diag(float *__restrict__ G, long long n, float lam) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) G[i * n + i] += lam;
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

// Directions of one component (composite affine of each) into d_dirs.
cudaError_t upload_dirs(synim_ctx *ctx, int w, int d, int n_dir, const double *dirs, ProjDir *d_dirs,
                        cudaStream_t st) {
    std::vector<ProjDir> hd((size_t)n_dir);
    WfsHost view = ctx->wh[w];
    view.H = 0.0;
    view.rot = 0.0;
    view.mag[0] = view.mag[1] = 1.0;
    view.shift[0] = view.shift[1] = 0.0;
    for (int j = 0; j < n_dir; ++j) {
        view.th[0] = dirs[2 * j];
        view.th[1] = dirs[2 * j + 1];
        const synim_misreg m{0.0, 0.0, 0.0, 1.0};
        composite(ctx->dmh[d], view, m, hd[j].A, hd[j].b);
    }
    // pageable source: the copy is staged before the call returns
    return cudaMemcpyAsync(d_dirs, hd.data(), sizeof(ProjDir) * n_dir, cudaMemcpyHostToDevice, st);
}

// Box-stored projection columns of the listed components (columns in order):
// boxes, value offsets and values on the device, union boxes on both sides.
struct BoxBuild {
    BoxSet dev{};
    std::vector<int4> uni;
    long long cols = 0;
};

synim_status build_boxes(synim_ctx *ctx, int w, int n_dir, const double *dirs, int bin, int n_comp, const int *comps,
                         const uint8_t *d_pupil, ProjScratch &sc, BoxBuild &out, cudaStream_t st) {
    const int M = ctx->wh[w].M;
    const long long ncols = n_cols(ctx, n_comp, comps);
    out.cols = ncols;
    int4 *d_box = nullptr, *d_uni = nullptr;
    ProjDir *d_dirs = nullptr;
    long long *d_off = nullptr;
    float *d_val = nullptr;
    cudaError_t e = sc.alloc(&d_box, (size_t)ncols * n_dir);
    if (e == cudaSuccess) e = sc.alloc(&d_dirs, (size_t)n_comp * n_dir);
    if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_OOM, "projection boxes");
    long long col = 0;
    for (int c = 0; c < n_comp; ++c) {
        const int d = comps[c];
        const int n_act = ctx->dmh[d].n_act;
        if ((e = upload_dirs(ctx, w, d, n_dir, dirs, d_dirs + (size_t)c * n_dir, st)) != cudaSuccess) break;
        const long long n = (long long)n_act * n_dir;
        k_proj_boxes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctx->geo.dm[d], d_dirs + (size_t)c * n_dir, M, bin,
                                                                  n_act, n_dir, col, d_box);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        col += n_act;
    }
    std::vector<int4> hbox((size_t)ncols * n_dir);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hbox.data(), d_box, sizeof(int4) * hbox.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_CUDA, std::string("projection boxes: ") + cudaGetErrorString(e));
    std::vector<long long> hoff(hbox.size());
    out.uni.assign((size_t)ncols, make_int4(0, -1, 0, -1));
    long long total = 0;
    for (long long q = 0; q < ncols; ++q) {
        int4 u = make_int4(INT_MAX, INT_MIN, INT_MAX, INT_MIN);
        for (int j = 0; j < n_dir; ++j) {
            const int4 b = hbox[(size_t)q * n_dir + j];
            hoff[(size_t)q * n_dir + j] = total;
            if (b.y < b.x || b.w < b.z) continue;
            total += (long long)(b.y - b.x + 1) * (b.w - b.z + 1);
            u = make_int4(std::min(u.x, b.x), std::max(u.y, b.y), std::min(u.z, b.z), std::max(u.w, b.w));
        }
        if (u.x <= u.y) out.uni[(size_t)q] = u;
    }
    e = sc.alloc(&d_off, hoff.size());
    if (e == cudaSuccess) e = sc.alloc(&d_uni, (size_t)ncols);
    if (e == cudaSuccess) e = sc.alloc(&d_val, (size_t)std::max<long long>(total, 1));
    if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_OOM, "projection box values");
    e = cudaMemcpyAsync(d_off, hoff.data(), sizeof(long long) * hoff.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_uni, out.uni.data(), sizeof(int4) * out.uni.size(), cudaMemcpyHostToDevice, st);
    col = 0;
    for (int c = 0; c < n_comp && e == cudaSuccess; ++c) {
        const int d = comps[c];
        dim3 grid((unsigned)ctx->dmh[d].n_act, (unsigned)n_dir);
        k_proj_vals<<<grid, kProjThreads, 0, st>>>(ctx->geo.dm[d], d_dirs + (size_t)c * n_dir, d_pupil, M, bin, n_dir,
                                                   col, d_off, d_val);
        e = cudaGetLastError();
        col += ctx->dmh[d].n_act;
    }
    // the host vectors above must outlive the copies that read them
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_CUDA, std::string("projection box values: ") + cudaGetErrorString(e));
    out.dev = BoxSet{d_box, d_off, d_val, d_uni};
    return SYNIM_OK;
}

// Bucket grid of a column set by the top-left cell of each union box.
struct Buckets {
    int cell = 16, n_cr = 0, n_cc = 0, max_h = 1, max_w = 1;
    int *start = nullptr, *item = nullptr;
};

synim_status build_buckets(synim_ctx *ctx, const BoxBuild &bb, int Mb, ProjScratch &sc, Buckets &out,
                           cudaStream_t st, std::vector<int> &hstart, std::vector<int> &hitem) {
    out.n_cr = out.n_cc = (Mb + out.cell - 1) / out.cell;
    const size_t n_cells = (size_t)out.n_cr * out.n_cc;
    hstart.assign(n_cells + 1, 0);
    for (const int4 &u : bb.uni) {
        if (u.y < u.x) continue;
        ++hstart[(size_t)(u.x / out.cell) * out.n_cc + u.z / out.cell + 1];
        out.max_h = std::max(out.max_h, u.y - u.x + 1);
        out.max_w = std::max(out.max_w, u.w - u.z + 1);
    }
    for (size_t q = 0; q < n_cells; ++q) hstart[q + 1] += hstart[q];
    hitem.assign((size_t)std::max(hstart[n_cells], 1), 0);
    std::vector<int> fill(hstart.begin(), hstart.end() - 1);
    for (size_t l = 0; l < bb.uni.size(); ++l) {
        const int4 u = bb.uni[l];
        if (u.y < u.x) continue;
        hitem[(size_t)fill[(size_t)(u.x / out.cell) * out.n_cc + u.z / out.cell]++] = (int)l;
    }
    cudaError_t e = sc.alloc(&out.start, hstart.size());
    if (e == cudaSuccess) e = sc.alloc(&out.item, hitem.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.start, hstart.data(), sizeof(int) * hstart.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.item, hitem.data(), sizeof(int) * hitem.size(), cudaMemcpyHostToDevice, st);
    return e == cudaSuccess ? SYNIM_OK : pfail(ctx, SYNIM_ERR_OOM, "projection buckets");
}

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
    float *G = nullptr;
    int *info = nullptr;
    cudaError_t e = sc.alloc(&d_pupil, (size_t)M * M);
    if (e == cudaSuccess) e = sc.alloc(&G, (size_t)nd * nd);
    if (e == cudaSuccess) e = sc.alloc(&info, 2);
    if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pupil, ctx->pupil[wfs].data(), (size_t)M * M, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_OOM, std::string("projection scratch: ") + cudaGetErrorString(e));
    // box-stored columns of both sets, bucket grids of the right-hand sets
    BoxBuild bd, bl;
    if ((s = build_boxes(ctx, wfs, n_dir, dirs_rad, bin, n_dm, dms, d_pupil, sc, bd, st)) != SYNIM_OK) return s;
    if ((s = build_boxes(ctx, wfs, n_dir, dirs_rad, bin, n_layer, layers, d_pupil, sc, bl, st)) != SYNIM_OK) return s;
    Buckets kd, kl;
    std::vector<int> hs1, hi1, hs2, hi2;   // host copies outlive their uploads (synchronised below)
    const int Mb = M / bin;
    if ((s = build_buckets(ctx, bd, Mb, sc, kd, st, hs1, hi1)) != SYNIM_OK) return s;
    if ((s = build_buckets(ctx, bl, Mb, sc, kl, st, hs2, hi2)) != SYNIM_OK) return s;
    // R = P_DM^T P_Layer into p_opt, G = P_DM^T P_DM (both triangles)
    e = cudaMemsetAsync(p_opt, 0, sizeof(float) * (size_t)nd * nl, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, sizeof(float) * (size_t)nd * nd, st);
    if (e != cudaSuccess) return pfail(ctx, SYNIM_ERR_CUDA, std::string("projection: ") + cudaGetErrorString(e));
    k_box_dot<<<(unsigned)nd, kProjThreads, 0, st>>>(bd.dev, bl.dev, n_dir, kl.start, kl.item, kl.cell, kl.n_cr,
                                                      kl.n_cc, kl.max_h, kl.max_w, nd, p_opt);
    k_box_dot<<<(unsigned)nd, kProjThreads, 0, st>>>(bd.dev, bd.dev, n_dir, kd.start, kd.item, kd.cell, kd.n_cr,
                                                      kd.n_cc, kd.max_h, kd.max_w, nd, G);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return pfail(ctx, SYNIM_ERR_CUDA, std::string("k_box_dot: ") + cudaGetErrorString(e));
    // G + lambda I = L L^T (blocked Cholesky on the tensor cores), then
    // P_opt = (G + lambda I)^-1 R: p_opt is R column-major, i.e. R^T
    // row-major (n_layer x n_dm), and R^T G^-1 = (G^-1 R)^T in place
    k_add_diag<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(G, nd, (float)lambda);
    float *linvs = nullptr, *work = nullptr;
    const size_t wrows = (size_t)std::max<long long>(nd, nl);
    if ((e = sc.alloc(&linvs, (size_t)dense_blocks((int)nd) * 128 * 128)) != cudaSuccess ||
        (e = sc.alloc(&work, wrows * 128)) != cudaSuccess)
        return pfail(ctx, SYNIM_ERR_OOM, "projection solver workspace");
    if ((e = dense_potrf(G, nd, (int)nd, linvs, work, info, info + 1, st)) != cudaSuccess ||
        (e = dense_posolve_right(G, nd, (int)nd, linvs, p_opt, nd, (int)nl, work, info + 1, st)) != cudaSuccess)
        return pfail(ctx, SYNIM_ERR_CUDA, std::string("projection solve: ") + cudaGetErrorString(e));
    int h_info[2] = {0, 0};
    if ((e = cudaMemcpyAsync(h_info, info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return pfail(ctx, SYNIM_ERR_CUDA, std::string("projection: ") + cudaGetErrorString(e));
    if (h_info[1] != 0) return pfail(ctx, SYNIM_ERR_TIMEOUT, "projection: a tensor-core wait gave up");
    if (h_info[0] != 0)
        return pfail(ctx, SYNIM_ERR_NOT_CONVERGED,
                     "projection: P_DM^T P_DM + lambda I is not positive definite (raise lambda)");
    return SYNIM_OK;
}

}  // extern "C"
