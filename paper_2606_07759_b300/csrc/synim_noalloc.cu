// synim_noalloc.cu -- IM of one (DM, sensor) pair without any memory allocation.
//
// Who needs this: callers that must not allocate device memory while they
// run -- e.g. a real-time controller whose GPU memory is reserved once at
// start-up and may not grow, or a host framework whose pooled allocator owns
// all device memory, so a stray cudaMalloc would fail or fragment it.  The
// context API (synim_im_create) allocates its windows, tables and state maps;
// this entry point instead places every intermediate buffer in one fixed,
// file-scope device array, so it calls neither cudaMalloc nor cudaFree nor any
// allocating library routine, and uses no host heap either.
//
// It runs the same kernels as the context path (support scan, window packing,
// pixel classes, IM kernel) plus small kernels that build the sensor tables on
// the device.  The array lives on every GPU that loads the library until the
// process exits (SYNIM_NOALLOC_SCRATCH_BYTES).  All calls share it and it
// keeps the previous call's contents, so everything that must start at zero
// is cleared on each call, and two calls whose GPU work overlaps (different
// host threads or streams) race on it.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "synim.h"
#include "synim_internal.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[SYNIM_NOALLOC_SCRATCH_BYTES];

namespace synim {
namespace {

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;
thread_local char g_noalloc_error[256];

synim_status na_fail(synim_status s, const char *msg) {
    std::snprintf(g_noalloc_error, sizeof(g_noalloc_error), "%s", msg);
    return s;
}

__global__ void k_na_binarize(uint8_t *m, long n) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) m[q] = m[q] ? 1 : 0;
}

// Device address of the scratch array on the current device (looked up once
// per device; host code must not use the symbol itself as a pointer).
cudaError_t scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Header words at the start of the scratch.
enum { H_RESERVED = 0, H_ERR = 1, H_W = 2, H_NV = 3, H_NIRR = 4, H_WORDS = 64 };

struct Layout {
    size_t pair, box, org, dmmask, mcls, P, vin, lit, ros, vsub, vsj, fac, vrow, xcode, ycode, irrsr, irrsub,
        irrpix, irrw, irrc, irrcrow, pst, lines, win, fixed_end;
};

Layout make_layout(int n_act, int N, int M, int n, bool has_mask, bool has_vin) {
    const int k = M / n;
    Layout L{};
    size_t o = up256(sizeof(int) * H_WORDS);
    auto take = [&](size_t bytes) { const size_t at = o; o = up256(o + bytes); return at; };
    L.pair = take(sizeof(DevPair));
    L.box = take(sizeof(int) * (4 * (size_t)n_act + 1));
    L.org = take(sizeof(int) * 2 * (size_t)n_act);
    L.dmmask = has_mask ? take((size_t)N * N) : 0;
    L.mcls = take((size_t)(N + 1) * (N + 1));
    L.P = take((size_t)M * M);
    L.vin = has_vin ? take((size_t)n * n) : 0;
    L.lit = take(sizeof(int) * (size_t)n * n);
    L.ros = take(sizeof(int) * (size_t)n * n);
    L.vsub = take(sizeof(int) * (size_t)n * n);
    L.vsj = take(sizeof(short) * ((size_t)n * n + 4));
    L.fac = take(sizeof(float) * (size_t)n * n);
    L.vrow = take(sizeof(int) * (size_t)(n + 1));
    L.xcode = take((size_t)(n + 1) * M);
    L.ycode = take((size_t)(n + 1) * M);
    L.irrsr = take(sizeof(int) * ((size_t)n * n * k + 1));
    L.irrsub = take(sizeof(int) * ((size_t)n * n + 1));
    L.irrpix = take(sizeof(int) * (size_t)M * M);
    L.irrw = take(2 * (size_t)M * M);
    L.irrc = take(sizeof(int4) * (size_t)n * n);
    L.irrcrow = take(sizeof(int) * (size_t)(n + 1));
    L.pst = take((size_t)M * M);
    L.lines = take(2 * (size_t)M * (n + 1));
    L.win = o;
    L.fixed_end = o;
    return L;
}

// ---- sensor tables on the device (same rules as the context path) ----

__global__ void k_na_annulus(uint8_t *P, int M, double obstruction) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)M * M) return;
    const int i = (int)(q / M), j = (int)(q - (long)i * M);
    // the same FP64 expression as the context path: the squares of the
    // half-integer offsets and their sum are exact, and sqrt is correctly
    // rounded on host and device alike
    const double c = (M - 1) * 0.5, ro = M * 0.5, ri = obstruction * M * 0.5;
    const double dx = (double)j - c, dy = (double)i - c;
    const double r = sqrt(dx * dx + dy * dy);
    P[q] = (r <= ro && r >= ri) ? 1 : 0;
}

__global__ void k_na_lit(const uint8_t *P, int M, int n, int k, int *lit) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)M * M) return;
    const int i = (int)(q / M), j = (int)(q - (long)i * M);
    if (P[q]) atomicAdd(&lit[(i / k) * n + j / k], 1);
}

// One CTA: validity, row ranks (row-major), scale factors, first row per subaperture row.
__global__ void k_na_valid(const int *lit, const uint8_t *vin, int n, int k, double scale, double dw,
                           int *ros, int *vsub, short *vsj, float *fac, int *vrow, int *hdr) {
    __shared__ int cnt[1024];
    const int ns = n * n, T = blockDim.x, t = threadIdx.x;
    const int C = (ns + T - 1) / T, a = t * C, b = min(ns, a + C);
    int c = 0;
    for (int s = a; s < b; ++s) {
        const int l = lit[s];
        bool ok = vin ? vin[s] != 0 : (2 * l >= k * k);
        if (l == 0) ok = false;
        c += ok;
    }
    cnt[t] = c;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int q = 0; q < T; ++q) { const int v = cnt[q]; cnt[q] = run; run += v; }
        vrow[n] = run;
        hdr[H_NV] = run;
        for (int q = 0; q < 4; ++q) vsj[run + q] = -1;
    }
    __syncthreads();
    int r = cnt[t];
    for (int s = a; s < b; ++s) {
        const int si = s / n, sj = s - si * n;
        if (sj == 0) vrow[si] = r;
        const int l = lit[s];
        bool ok = vin ? vin[s] != 0 : (2 * l >= k * k);
        if (l == 0) ok = false;
        ros[s] = ok ? r : -1;
        if (ok) {
            vsub[r] = (si << 16) | sj;
            vsj[r] = (short)sj;
            fac[r] = (float)(scale / (2.0 * dw * l));
            ++r;
        }
    }
}

__device__ __forceinline__ int na_P(const uint8_t *P, int M, int i, int j) {
    return (i >= 0 && j >= 0 && i < M && j < M) ? P[(long)i * M + j] : 0;
}
__device__ __forceinline__ int na_V(const int *ros, int n, int si, int sj) {
    return (si >= 0 && sj >= 0 && si < n && sj < n) ? (ros[si * n + sj] >= 0) : 0;
}

__global__ void k_na_codes(const uint8_t *P, const int *ros, int M, int n, int k, uint8_t *xcode,
                           uint8_t *ycode) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)(n + 1) * M) return;
    const int b = (int)(q / M), x = (int)(q - (long)b * M);
    const int c0 = b * k - 1, c1 = b * k;
    {
        const int i = x, si = i / k;
        int code = 0;
        if (c0 >= 0) {
            if (na_P(P, M, i, c0 - 1) && na_V(ros, n, si, b - 1)) code |= 1;
            if (na_P(P, M, i, c0 + 1) && na_V(ros, n, si, b)) code |= 2;
        }
        if (c1 < M) {
            if (na_P(P, M, i, c1 - 1) && na_V(ros, n, si, b - 1)) code |= 4;
            if (na_P(P, M, i, c1 + 1) && na_V(ros, n, si, b)) code |= 8;
        }
        xcode[q] = (uint8_t)code;
    }
    {
        const int j = x, sj = j / k;
        int code = 0;
        if (c0 >= 0) {
            if (na_P(P, M, c0 - 1, j) && na_V(ros, n, b - 1, sj)) code |= 1;
            if (na_P(P, M, c0 + 1, j) && na_V(ros, n, b, sj)) code |= 2;
        }
        if (c1 < M) {
            if (na_P(P, M, c1 - 1, j) && na_V(ros, n, b - 1, sj)) code |= 4;
            if (na_P(P, M, c1 + 1, j) && na_V(ros, n, b, sj)) code |= 8;
        }
        ycode[q] = (uint8_t)code;
    }
}

__device__ __forceinline__ void na_irr_weights(const uint8_t *P, int M, int k, int i, int j, int si,
                                               int sj, int &wx, int &wy) {
    const int jm = j - sj * k, im = i - si * k;
    wx = (jm != 0 && jm != k - 1) ? na_P(P, M, i, j - 1) - na_P(P, M, i, j + 1) : 0;
    wy = (im != 0 && im != k - 1) ? na_P(P, M, i - 1, j) - na_P(P, M, i + 1, j) : 0;
}

// Irregular pixels, counted per (subaperture, pixel row inside it).
__global__ void k_na_irr_count(const uint8_t *P, const int *ros, int M, int n, int k, int *irrsr) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)n * n * k) return;
    const int s = (int)(q / k), r = (int)(q - (long)s * k);
    int c = 0;
    if (ros[s] >= 0) {
        const int si = s / n, sj = s - si * n, i = si * k + r;
        for (int j = sj * k; j < (sj + 1) * k; ++j) {
            int wx, wy;
            na_irr_weights(P, M, k, i, j, si, sj, wx, wy);
            c += (wx || wy);
        }
    }
    irrsr[q] = c;
}

// One CTA: exclusive scan of the (subaperture, row) counts -> write offsets.
__global__ void k_na_irr_scan(int *irrsr, int n, int k, int *irr_sub, int *hdr) {
    __shared__ int cnt[1024];
    const long tot = (long)n * n * k;
    const int T = blockDim.x, t = threadIdx.x;
    const long C = (tot + T - 1) / T, a = t * C, b = min(tot, a + C);
    int c = 0;
    for (long q = a; q < b; ++q) c += irrsr[q];
    cnt[t] = c;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int q = 0; q < T; ++q) { const int v = cnt[q]; cnt[q] = run; run += v; }
        irr_sub[n * n] = run;
        irrsr[tot] = run;
        hdr[H_NIRR] = run;
    }
    __syncthreads();
    int run = cnt[t];
    for (long q = a; q < b; ++q) {
        const int v = irrsr[q];
        irrsr[q] = run;
        if (q % k == 0) irr_sub[q / k] = run;
        run += v;
    }
}

__global__ void k_na_irr_fill(const uint8_t *P, const int *ros, int M, int n, int k, const int *irrsr,
                              int *irr_pix, int8_t *irr_w) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)n * n * k) return;
    const int s = (int)(q / k), r = (int)(q - (long)s * k);
    if (ros[s] < 0) return;
    const int si = s / n, sj = s - si * n, i = si * k + r;
    int at = irrsr[q];
    for (int j = sj * k; j < (sj + 1) * k; ++j) {
        int wx, wy;
        na_irr_weights(P, M, k, i, j, si, sj, wx, wy);
        if (wx || wy) {
            irr_pix[at] = (i << 16) | j;
            irr_w[2 * at] = (int8_t)wx;
            irr_w[2 * at + 1] = (int8_t)wy;
            ++at;
        }
    }
}

// One thread: subapertures with pupil-edge pixels, grouped by subaperture row.
__global__ void k_na_irr_cand(const int *irr_sub, int n, int4 *irrc, int *irrc_row) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int q = 0;
    for (int si = 0; si < n; ++si) {
        irrc_row[si] = q;
        for (int sj = 0; sj < n; ++sj) {
            const int e0 = irr_sub[si * n + sj], e1 = irr_sub[si * n + sj + 1];
            if (e1 > e0) irrc[q++] = make_int4(sj, e0, e1, 0);
        }
    }
    irrc_row[n] = q;
}

// ---- support windows ----
__global__ void k_na_wmax(const int *box, int n_act, int *hdr) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_act) return;
    const int *bx = box + 4 * a;
    if (bx[1] < bx[0]) return;
    atomicMax(&hdr[H_W], max(bx[1] - bx[0] + 1, bx[3] - bx[2] + 1));
}

__global__ void k_na_org(const int *box, int n_act, int N, int W, int *org) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_act) return;
    const int *bx = box + 4 * a;
    int x0 = 0, y0 = 0;
    if (bx[1] >= bx[0]) {
        x0 = max(0, min(bx[0], N - W));
        y0 = max(0, min(bx[2], N - W));
    }
    org[2 * a] = x0;
    org[2 * a + 1] = y0;
}

inline unsigned grid_for(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace synim

using namespace synim;

namespace synim {
const char *noalloc_last_error() { return g_noalloc_error; }
}  // namespace synim

extern "C" synim_status synim_im_compute_noalloc(const synim_dm_desc *dm, const synim_wfs_desc *wfs,
                                                 const synim_misreg *mis, float *im, int64_t *n_rows,
                                                 void *cuda_stream) {
    g_noalloc_error[0] = '\0';
    clear_create_error();
    if (!dm || !wfs || !mis) return na_fail(SYNIM_ERR_INVALID_ARG, "dm, wfs and mis must not be NULL");
    if (!dm->ifs || dm->ifs_on_device != 1)
        return na_fail(SYNIM_ERR_INVALID_ARG, "the IF cube must already be on the device (ifs_on_device = 1)");
    if (dm->n_act < 1 || dm->grid_n < 4 || dm->grid_n > 32767 || !(dm->pixel_pitch_m > 0) ||
        !(dm->altitude_m >= 0) || !(dm->support_eps >= 0))
        return na_fail(SYNIM_ERR_INVALID_ARG, "invalid DM descriptor");
    if (wfs->n_sub < 1 || wfs->grid_m < 2 || wfs->grid_m > 32767 || !(wfs->pupil_diam_m > 0) ||
        !(wfs->mag[0] != 0) || !(wfs->mag[1] != 0))
        return na_fail(SYNIM_ERR_INVALID_ARG, "invalid sensor descriptor");
    if (wfs->grid_m % wfs->n_sub != 0 || wfs->grid_m / wfs->n_sub < 2)
        return na_fail(SYNIM_ERR_SHAPE, "grid_m must be k * n_sub with k >= 2");
    if (!(mis->mag > 0) || !std::isfinite(mis->shift_x_px) || !std::isfinite(mis->shift_y_px) ||
        !std::isfinite(mis->rot_deg) || !std::isfinite(mis->mag))
        return na_fail(SYNIM_ERR_INVALID_ARG, "invalid misregistration");

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return na_fail(SYNIM_ERR_CUDA, "no current device");
    unsigned char *base = nullptr;
    if ((e = scratch_address(dev, &base)) != cudaSuccess)
        return na_fail(SYNIM_ERR_CUDA, "cudaGetSymbolAddress failed for the scratch array");

    const int n_act = dm->n_act, N = dm->grid_n, M = wfs->grid_m, n = wfs->n_sub, k = M / n;
    const Layout L = make_layout(n_act, N, M, n, dm->mask != nullptr, wfs->subap_valid != nullptr);
    char msg[200];
    if (L.fixed_end > (size_t)SYNIM_NOALLOC_SCRATCH_BYTES) {
        std::snprintf(msg, sizeof(msg), "tables need %zu bytes, more than the %u-byte scratch",
                      L.fixed_end, (unsigned)SYNIM_NOALLOC_SCRATCH_BYTES);
        return na_fail(SYNIM_ERR_SHAPE, msg);
    }
    int *hdr = reinterpret_cast<int *>(base);
    auto ptr = [&](size_t off) { return base + off; };
    const double dw = wfs->pupil_diam_m / M;
    // clear what accumulates; copy the host masks into the scratch
    e = cudaMemsetAsync(hdr, 0, sizeof(int) * H_WORDS, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ptr(L.lit), 0, sizeof(int) * (size_t)n * n, st);
    if (e == cudaSuccess && dm->mask) e = cudaMemcpyAsync(ptr(L.dmmask), dm->mask, (size_t)N * N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && wfs->pupil_mask)
        e = cudaMemcpyAsync(ptr(L.P), wfs->pupil_mask, (size_t)M * M, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && wfs->subap_valid)
        e = cudaMemcpyAsync(ptr(L.vin), wfs->subap_valid, (size_t)n * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return na_fail(SYNIM_ERR_CUDA, "scratch initialisation failed");
    uint8_t *P = reinterpret_cast<uint8_t *>(ptr(L.P));
    int *lit = reinterpret_cast<int *>(ptr(L.lit)), *ros = reinterpret_cast<int *>(ptr(L.ros));
    int *vsub = reinterpret_cast<int *>(ptr(L.vsub)), *vrow = reinterpret_cast<int *>(ptr(L.vrow));
    short *vsj = reinterpret_cast<short *>(ptr(L.vsj));
    float *fac = reinterpret_cast<float *>(ptr(L.fac));
    uint8_t *xcode = ptr(L.xcode), *ycode = ptr(L.ycode);
    int *irrsr = reinterpret_cast<int *>(ptr(L.irrsr)), *irrsub = reinterpret_cast<int *>(ptr(L.irrsub));
    int *irrpix = reinterpret_cast<int *>(ptr(L.irrpix));
    int8_t *irrw = reinterpret_cast<int8_t *>(ptr(L.irrw));
    int *box = reinterpret_cast<int *>(ptr(L.box)), *org = reinterpret_cast<int *>(ptr(L.org));
    // binary masks: any non-zero byte counts as 1, as in the context path
    const long MM = (long)M * M;
    if (!wfs->pupil_mask) k_na_annulus<<<grid_for(MM, 256), 256, 0, st>>>(P, M, wfs->obstruction);
    else k_na_binarize<<<grid_for(MM, 256), 256, 0, st>>>(P, MM);
    if (dm->mask) k_na_binarize<<<grid_for((long)N * N, 256), 256, 0, st>>>(ptr(L.dmmask), (long)N * N);
    k_na_lit<<<grid_for(MM, 256), 256, 0, st>>>(P, M, n, k, lit);
    k_na_valid<<<1, 1024, 0, st>>>(lit, wfs->subap_valid ? ptr(L.vin) : nullptr, n, k, wfs->slope_scale, dw,
                                   ros, vsub, vsj, fac, vrow, hdr);
    k_na_codes<<<grid_for((long)(n + 1) * M, 256), 256, 0, st>>>(P, ros, M, n, k, xcode, ycode);
    k_na_irr_count<<<grid_for((long)n * n * k, 256), 256, 0, st>>>(P, ros, M, n, k, irrsr);
    k_na_irr_scan<<<1, 1024, 0, st>>>(irrsr, n, k, irrsub, hdr);
    k_na_irr_fill<<<grid_for((long)n * n * k, 256), 256, 0, st>>>(P, ros, M, n, k, irrsr, irrpix, irrw);
    int4 *irrc = reinterpret_cast<int4 *>(ptr(L.irrc));
    int *irrcrow = reinterpret_cast<int *>(ptr(L.irrcrow));
    k_na_irr_cand<<<1, 32, 0, st>>>(irrsub, n, irrc, irrcrow);
    int h[H_WORDS];
    if (!im) {
        // size query: the row count needs only the sensor tables
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(h, hdr, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return na_fail(SYNIM_ERR_CUDA, cudaGetErrorString(e));
        if (n_rows) *n_rows = 2LL * h[H_NV];
        if (h[H_NV] == 0) return na_fail(SYNIM_ERR_SHAPE, "sensor has no valid subaperture");
        return SYNIM_OK;
    }
    uint8_t *mcls = ptr(L.mcls);
    if ((e = launch_mcls(dm->mask ? ptr(L.dmmask) : nullptr, N, mcls, st)) != cudaSuccess)
        return na_fail(SYNIM_ERR_CUDA, "mask interior map launch failed");
    // support windows
    if ((e = launch_support(dm->ifs, n_act, N, dm->support_eps, box, st)) != cudaSuccess)
        return na_fail(SYNIM_ERR_CUDA, "support scan launch failed");
    k_na_wmax<<<grid_for(n_act, 256), 256, 0, st>>>(box, n_act, hdr);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(h, hdr, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return na_fail(SYNIM_ERR_CUDA, cudaGetErrorString(e));
    const int nv = h[H_NV];
    if (n_rows) *n_rows = 2LL * nv;
    if (nv == 0) return na_fail(SYNIM_ERR_SHAPE, "sensor has no valid subaperture");
    const int W = std::min(std::max(h[H_W], 1), N);
    int Wp = W + 2;
    if ((Wp & 1) == 0) ++Wp;
    const int stride = (Wp * Wp + 3) / 4 * 4;
    const size_t need = L.win + sizeof(float) * (size_t)stride * n_act;
    if (need > (size_t)SYNIM_NOALLOC_SCRATCH_BYTES) {
        std::snprintf(msg, sizeof(msg),
                      "%d support windows of %d x %d px need %zu bytes, more than the %u-byte scratch",
                      n_act, W, W, need, (unsigned)SYNIM_NOALLOC_SCRATCH_BYTES);
        return na_fail(SYNIM_ERR_SHAPE, msg);
    }
    float *win = reinterpret_cast<float *>(ptr(L.win));
    k_na_org<<<grid_for(n_act, 256), 256, 0, st>>>(box, n_act, N, W, org);
    if ((e = launch_pack(dm->ifs, n_act, N, org, W, Wp, stride, win, st)) != cudaSuccess)
        return na_fail(SYNIM_ERR_CUDA, "window packing launch failed");
    // geometry of the pair (host, FP64) and the kernel parameters
    DmHost Dh;
    Dh.n_act = n_act; Dh.N = N; Dh.W = W; Dh.Wp = Wp; Dh.dd = dm->pixel_pitch_m; Dh.h = dm->altitude_m;
    WfsHost Wh;
    Wh.n_sub = n; Wh.M = M; Wh.k = k; Wh.nv = nv; Wh.CH = largest_divisor_le(k, 32);
    Wh.D = wfs->pupil_diam_m; Wh.H = wfs->src_height_m;
    Wh.th[0] = wfs->field_rad[0]; Wh.th[1] = wfs->field_rad[1];
    Wh.rot = wfs->rot_deg; Wh.mag[0] = wfs->mag[0]; Wh.mag[1] = wfs->mag[1];
    Wh.shift[0] = wfs->shift_m[0]; Wh.shift[1] = wfs->shift_m[1]; Wh.scale = wfs->slope_scale;
    DevPair pair;
    std::memset(&pair, 0, sizeof(pair));
    composite(Dh, Wh, *mis, pair.A, pair.b);
    if (!invert2(pair.A, pair.Ai)) return na_fail(SYNIM_ERR_INVALID_ARG, "singular composite affine");
    composite_jac(Dh, *mis, pair.A, pair.b, pair.dA, pair.db);
    split_pair(pair);
    pair.im = im;
    pair.pst = ptr(L.pst);
    pair.xcc = ptr(L.lines);
    pair.ycc = pair.xcc + (size_t)M * (n + 1);
    pair.vec4 = ((2 * nv) % 4 == 0 && (reinterpret_cast<uintptr_t>(im) & 15u) == 0) ? 1 : 0;
    const long long seg = (seg_need(Dh, Wh, pair.Ai, 1) + 3) / 4 * 4;
    DevPair *d_pair = reinterpret_cast<DevPair *>(ptr(L.pair));
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    if ((e = cudaMemcpyAsync(d_pair, &pair, sizeof(pair), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return na_fail(SYNIM_ERR_CUDA, "parameter upload failed");
    Geo g;
    std::memset(&g, 0, sizeof(g));
    DevDM &G = g.dm[0];
    G.win = win; G.org = org; G.mask = dm->mask ? ptr(L.dmmask) : nullptr; G.mcls = mcls;
    G.n_act = n_act; G.N = N; G.W = W; G.Wp = Wp; G.win_stride = stride;
    DevWFS &F = g.wfs[0];
    F.xcode = xcode; F.ycode = ycode; F.irr_pix = irrpix; F.irr_w = irrw; F.irr_sub = irrsub;
    F.fac = fac; F.vsub = vsub; F.vrow = vrow; F.irrc = irrc; F.irrc_row = irrcrow; F.irr_sr = irrsr; F.vsj = vsj; F.vidx = ros;
    F.n_sub = n; F.M = M; F.k = k; F.nv = nv; F.CH = Wh.CH;
    F.n_irr = M * M;   // the capacity of irr_pix in the layout
    g.n_dm = 1; g.n_wfs = 1; g.n_items = n_act;
    g.order_dm[0] = 0; g.order_start[0] = 0; g.order_start[1] = n_act;
    g.seg_floats = (int)seg;
    const size_t smem = im_smem_bytes(g, 256);
    int dev_max = 0, n_sm = 0, bps = 0;
    cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (smem > (size_t)dev_max) return na_fail(SYNIM_ERR_SHAPE, "boundary segments exceed the shared memory of a CTA");
    if ((e = im_prepare(MODE_FWD, 256, smem, &bps)) != cudaSuccess || bps < 1)
        return na_fail(SYNIM_ERR_CUDA, "IM kernel attributes");
    const int grid = std::max(1, std::min(n_act, n_sm * bps));
    if ((e = cudaMemsetAsync(hdr, 0, 2 * sizeof(int), st)) != cudaSuccess ||
        (e = launch_pst(g, d_pair, M * M, M * (n + 1), st)) != cudaSuccess ||
        (e = launch_im(MODE_FWD, g, d_pair, hdr + H_ERR, nullptr, grid, 256, smem, st)) != cudaSuccess)
        return na_fail(SYNIM_ERR_CUDA, cudaGetErrorString(e));
    int err_flag = 0;
    if ((e = cudaMemcpyAsync(&err_flag, hdr + H_ERR, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return na_fail(SYNIM_ERR_CUDA, cudaGetErrorString(e));
    if (err_flag & ERR_TIMEOUT) return na_fail(SYNIM_ERR_TIMEOUT, "a bounded device wait timed out");
    if (err_flag & ERR_ARENA) return na_fail(SYNIM_ERR_SHAPE, "slope values exceeded their shared-memory buffer");
    if (err_flag & ERR_BOUNDS) return na_fail(SYNIM_ERR_BOUNDS, "an IM kernel index left its buffer (access skipped)");
    return SYNIM_OK;
}
