// synim_kernels.cu -- sm_103a kernels of the synthetic interaction-matrix path.
//
// k_support / k_pack  (create time) scan each influence function for its
//                     support box and pack it into a zero-bordered window.
// k_pst_core / _ring  (every call) edge-repair pixel classes per pair,
//                     Sec. 2.3 steps 1-2: the DM mask carried by the composite
//                     affine, strictly binarised at 0.999999 (decided in FP64,
//                     exactly as the definition), and the cross-dilated ring.
// k_im<MODE>          (every call) one persistent launch over all actuators of
//                     all DMs; each CTA stages one actuator's window into
//                     shared memory with a 1-D bulk copy (TMA) and reuses it
//                     for every sensor (Sec. 4.2: each IF fetched once).  For
//                     each sensor it resamples the IF (Sec. 2.1), repairs the
//                     ring (Sec. 2.3) and forms the subaperture means of the
//                     central differences (Sec. 2.2), then streams the full
//                     dense column out with 16-byte stores.
//
// The subaperture sum of central differences is evaluated in telescoped
// form: sum_{p in s} P(p) (phi(p+x) - phi(p-x)) = sum_q phi(q) w_s(q) where
// w_s(q) = P(q-x)[q-x in s] - P(q+x)[q+x in s] is non-zero only on the two
// pixel columns at each subaperture boundary and where the pupil edge cuts a
// subaperture.  This is the same sum, reordered; only those pixels are
// resampled.
#include <cfloat>
#include <climits>

#include "synim_internal.h"

namespace synim {

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier + 1-D bulk copy global -> shared (TMA unit)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~2^31 clocks (about a second) instead of hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------
template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T ident) {
    __shared__ T red[32];
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : ident;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (threadIdx.x == 0) red[0] = v;
    __syncthreads();
    return red[0];
}

struct MaxF { __device__ float operator()(float a, float b) const { return fmaxf(a, b); } };
struct MinI { __device__ int operator()(int a, int b) const { return min(a, b); } };
struct MaxI { __device__ int operator()(int a, int b) const { return max(a, b); } };

// ---------------------------------------------------------------------------
// Create time: support box and window packing
// ---------------------------------------------------------------------------
// box[a] = {x0, x1, y0, y1} of |IF_a| > eps * max|IF_a| (x1 < x0 if empty).
__global__ void k_support(const float *__restrict__ cube, int N, float eps, int *__restrict__ box) {
    const int a = blockIdx.x;
    const size_t NN = (size_t)N * N;
    const float *img = cube + (size_t)a * NN;
    float m = 0.f;
    for (size_t p = threadIdx.x; p < NN; p += blockDim.x) m = fmaxf(m, fabsf(img[p]));
    m = block_reduce(m, MaxF(), 0.f);
    const float thr = eps * m;
    int x0 = INT_MAX, x1 = -1, y0 = INT_MAX, y1 = -1;
    for (size_t p = threadIdx.x; p < NN; p += blockDim.x) {
        if (fabsf(img[p]) > thr) {
            const int y = (int)(p / N), x = (int)(p - (size_t)y * N);
            x0 = min(x0, x); x1 = max(x1, x); y0 = min(y0, y); y1 = max(y1, y);
        }
    }
    x0 = block_reduce(x0, MinI(), INT_MAX);
    x1 = block_reduce(x1, MaxI(), -1);
    y0 = block_reduce(y0, MinI(), INT_MAX);
    y1 = block_reduce(y1, MaxI(), -1);
    if (threadIdx.x == 0) {
        box[4 * a + 0] = x0; box[4 * a + 1] = x1; box[4 * a + 2] = y0; box[4 * a + 3] = y1;
    }
}

// win[a][r][c] = IF_a(wy0 + r - 1, wx0 + c - 1) for 1 <= r, c <= W, zero elsewhere.
__global__ void k_pack(const float *__restrict__ cube, int N, const int *__restrict__ org, int W,
                       int Wp, int stride, float *__restrict__ win) {
    const int a = blockIdx.x;
    const int wx0 = org[2 * a], wy0 = org[2 * a + 1];
    const float *img = cube + (size_t)a * N * N;
    float *dst = win + (size_t)a * stride;
    for (int idx = threadIdx.x; idx < stride; idx += blockDim.x) {
        float v = 0.f;
        const int r = idx / Wp, c = idx - r * Wp;
        if (idx < Wp * Wp && r >= 1 && r <= W && c >= 1 && c <= W) {
            const int x = wx0 + c - 1, y = wy0 + r - 1;
            if (x >= 0 && x < N && y >= 0 && y < N) v = img[(size_t)y * N + x];
        }
        dst[idx] = v;
    }
}

cudaError_t launch_support(const float *cube, int n_act, int N, float eps, int *box,
                           cudaStream_t s) {
    k_support<<<n_act, 256, 0, s>>>(cube, N, eps, box);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float *cube, int n_act, int N, const int *org, int W, int Wp,
                        int stride, float *win, cudaStream_t s) {
    k_pack<<<n_act, 256, 0, s>>>(cube, N, org, W, Wp, stride, win);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Every call: pixel classes (Sec. 2.3 steps 1-2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int mask_tap(const uint8_t *__restrict__ mask, int N, long x, long y) {
    if (x < 0 || y < 0 || x >= N || y >= N) return 0;
    return mask ? (int)mask[y * (long)N + x] : 1;
}

// Strict core: bilinear(DM mask) >= 0.999999 at the composite-affine image of
// each sensor pixel.  The decision is taken in FP64 with the operations of
// the definition (no contraction); an FP32 pre-test settles the cells whose
// four taps agree and whose fractional position is far from an integer.
__global__ void k_pst_core(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs) {
    const int p = blockIdx.y;
    const int d = p / g.n_wfs, w = p - d * g.n_wfs;
    const int M = g.wfs[w].M;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)M * M) return;
    uint8_t *pst = pairs[p].pst;
    if (!pst) return;
    const int i = (int)(idx / M), j = (int)(idx - (long)i * M);
    const int N = g.dm[d].N;
    const uint8_t *mask = g.dm[d].mask;
    const double *A = pairs[p].A, *b = pairs[p].b;
    const float xf = fmaf((float)A[0], (float)j, fmaf((float)A[1], (float)i, (float)b[0]));
    const float yf = fmaf((float)A[2], (float)j, fmaf((float)A[3], (float)i, (float)b[1]));
    const float fx0 = floorf(xf), fy0 = floorf(yf);
    const float fxf = xf - fx0, fyf = yf - fy0;
    int core;
    if (fxf > 0.01f && fxf < 0.99f && fyf > 0.01f && fyf < 0.99f && fabsf(xf) < 1e6f &&
        fabsf(yf) < 1e6f) {
        // FP32 coordinate error < 1e-3 px here, so the cell is certain; every
        // weight is > 1e-4, so any zero tap puts the mask below 0.999999.
        const long ix = (long)fx0, iy = (long)fy0;
        core = mask_tap(mask, N, ix, iy) & mask_tap(mask, N, ix + 1, iy) &
               mask_tap(mask, N, ix, iy + 1) & mask_tap(mask, N, ix + 1, iy + 1);
    } else {
        const double x = __dadd_rn(__dadd_rn(__dmul_rn(A[0], (double)j), __dmul_rn(A[1], (double)i)), b[0]);
        const double y = __dadd_rn(__dadd_rn(__dmul_rn(A[2], (double)j), __dmul_rn(A[3], (double)i)), b[1]);
        const double x0 = floor(x), y0 = floor(y);
        const double fx = __dsub_rn(x, x0), fy = __dsub_rn(y, y0);
        const double gx = __dsub_rn(1.0, fx), gy = __dsub_rn(1.0, fy);
        const long ix = (long)x0, iy = (long)y0;
        double m = __dmul_rn(__dmul_rn(gx, gy), (double)mask_tap(mask, N, ix, iy));
        m = __dadd_rn(m, __dmul_rn(__dmul_rn(fx, gy), (double)mask_tap(mask, N, ix + 1, iy)));
        m = __dadd_rn(m, __dmul_rn(__dmul_rn(gx, fy), (double)mask_tap(mask, N, ix, iy + 1)));
        m = __dadd_rn(m, __dmul_rn(__dmul_rn(fx, fy), (double)mask_tap(mask, N, ix + 1, iy + 1)));
        core = (m >= 0.999999) ? 1 : 0;
    }
    pst[idx] = (uint8_t)core;
}

// Ring: non-core pixels with a core 4-neighbour.  Only 0 -> 2 transitions are
// written and only "== 1" is read, so the in-place update is race-free.
__global__ void k_pst_ring(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs) {
    const int p = blockIdx.y;
    const int w = p % g.n_wfs;
    const int M = g.wfs[w].M;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)M * M) return;
    uint8_t *pst = pairs[p].pst;
    if (!pst || pst[idx] != 0) return;
    const int i = (int)(idx / M), j = (int)(idx - (long)i * M);
    const bool ring = (j + 1 < M && pst[idx + 1] == 1) || (j >= 1 && pst[idx - 1] == 1) ||
                      (i + 1 < M && pst[idx + M] == 1) || (i >= 1 && pst[idx - M] == 1);
    if (ring) pst[idx] = 2;
}

cudaError_t launch_pst(const Geo &g, const DevPair *pairs, int max_mm, cudaStream_t s) {
    dim3 grid((max_mm + 255) / 256, g.n_dm * g.n_wfs);
    k_pst_core<<<grid, 256, 0, s>>>(g, pairs);
    k_pst_ring<<<grid, 256, 0, s>>>(g, pairs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The IM kernel
// ---------------------------------------------------------------------------
struct ItemWfs {
    int pi0, pi1, pj0, pj1;  // pixel box where phi may be non-zero (inclusive)
    int si0, si1, sj0, sj1;  // subapertures whose slopes may be non-zero (inclusive)
    int nxc, nb, nyc, nbr;   // row chunks x column boundaries; column chunks x row boundaries
    int ntask, need, arena, empty;
    float xo, yo;            // padded-window coordinates of pixel (pi0, pj0)
    float a00, a01, a10, a11;
    float dxo[4], dyo[4], da[16];  // tangents of the coordinates (MODE_TAN / MODE_VJP)
    const uint8_t *pst;
};

template <int NV>
struct Eval {
    const float *win;
    const uint8_t *pst;
    int Wp, M, pi0, pj0;
    float Wf1, xo, yo, a00, a01, a10, a11;
    float dxo[4], dyo[4], da[16];

    __device__ __forceinline__ void load(const ItemWfs &s, const float *w, int wp, int W, int m) {
        win = w; pst = s.pst; Wp = wp; M = m; pi0 = s.pi0; pj0 = s.pj0;
        Wf1 = (float)(W + 1); xo = s.xo; yo = s.yo;
        a00 = s.a00; a01 = s.a01; a10 = s.a10; a11 = s.a11;
        if (NV == 5) {
#pragma unroll
            for (int k = 0; k < 4; ++k) { dxo[k] = s.dxo[k]; dyo[k] = s.dyo[k]; }
#pragma unroll
            for (int k = 0; k < 16; ++k) da[k] = s.da[k];
        }
    }

    // Bilinear resample of the staged window at sensor pixel (i, j) (Sec. 2.1);
    // v[0] = phi, v[1..4] = d phi / d p_k (chain rule through the floor cell).
    __device__ __forceinline__ void bil(int i, int j, float *v) const {
        const float di = (float)(i - pi0), dj = (float)(j - pj0);
        const float x = fmaf(a00, dj, fmaf(a01, di, xo));
        const float y = fmaf(a10, dj, fmaf(a11, di, yo));
        if (!(x > 0.f && x < Wf1 && y > 0.f && y < Wf1)) {
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = 0.f;
            return;
        }
        const float fx0 = floorf(x), fy0 = floorf(y);
        const int ix = (int)fx0, iy = (int)fy0;
        const float fx = x - fx0, fy = y - fy0;
        const float *q = win + iy * Wp + ix;
        const float v00 = q[0], v10 = q[1], v01 = q[Wp], v11 = q[Wp + 1];
        const float ex = v10 - v00, ex1 = v11 - v01;
        const float top = fmaf(fx, ex, v00), bot = fmaf(fx, ex1, v01);
        v[0] = fmaf(fy, bot - top, top);
        if (NV == 5) {
            const float gx = fmaf(fy, ex1 - ex, ex), gy = bot - top;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float dx = fmaf(da[4 * k + 0], dj, fmaf(da[4 * k + 1], di, dxo[k]));
                const float dy = fmaf(da[4 * k + 2], dj, fmaf(da[4 * k + 3], di, dyo[k]));
                v[1 + k] = fmaf(gx, dx, gy * dy);
            }
        }
    }

    // Edge repair step 3 (Sec. 2.3) at a ring pixel.
    __device__ void ring(int i, int j, float *v) const {
        float acc[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) acc[t] = 0.f;
        int n = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int di = (d == 2) ? 1 : (d == 3 ? -1 : 0);
            const int dj = (d == 0) ? 1 : (d == 1 ? -1 : 0);
            const int i1 = i + di, j1 = j + dj;
            if (i1 < 0 || i1 >= M || j1 < 0 || j1 >= M) continue;
            if (pst[i1 * M + j1] != 1) continue;
            float v1[NV];
            bil(i1, j1, v1);
            const int i2 = i1 + di, j2 = j1 + dj;
            if (i2 >= 0 && i2 < M && j2 >= 0 && j2 < M && pst[i2 * M + j2] == 1) {
                float v2[NV];
                bil(i2, j2, v2);
#pragma unroll
                for (int t = 0; t < NV; ++t) acc[t] += 2.f * v1[t] - v2[t];
            } else {
#pragma unroll
                for (int t = 0; t < NV; ++t) acc[t] += v1[t];
            }
            ++n;
        }
        const float inv = n ? 1.f / (float)n : 0.f;
#pragma unroll
        for (int t = 0; t < NV; ++t) v[t] = acc[t] * inv;
    }

    // Repaired phase (and tangents) at sensor pixel (i, j).
    __device__ __forceinline__ void eval(int i, int j, float *v) const {
        const int st = pst[i * M + j];
        if (st == 1) {
            bil(i, j, v);
            return;
        }
        if (st == 0) {
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = 0.f;
            return;
        }
        ring(i, j, v);
    }
};

__device__ __forceinline__ void decode_item(const Geo &g, int item, int &d, int &a) {
    int pos = 0;
    while (pos + 1 < g.n_dm && item >= g.order_start[pos + 1]) ++pos;
    d = g.order_dm[pos];
    a = item - g.order_start[pos];
}

__device__ __forceinline__ void issue_window(const Geo &g, int item, float *s_win, uint32_t bar) {
    int d, a;
    decode_item(g, item, d, a);
    const DevDM &D = g.dm[d];
    const uint32_t bytes = (uint32_t)D.win_stride * 4u;
    mbar_expect_tx(bar, bytes);
    bulk_g2s(smem_u32(s_win), D.win + (size_t)a * D.win_stride, bytes, bar);
}

template <int MODE>
__device__ __forceinline__ bool pair_active(const DevPair &P) {
    if (MODE == MODE_FWD) return P.im != nullptr;
    if (MODE == MODE_TAN)
        return P.im || P.dim[0] || P.dim[1] || P.dim[2] || P.dim[3];
    return P.gim != nullptr;
}

// Pixel box of actuator a on sensor w, task counts and local coordinates.
template <int MODE, int NV>
__device__ void make_info(const Geo &g, const DevPair *__restrict__ pairs, int d, int a, int w,
                          ItemWfs &s) {
    const DevPair &P = pairs[d * g.n_wfs + w];
    const DevWFS &WF = g.wfs[w];
    const DevDM &D = g.dm[d];
    const int M = WF.M, k = WF.k, CH = WF.CH;
    s.pst = P.pst;
    s.empty = 1;
    s.ntask = 0;
    s.need = 0;
    s.si0 = 1; s.si1 = 0; s.sj0 = 1; s.sj1 = 0;
    s.pi0 = 1; s.pi1 = 0; s.pj0 = 1; s.pj1 = 0;
    if (!pair_active<MODE>(P)) return;
    const int wx0 = D.org[2 * a], wy0 = D.org[2 * a + 1];
    // Cells that touch the window: x in (wx0 - 1, wx0 + W), y likewise.
    double jmin = 1e300, jmax = -1e300, imin = 1e300, imax = -1e300;
#pragma unroll
    for (int cx = 0; cx < 2; ++cx)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            const double dx = (cx ? (double)(wx0 + D.W) : (double)(wx0 - 1)) - P.b[0];
            const double dy = (cy ? (double)(wy0 + D.W) : (double)(wy0 - 1)) - P.b[1];
            const double jj = P.Ai[0] * dx + P.Ai[1] * dy;
            const double ii = P.Ai[2] * dx + P.Ai[3] * dy;
            jmin = fmin(jmin, jj); jmax = fmax(jmax, jj);
            imin = fmin(imin, ii); imax = fmax(imax, ii);
        }
    // ring reach 2 + 1 pixel of rounding margin
    const double lo = -8.0, hi = (double)M + 8.0;
    jmin = fmax(jmin, lo); imin = fmax(imin, lo); jmax = fmin(jmax, hi); imax = fmin(imax, hi);
    const int pj0 = max(0, (int)floor(jmin) - 3), pj1 = min(M - 1, (int)ceil(jmax) + 3);
    const int pi0 = max(0, (int)floor(imin) - 3), pi1 = min(M - 1, (int)ceil(imax) + 3);
    if (pj0 > pj1 || pi0 > pi1) return;
    s.empty = 0;
    s.pi0 = pi0; s.pi1 = pi1; s.pj0 = pj0; s.pj1 = pj1;
    // slopes reach one pixel further (the central difference)
    s.si0 = max(pi0 - 1, 0) / k; s.si1 = min(pi1 + 1, M - 1) / k;
    s.sj0 = max(pj0 - 1, 0) / k; s.sj1 = min(pj1 + 1, M - 1) / k;
    s.nxc = pi1 / CH - pi0 / CH + 1;
    s.nb = s.sj1 - s.sj0 + 2;
    s.nyc = pj1 / CH - pj0 / CH + 1;
    s.nbr = s.si1 - s.si0 + 2;
    const int nsub = (s.si1 - s.si0 + 1) * (s.sj1 - s.sj0 + 1);
    s.ntask = s.nxc * s.nb + s.nyc * s.nbr;
    s.need = NV * (2 * s.nxc * s.nb + 2 * s.nyc * s.nbr + 2 * nsub);
    s.xo = (float)(P.A[0] * pj0 + P.A[1] * pi0 + P.b[0] - (double)(wx0 - 1));
    s.yo = (float)(P.A[2] * pj0 + P.A[3] * pi0 + P.b[1] - (double)(wy0 - 1));
    s.a00 = (float)P.A[0]; s.a01 = (float)P.A[1]; s.a10 = (float)P.A[2]; s.a11 = (float)P.A[3];
    if (NV == 5) {
        for (int q = 0; q < 4; ++q) {
            s.dxo[q] = (float)(P.dA[4 * q + 0] * pj0 + P.dA[4 * q + 1] * pi0 + P.db[2 * q + 0]);
            s.dyo[q] = (float)(P.dA[4 * q + 2] * pj0 + P.dA[4 * q + 3] * pi0 + P.db[2 * q + 1]);
        }
        for (int q = 0; q < 16; ++q) s.da[q] = (float)P.dA[q];
    }
}

// One telescoped line task: a column pair (XB) over a chunk of rows, or a row
// pair (YB) over a chunk of columns.
template <int NV>
__device__ void line_task(const DevWFS &WF, const ItemWfs &s, int u, const Eval<NV> &ev,
                          float *base) {
    const int k = WF.k, M = WF.M, CH = WF.CH;
    const int nxb = s.nxc * s.nb, nyb = s.nyc * s.nbr;
    float L[NV], R[NV], v[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) L[t] = R[t] = 0.f;
    if (u < nxb) {
        const int c = u / s.nb, bq = u - c * s.nb, b = s.sj0 + bq;
        const int cid = s.pi0 / CH + c;
        const int r_lo = max(cid * CH, s.pi0), r_hi = min(cid * CH + CH - 1, s.pi1);
        const int c0 = b * k - 1, c1 = b * k;
        const bool use0 = c0 >= s.pj0 && c0 <= s.pj1, use1 = c1 >= s.pj0 && c1 <= s.pj1;
        const uint8_t *xc = WF.xcode + (size_t)b * M;
        for (int r = r_lo; r <= r_hi; ++r) {
            const int code = xc[r];
            if (use0 && (code & 3)) {
                ev.eval(r, c0, v);
                if (code & 1) for (int t = 0; t < NV; ++t) L[t] += v[t];
                if (code & 2) for (int t = 0; t < NV; ++t) R[t] += v[t];
            }
            if (use1 && (code & 12)) {
                ev.eval(r, c1, v);
                if (code & 4) for (int t = 0; t < NV; ++t) L[t] += v[t];
                if (code & 8) for (int t = 0; t < NV; ++t) R[t] += v[t];
            }
        }
        float *CBL = base, *CBR = base + NV * nxb;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            CBL[(c * s.nb + bq) * NV + t] = L[t];
            CBR[(c * s.nb + bq) * NV + t] = R[t];
        }
    } else {
        u -= nxb;
        const int c = u / s.nbr, bq = u - c * s.nbr, b = s.si0 + bq;
        const int cid = s.pj0 / CH + c;
        const int c_lo = max(cid * CH, s.pj0), c_hi = min(cid * CH + CH - 1, s.pj1);
        const int r0 = b * k - 1, r1 = b * k;
        const bool use0 = r0 >= s.pi0 && r0 <= s.pi1, use1 = r1 >= s.pi0 && r1 <= s.pi1;
        const uint8_t *yc = WF.ycode + (size_t)b * M;
        for (int col = c_lo; col <= c_hi; ++col) {
            const int code = yc[col];
            if (use0 && (code & 3)) {
                ev.eval(r0, col, v);
                if (code & 1) for (int t = 0; t < NV; ++t) L[t] += v[t];
                if (code & 2) for (int t = 0; t < NV; ++t) R[t] += v[t];
            }
            if (use1 && (code & 12)) {
                ev.eval(r1, col, v);
                if (code & 4) for (int t = 0; t < NV; ++t) L[t] += v[t];
                if (code & 8) for (int t = 0; t < NV; ++t) R[t] += v[t];
            }
        }
        float *RBU = base + 2 * NV * nxb, *RBD = RBU + NV * nyb;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            RBU[(c * s.nbr + bq) * NV + t] = L[t];
            RBD[(c * s.nbr + bq) * NV + t] = R[t];
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(256)
    k_im(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs, int *__restrict__ counter,
         int *__restrict__ err, double *__restrict__ gp) {
    constexpr int NV = (MODE == MODE_FWD) ? 1 : 5;
    extern __shared__ __align__(128) unsigned char smem[];
    float *s_win = reinterpret_cast<float *>(smem);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + (size_t)g.max_win_floats * 4);
    ItemWfs *s_info = reinterpret_cast<ItemWfs *>(s_bar + 2);
    float *s_arena = reinterpret_cast<float *>(s_info + SYNIM_MAX_WFS);
    __shared__ int s_item, s_next, s_abort, s_ng;
    __shared__ int s_tpre[SYNIM_MAX_WFS + 1];
    __shared__ int s_gbeg[SYNIM_MAX_WFS + 1];
    __shared__ double s_gp[MODE == MODE_VJP ? SYNIM_MAX_PAIRS * 4 : 1];

    const int tid = threadIdx.x, nth = blockDim.x;
    const uint32_t bar = smem_u32(s_bar);
    if (MODE == MODE_VJP)
        for (int q = tid; q < SYNIM_MAX_PAIRS * 4; q += nth) s_gp[q] = 0.0;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        s_abort = 0;
        const int it = atomicAdd(counter, 1);
        s_item = it;
        if (it < g.n_items) issue_window(g, it, s_win, bar);
    }
    __syncthreads();
    int item = s_item;
    uint32_t phase = 0;
    while (item < g.n_items) {
        int d, a;
        decode_item(g, item, d, a);
        const DevDM &D = g.dm[d];
        for (int w = tid; w < g.n_wfs; w += nth) make_info<MODE, NV>(g, pairs, d, a, w, s_info[w]);
        __syncthreads();
        if (tid == 0) {
            // group sensors so that their accumulators fit the arena
            int used = 0, ng = 0, tp = 0;
            s_gbeg[0] = 0;
            for (int w = 0; w < g.n_wfs; ++w) {
                ItemWfs &s = s_info[w];
                if (s.need > g.arena_floats) {
                    atomicOr(err, ERR_ARENA);
                    s.empty = 1; s.ntask = 0; s.need = 0;
                    s.si0 = 1; s.si1 = 0; s.sj0 = 1; s.sj1 = 0;
                }
                if (used + s.need > g.arena_floats && w > s_gbeg[ng]) {
                    ++ng;
                    s_gbeg[ng] = w;
                    used = 0;
                }
                s.arena = used;
                used += s.need;
                s_tpre[w] = tp;
                tp += s.ntask;
            }
            s_tpre[g.n_wfs] = tp;
            ++ng;
            s_gbeg[ng] = g.n_wfs;
            s_ng = ng;
        }
        if (!mbar_wait_bounded(bar, phase)) {
            s_abort = 1;
            atomicOr(err, ERR_TIMEOUT);
        }
        __syncthreads();
        if (s_abort) break;
        phase ^= 1u;
        const int ng = s_ng;
        for (int gi = 0; gi < ng; ++gi) {
            const int w0 = s_gbeg[gi], w1 = s_gbeg[gi + 1];
            const int z0 = s_info[w0].arena, z1 = s_info[w1 - 1].arena + s_info[w1 - 1].need;
            for (int q = z0 + tid; q < z1; q += nth) s_arena[q] = 0.f;
            __syncthreads();
            // telescoped boundary lines
            const int t0 = s_tpre[w0], t1 = s_tpre[w1];
            for (int t = t0 + tid; t < t1; t += nth) {
                int w = w0;
                while (s_tpre[w + 1] <= t) ++w;
                const ItemWfs &s = s_info[w];
                Eval<NV> ev;
                ev.load(s, s_win, D.Wp, D.W, g.wfs[w].M);
                line_task<NV>(g.wfs[w], s, t - s_tpre[w], ev, s_arena + s.arena);
            }
            // pixels where the pupil edge cuts a subaperture: one warp per
            // subaperture, lane-strided in entry order + butterfly reduction,
            // so the sums are deterministic
            {
                const int warp = tid >> 5, lane = tid & 31, nwarps = nth >> 5;
                for (int w = w0; w < w1; ++w) {
                    const ItemWfs &s = s_info[w];
                    if (s.empty) continue;
                    const DevWFS &WF = g.wfs[w];
                    Eval<NV> ev;
                    ev.load(s, s_win, D.Wp, D.W, WF.M);
                    const int nsj = s.sj1 - s.sj0 + 1, nsub = (s.si1 - s.si0 + 1) * nsj;
                    float *S = s_arena + s.arena + NV * (2 * s.nxc * s.nb + 2 * s.nyc * s.nbr);
                    for (int idx = warp; idx < nsub; idx += nwarps) {
                        const int si = s.si0 + idx / nsj, sj = s.sj0 + idx % nsj;
                        const int e0 = WF.irr_sub[si * WF.n_sub + sj];
                        const int e1 = WF.irr_sub[si * WF.n_sub + sj + 1];
                        if (e0 == e1) continue;
                        float ax[NV], ay[NV], v[NV];
#pragma unroll
                        for (int t = 0; t < NV; ++t) ax[t] = ay[t] = 0.f;
                        for (int e = e0 + lane; e < e1; e += 32) {
                            const int pix = WF.irr_pix[e];
                            const int i = pix >> 16, j = pix & 0xffff;
                            if (i < s.pi0 || i > s.pi1 || j < s.pj0 || j > s.pj1) continue;
                            ev.eval(i, j, v);
                            const float wx = WF.irr_w[2 * e], wy = WF.irr_w[2 * e + 1];
#pragma unroll
                            for (int t = 0; t < NV; ++t) {
                                ax[t] = fmaf(wx, v[t], ax[t]);
                                ay[t] = fmaf(wy, v[t], ay[t]);
                            }
                        }
#pragma unroll
                        for (int t = 0; t < NV; ++t)
                            for (int o = 16; o > 0; o >>= 1) {
                                ax[t] += __shfl_xor_sync(0xffffffffu, ax[t], o);
                                ay[t] += __shfl_xor_sync(0xffffffffu, ay[t], o);
                            }
                        if (lane == 0) {
#pragma unroll
                            for (int t = 0; t < NV; ++t) {
                                S[idx * NV + t] = ax[t];
                                S[(nsub + idx) * NV + t] = ay[t];
                            }
                        }
                    }
                }
            }
            __syncthreads();
            if (gi == ng - 1 && tid == 0) {
                // the window is no longer read: prefetch the next actuator
                const int nx = atomicAdd(counter, 1);
                s_next = nx;
                if (nx < g.n_items) {
                    fence_proxy_async_smem();
                    issue_window(g, nx, s_win, bar);
                }
            }
            // finalize: add the telescoped line sums into each subaperture
            for (int w = w0; w < w1; ++w) {
                const ItemWfs &s = s_info[w];
                if (s.empty) continue;
                const DevWFS &WF = g.wfs[w];
                const int k = WF.k, CH = WF.CH;
                const int nsj = s.sj1 - s.sj0 + 1, nsub = (s.si1 - s.si0 + 1) * nsj;
                const int nxb = s.nxc * s.nb, nyb = s.nyc * s.nbr;
                float *base = s_arena + s.arena;
                const float *CBL = base, *CBR = base + NV * nxb;
                const float *RBU = base + 2 * NV * nxb, *RBD = RBU + NV * nyb;
                float *S = base + NV * (2 * nxb + 2 * nyb);
                for (int idx = tid; idx < nsub; idx += nth) {
                    const int si = s.si0 + idx / nsj, sj = s.sj0 + idx % nsj;
                    float sx[NV], sy[NV];
#pragma unroll
                    for (int t = 0; t < NV; ++t) { sx[t] = S[idx * NV + t]; sy[t] = S[(nsub + idx) * NV + t]; }
                    const int cx_lo = max(si * k / CH, s.pi0 / CH), cx_hi = min(((si + 1) * k - 1) / CH, s.pi1 / CH);
                    for (int cid = cx_lo; cid <= cx_hi; ++cid) {
                        const int c = cid - s.pi0 / CH;
#pragma unroll
                        for (int t = 0; t < NV; ++t)
                            sx[t] += CBL[(c * s.nb + sj + 1 - s.sj0) * NV + t] - CBR[(c * s.nb + sj - s.sj0) * NV + t];
                    }
                    const int cy_lo = max(sj * k / CH, s.pj0 / CH), cy_hi = min(((sj + 1) * k - 1) / CH, s.pj1 / CH);
                    for (int cid = cy_lo; cid <= cy_hi; ++cid) {
                        const int c = cid - s.pj0 / CH;
#pragma unroll
                        for (int t = 0; t < NV; ++t)
                            sy[t] += RBU[(c * s.nbr + si + 1 - s.si0) * NV + t] - RBD[(c * s.nbr + si - s.si0) * NV + t];
                    }
#pragma unroll
                    for (int t = 0; t < NV; ++t) { S[idx * NV + t] = sx[t]; S[(nsub + idx) * NV + t] = sy[t]; }
                }
            }
            __syncthreads();
            // output: dense columns (MODE_FWD / MODE_TAN) or the VJP reduction
            for (int w = w0; w < w1; ++w) {
                const ItemWfs &s = s_info[w];
                const DevWFS &WF = g.wfs[w];
                const int pidx = d * g.n_wfs + w;
                const DevPair &P = pairs[pidx];
                const int nv = WF.nv, n2 = 2 * nv;
                const int nsj = s.sj1 - s.sj0 + 1, nsub = (s.si1 - s.si0 + 1) * nsj;
                const float *S = s_arena + s.arena + NV * (2 * s.nxc * s.nb + 2 * s.nyc * s.nbr);
                const int x_lo = s.empty ? 0 : WF.vrow[s.si0];
                const int x_hi = s.empty ? 0 : WF.vrow[s.si1 + 1];
                auto value = [&](int r, int t) -> float {
                    const int comp = r >= nv ? 1 : 0;
                    const int rr = r - comp * nv;
                    const int sub = WF.vsub[rr];
                    const int si = sub >> 16, sj = sub & 0xffff;
                    if (si < s.si0 || si > s.si1 || sj < s.sj0 || sj > s.sj1) return 0.f;
                    return S[(comp * nsub + (si - s.si0) * nsj + (sj - s.sj0)) * NV + t] * WF.fac[rr];
                };
                if (MODE == MODE_VJP) {
                    if (!P.gim || s.empty) continue;
                    const float *src = P.gim + (size_t)a * n2;
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    const int span = x_hi - x_lo;
                    for (int q = tid; q < 2 * span; q += nth) {
                        const int r = (q < span) ? x_lo + q : nv + x_lo + (q - span);
                        const float gv = src[r];
                        if (gv != 0.f)
#pragma unroll
                            for (int t = 0; t < 4; ++t) acc[t] = fmaf(gv, value(r, t + 1), acc[t]);
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        float vsum = acc[t];
                        for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
                        if ((tid & 31) == 0 && vsum != 0.f) atomicAdd(&s_gp[pidx * 4 + t], (double)vsum);
                    }
                    continue;
                }
                const int nout = (MODE == MODE_FWD) ? 1 : 5;
                for (int t = 0; t < nout; ++t) {
                    float *dst = (t == 0) ? P.im : P.dim[t - 1];
                    if (!dst) continue;
                    dst += (size_t)a * n2;
                    if ((nv & 1) == 0) {
                        for (int q = tid; q < n2 / 4; q += nth) {
                            const int r0 = 4 * q;
                            float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
                            const bool hit = (r0 + 4 > x_lo && r0 < x_hi) ||
                                             (r0 + 4 > nv + x_lo && r0 < nv + x_hi);
                            if (hit) {
                                o.x = value(r0, t); o.y = value(r0 + 1, t);
                                o.z = value(r0 + 2, t); o.w = value(r0 + 3, t);
                            }
                            __stcs(reinterpret_cast<float4 *>(dst + r0), o);
                        }
                    } else {
                        for (int q = tid; q < nv; q += nth) {
                            const int r0 = 2 * q;
                            float2 o = make_float2(0.f, 0.f);
                            const bool hit = (r0 + 2 > x_lo && r0 < x_hi) ||
                                             (r0 + 2 > nv + x_lo && r0 < nv + x_hi);
                            if (hit) { o.x = value(r0, t); o.y = value(r0 + 1, t); }
                            __stcs(reinterpret_cast<float2 *>(dst + r0), o);
                        }
                    }
                }
            }
            __syncthreads();
        }
        item = s_next;
    }
    if (MODE == MODE_VJP) {
        __syncthreads();
        const int np = g.n_dm * g.n_wfs;
        for (int q = tid; q < np * 4; q += nth)
            if (s_gp[q] != 0.0) atomicAdd(&gp[q], s_gp[q]);
    }
}

size_t im_smem_bytes(const Geo &g) {
    return (size_t)g.max_win_floats * 4 + 16 + sizeof(ItemWfs) * SYNIM_MAX_WFS +
           (size_t)g.arena_floats * 4;
}

template <int MODE>
static cudaError_t prepare_one(int threads, size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_im<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_im<MODE>, threads, smem);
}

cudaError_t im_prepare(int mode, int threads, size_t smem, int *bps) {
    switch (mode) {
        case MODE_FWD: return prepare_one<MODE_FWD>(threads, smem, bps);
        case MODE_TAN: return prepare_one<MODE_TAN>(threads, smem, bps);
        default: return prepare_one<MODE_VJP>(threads, smem, bps);
    }
}

cudaError_t launch_im(int mode, const Geo &g, const DevPair *pairs, int *counter, int *err,
                      double *gp, int grid, int threads, size_t smem, cudaStream_t s) {
    switch (mode) {
        case MODE_FWD: k_im<MODE_FWD><<<grid, threads, smem, s>>>(g, pairs, counter, err, gp); break;
        case MODE_TAN: k_im<MODE_TAN><<<grid, threads, smem, s>>>(g, pairs, counter, err, gp); break;
        default: k_im<MODE_VJP><<<grid, threads, smem, s>>>(g, pairs, counter, err, gp); break;
    }
    return cudaGetLastError();
}

}  // namespace synim
