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
#include "synim_device.cuh"

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
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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
// peak[a] = max |IF_a|; the DM's largest is folded into *dm_peak (float bits,
// non-negative, so an integer max orders them).
__global__ void k_peak(const float *__restrict__ cube, int N, unsigned *__restrict__ dm_peak) {
    const int a = blockIdx.x;
    const size_t NN = (size_t)N * N;
    const float *img = cube + (size_t)a * NN;
    float m = 0.f;
    for (size_t p = threadIdx.x; p < NN; p += blockDim.x) m = fmaxf(m, fabsf(img[p]));
    m = block_reduce(m, MaxF(), 0.f);
    if (threadIdx.x == 0) atomicMax(dm_peak, __float_as_uint(m));
}

// box[a] = {x0, x1, y0, y1} of |IF_a| > eps * (largest |IF| of the DM) (x1 < x0 if empty).
__global__ void k_support(const float *__restrict__ cube, int N, float eps, const unsigned *__restrict__ dm_peak,
                          int *__restrict__ box) {
    const int a = blockIdx.x;
    const size_t NN = (size_t)N * N;
    const float *img = cube + (size_t)a * NN;
    const float thr = eps * __uint_as_float(*dm_peak);
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
    // box holds 4 * n_act + 1 ints: the last one is the DM peak
    unsigned *peak = reinterpret_cast<unsigned *>(box + 4 * (size_t)n_act);
    cudaError_t e = cudaMemsetAsync(peak, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_peak<<<n_act, 256, 0, s>>>(cube, N, peak);
    k_support<<<n_act, 256, 0, s>>>(cube, N, eps, peak, box);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float *cube, int n_act, int N, const int *org, int W, int Wp,
                        int stride, float *win, cudaStream_t s) {
    k_pack<<<n_act, 256, 0, s>>>(cube, N, org, W, Wp, stride, win);
    return cudaGetLastError();
}

// Interior map of a DM mask for the strict-core test: for the bilinear cell
// (cx, cy) (taps cx..cx+1, cy..cy+1; cx, cy in [-1, N-1]) record whether all
// 16 taps of the 3 x 3 cells around it are 0, all 1, or mixed.  A FP32 cell
// can be off by one, so a uniform neighbourhood settles the core decision.
__global__ void k_mcls(const uint8_t *__restrict__ mask, int N, uint8_t *__restrict__ mcls) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long N1 = N + 1;
    if (q >= N1 * N1) return;
    const int cy = (int)(q / N1) - 1, cx = (int)(q - (q / N1) * N1) - 1;
    int ones = 0;
    for (int y = cy - 1; y <= cy + 2; ++y)
        for (int x = cx - 1; x <= cx + 2; ++x)
            ones += (x >= 0 && y >= 0 && x < N && y < N) ? (mask ? (mask[(long)y * N + x] != 0) : 1) : 0;
    mcls[q] = ones == 0 ? 0 : (ones == 16 ? 1 : 2);
}

cudaError_t launch_mcls(const uint8_t *mask, int N, uint8_t *mcls, cudaStream_t s) {
    const long n = (long)(N + 1) * (N + 1);
    k_mcls<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mask, N, mcls);
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
// each sensor pixel.  The decision is the FP64 definition (no contraction);
// FP32 pre-tests settle every pixel whose neighbourhood of mask taps is
// uniform, and every pixel whose four taps agree and whose fractional position
// is far from an integer, so FP64 runs only at mask edges near cell lines.
__global__ void k_pst_core(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs) {
    const int p = blockIdx.y;
    const int d = p / g.n_wfs, w = p - d * g.n_wfs;
    const int M = g.wfs[w].M;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)M * M) return;
    const DevPair &P = pairs[p];
    uint8_t *pst = P.pst;
    if (!pst) return;
    const int i = (int)(idx / M), j = (int)(idx - (long)i * M);
    const int N = g.dm[d].N;
    const uint8_t *mask = g.dm[d].mask;
    const float xf = fmaf(P.Ahi[0], (float)j, fmaf(P.Ahi[1], (float)i, P.bhi[0]));
    const float yf = fmaf(P.Ahi[2], (float)j, fmaf(P.Ahi[3], (float)i, P.bhi[1]));
    int core = -1;
    if (!(fabsf(xf) < 1e6f && fabsf(yf) < 1e6f)) {
        core = 0;
    } else {
        const float fx0 = floorf(xf), fy0 = floorf(yf);
        const int ix = (int)fx0, iy = (int)fy0;
        if (ix < -2 || iy < -2 || ix > N || iy > N) {
            core = 0;  // every tap of every candidate cell is off the grid
        } else if (ix >= -1 && iy >= -1 && ix <= N - 1 && iy <= N - 1) {
            const int c = g.dm[d].mcls[(long)(iy + 1) * (N + 1) + (ix + 1)];
            if (c != 2) core = c;
        }
        if (core < 0) {
            const float fxf = xf - fx0, fyf = yf - fy0;
            if (fxf > 0.01f && fxf < 0.99f && fyf > 0.01f && fyf < 0.99f) {
                // FP32 coordinate error < 1e-3 px: the cell is certain; every
                // weight is > 1e-4, so any zero tap puts the mask below 0.999999.
                core = mask_tap(mask, N, ix, iy) & mask_tap(mask, N, ix + 1, iy) &
                       mask_tap(mask, N, ix, iy + 1) & mask_tap(mask, N, ix + 1, iy + 1);
            }
        }
    }
    if (core < 0) {
        const double *A = P.A, *b = P.b;
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

// Class of a sensor pixel from the core map: 1 core, 2 ring (Sec. 2.3 step 2:
// a non-core pixel with a core 4-neighbour), 0 otherwise.
__device__ __forceinline__ int pixel_class(const uint8_t *__restrict__ pst, int M, int i, int j) {
    const long q = (long)i * M + j;
    if (pst[q]) return 1;
    const bool ring = (j + 1 < M && pst[q + 1]) || (j >= 1 && pst[q - 1]) ||
                      (i + 1 < M && pst[q + M]) || (i >= 1 && pst[q - M]);
    return ring ? 2 : 0;
}

// Boundary-line bytes: for boundary b and pixel row i (x) / column j (y):
// bits 0-3 = stencil bits of the sensor, bits 4-5 / 6-7 = classes of the two
// line pixels (b k - 1 and b k).  Stored [i][b] so that consecutive b are
// consecutive bytes.
__global__ void k_pst_codes(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs) {
    const int p = blockIdx.y;
    const int w = p % g.n_wfs;
    const DevWFS &WF = g.wfs[w];
    const int M = WF.M, n1 = WF.n_sub + 1, k = WF.k;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2L * M * n1) return;
    const DevPair &P = pairs[p];
    if (!P.pst) return;
    const int dir = (int)(idx / ((long)M * n1));
    const long r = idx - (long)dir * M * n1;
    const int x = (int)(r / n1), b = (int)(r - (long)x * n1);
    const int c0 = b * k - 1, c1 = b * k;
    int code;
    if (dir == 0) {
        code = WF.xcode[(long)b * M + x];
        const int k0 = (c0 >= 0) ? pixel_class(P.pst, M, x, c0) : 0;
        const int k1 = (c1 < M) ? pixel_class(P.pst, M, x, c1) : 0;
        P.xcc[r] = (uint8_t)(code | (k0 << 4) | (k1 << 6));
    } else {
        code = WF.ycode[(long)b * M + x];
        const int k0 = (c0 >= 0) ? pixel_class(P.pst, M, c0, x) : 0;
        const int k1 = (c1 < M) ? pixel_class(P.pst, M, c1, x) : 0;
        P.ycc[r] = (uint8_t)(code | (k0 << 4) | (k1 << 6));
    }
}

cudaError_t launch_pst(const Geo &g, const DevPair *pairs, int max_mm, int max_lines, cudaStream_t s) {
    dim3 grid((max_mm + 255) / 256, g.n_dm * g.n_wfs);
    k_pst_core<<<grid, 256, 0, s>>>(g, pairs);
    dim3 grid2((2 * max_lines + 255) / 256, g.n_dm * g.n_wfs);
    k_pst_codes<<<grid2, 256, 0, s>>>(g, pairs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The IM kernel
// ---------------------------------------------------------------------------
struct ItemWfs {
    int pi0, pi1, pj0, pj1;  // pixel box where phi may be non-zero (inclusive)
    int si0, si1, sj0, sj1;  // subapertures whose slopes may be non-zero (inclusive)
    int nxc, nb, nyc, nbr;   // row chunks x column boundaries; column chunks x row boundaries
    int ntask, arena, group, empty;
    int xcid0, ycid0;        // first row / column chunk ids (pi0 / CH, pj0 / CH)
    float inv_nb, inv_nbr;   // 1 / nb, 1 / nbr (task decode without integer division)
    float xo, yo;            // padded-window coordinates of pixel (pi0, pj0)
    float a00, a01, a10, a11;
    float dxo[4], dyo[4], da[16];  // tangents of the coordinates (MODE_TAN / MODE_VJP)
    const uint8_t *pst, *xcc, *ycc;
};

// Bilinear sample of a zero-bordered window at padded coordinates (x, y);
// zero when the cell does not touch the window.
__device__ __forceinline__ float bil_xy(const float *__restrict__ win, int Wp, float Wf1, float x, float y) {
    if (!(x > 0.f && x < Wf1 && y > 0.f && y < Wf1)) return 0.f;
    const int ix = __float2int_rd(x), iy = __float2int_rd(y);
    const float fx = x - (float)ix, fy = y - (float)iy;
    const float *q = win + iy * Wp + ix;
    const float v00 = q[0], v10 = q[1], v01 = q[Wp], v11 = q[Wp + 1];
    const float top = fmaf(fx, v10 - v00, v00), bot = fmaf(fx, v11 - v01, v01);
    return fmaf(fy, bot - top, top);
}

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

    // Edge repair step 3 (Sec. 2.3) at a ring pixel: mean over the valid
    // cardinal directions of 2 P1 - P2 (or P1); P1, P2 must be strict core.
    __device__ __forceinline__ void ring(int i, int j, float *v) const {
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
            if (!pst[i1 * M + j1]) continue;
            float v1[NV];
            bil(i1, j1, v1);
            const int i2 = i1 + di, j2 = j1 + dj;
            if (i2 >= 0 && i2 < M && j2 >= 0 && j2 < M && pst[i2 * M + j2]) {
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

    // Repaired phase (and tangents) at (i, j) of known class (0 zero, 1 core, 2 ring).
    __device__ __forceinline__ void eval_cls(int i, int j, int cls, float *v) const {
        if (cls == 1) {
            bil(i, j, v);
        } else if (cls == 0) {
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = 0.f;
        } else {
            ring(i, j, v);
        }
    }
    __device__ __forceinline__ void eval(int i, int j, float *v) const {
        eval_cls(i, j, pixel_class(pst, M, i, j), v);
    }
};

__device__ __forceinline__ void decode_item(const Geo &g, int item, int &d, int &a) {
    int pos = 0;
    while (pos + 1 < g.n_dm && item >= g.order_start[pos + 1]) ++pos;
    d = g.order_dm[pos];
    a = item - g.order_start[pos];
}

__device__ __forceinline__ void prefetch_window(const Geo &g, int item) {
    int d, a;
    decode_item(g, item, d, a);
    const DevDM &D = g.dm[d];
    bulk_prefetch_l2(D.win + (size_t)a * D.win_stride, (uint32_t)D.win_stride * 4u);
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
                          ItemWfs &s, int *err) {
    const DevPair &P = pairs[d * g.n_wfs + w];
    const DevWFS &WF = g.wfs[w];
    const DevDM &D = g.dm[d];
    const int M = WF.M, k = WF.k, CH = WF.CH;
    s.pst = P.pst; s.xcc = P.xcc; s.ycc = P.ycc;
    s.arena = P.arena_off;
    s.group = P.group;
    s.empty = 1;
    s.ntask = 0;
    s.si0 = 1; s.si1 = 0; s.sj0 = 1; s.sj1 = 0;
    s.pi0 = 1; s.pi1 = 0; s.pj0 = 1; s.pj1 = 0;
    if (!pair_active<MODE>(P)) return;
    const int wx0 = D.org[2 * a], wy0 = D.org[2 * a + 1];
    // cells that touch the window: x in (wx0 - 1, wx0 + W), y likewise
    float jmin = 3e38f, jmax = -3e38f, imin = 3e38f, imax = -3e38f;
#pragma unroll
    for (int cx = 0; cx < 2; ++cx)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            const float dx = (float)(cx ? wx0 + D.W : wx0 - 1) - P.bhi[0];
            const float dy = (float)(cy ? wy0 + D.W : wy0 - 1) - P.bhi[1];
            const float jj = fmaf(P.Aif[0], dx, P.Aif[1] * dy);
            const float ii = fmaf(P.Aif[2], dx, P.Aif[3] * dy);
            jmin = fminf(jmin, jj); jmax = fmaxf(jmax, jj);
            imin = fminf(imin, ii); imax = fmaxf(imax, ii);
        }
    const float lo = -8.f, hi = (float)M + 8.f;
    jmin = fmaxf(jmin, lo); imin = fmaxf(imin, lo); jmax = fminf(jmax, hi); imax = fminf(imax, hi);
    // ring reach 2 + 1 pixel of rounding margin
    const int pj0 = max(0, (int)floorf(jmin) - 3), pj1 = min(M - 1, (int)ceilf(jmax) + 3);
    const int pi0 = max(0, (int)floorf(imin) - 3), pi1 = min(M - 1, (int)ceilf(imax) + 3);
    if (pj0 > pj1 || pi0 > pi1) return;
    // slopes reach one pixel further (the central difference)
    const int si0 = max(pi0 - 1, 0) / k, si1 = min(pi1 + 1, M - 1) / k;
    const int sj0 = max(pj0 - 1, 0) / k, sj1 = min(pj1 + 1, M - 1) / k;
    const int nxc = pi1 / CH - pi0 / CH + 1, nb = sj1 - sj0 + 2;
    const int nyc = pj1 / CH - pj0 / CH + 1, nbr = si1 - si0 + 2;
    const int nsub = (si1 - si0 + 1) * (sj1 - sj0 + 1);
    const int need = NV * (2 * nxc * nb + 2 * nyc * nbr + 2 * nsub);
    if (need > P.arena_len) {
        atomicOr(err, ERR_ARENA);
        return;
    }
    s.empty = 0;
    s.pi0 = pi0; s.pi1 = pi1; s.pj0 = pj0; s.pj1 = pj1;
    s.si0 = si0; s.si1 = si1; s.sj0 = sj0; s.sj1 = sj1;
    s.nxc = nxc; s.nb = nb; s.nyc = nyc; s.nbr = nbr;
    s.ntask = nxc * nb + nyc * nbr;
    s.xcid0 = pi0 / CH;
    s.ycid0 = pj0 / CH;
    s.inv_nb = 1.f / (float)nb;
    s.inv_nbr = 1.f / (float)nbr;
    s.xo = exact_affine(P.Ahi[0], P.Alo[0], P.Ahi[1], P.Alo[1], P.bhi[0], P.blo[0], pj0, pi0, wx0 - 1);
    s.yo = exact_affine(P.Ahi[2], P.Alo[2], P.Ahi[3], P.Alo[3], P.bhi[1], P.blo[1], pj0, pi0, wy0 - 1);
    s.a00 = P.Ahi[0]; s.a01 = P.Ahi[1]; s.a10 = P.Ahi[2]; s.a11 = P.Ahi[3];
    if (NV == 5) {
        for (int q = 0; q < 4; ++q) {
            s.dxo[q] = (float)(P.dA[4 * q + 0] * pj0 + P.dA[4 * q + 1] * pi0 + P.db[2 * q + 0]);
            s.dyo[q] = (float)(P.dA[4 * q + 2] * pj0 + P.dA[4 * q + 3] * pi0 + P.db[2 * q + 1]);
        }
        for (int q = 0; q < 16; ++q) s.da[q] = (float)P.dA[q];
    }
}

// floor(u / n) for 0 <= u < 2^24 from a float reciprocal, corrected to exact.
__device__ __forceinline__ int fast_div(int u, int n, float inv) {
    int c = __float2int_rz((float)u * inv);
    if (c * n > u) --c;
    else if ((c + 1) * n <= u) ++c;
    return c;
}

// One telescoped line task: a column pair (b k - 1, b k) over a chunk of
// rows (x slopes) or a row pair over a chunk of columns (y slopes).
struct LineTask {
    int lo, hi, l0, slot;  // line range, first line pixel, accumulator slot
    bool xdir, use0, use1;
    const uint8_t *cc;     // boundary-line bytes of this boundary (stride n_sub + 1)
};

__device__ __forceinline__ LineTask decode_task(const DevWFS &WF, const ItemWfs &s, int u) {
    const int k = WF.k, CH = WF.CH;
    const int nxb = s.nxc * s.nb;
    LineTask T;
    T.xdir = u < nxb;
    if (T.xdir) {
        const int c = fast_div(u, s.nb, s.inv_nb), bq = u - c * s.nb;
        const int b = s.sj0 + bq, cid = s.xcid0 + c;
        T.lo = max(cid * CH, s.pi0);
        T.hi = min(cid * CH + CH - 1, s.pi1);
        T.l0 = b * k - 1;
        T.use0 = T.l0 >= s.pj0 && T.l0 <= s.pj1;
        T.use1 = T.l0 + 1 >= s.pj0 && T.l0 + 1 <= s.pj1;
        T.cc = s.xcc + b;
        T.slot = c * s.nb + bq;
    } else {
        u -= nxb;
        const int c = fast_div(u, s.nbr, s.inv_nbr), bq = u - c * s.nbr;
        const int b = s.si0 + bq, cid = s.ycid0 + c;
        T.lo = max(cid * CH, s.pj0);
        T.hi = min(cid * CH + CH - 1, s.pj1);
        T.l0 = b * k - 1;
        T.use0 = T.l0 >= s.pi0 && T.l0 <= s.pi1;
        T.use1 = T.l0 + 1 >= s.pi0 && T.l0 + 1 <= s.pi1;
        T.cc = s.ycc + b;
        T.slot = c * s.nbr + bq;
    }
    return T;
}

// Up to 8 boundary-line bytes (rows r0 .. r0 + 7 of the task) in one register.
__device__ __forceinline__ unsigned long long load_codes(const LineTask &T, int n1, int r0) {
    const int cnt = min(8, T.hi - r0 + 1);
    unsigned long long pack = 0ull;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (q < cnt) pack |= (unsigned long long)__ldg(T.cc + (long)(r0 + q) * n1) << (8 * q);
    return pack;
}

// Resample the task's line pixels (the first 8 rows' bytes are given) and
// store its two telescoped partial sums.
template <int NV>
__device__ __forceinline__ void run_task(const DevWFS &WF, const ItemWfs &s, const LineTask &T,
                                         unsigned long long pack, const Eval<NV> &ev, float *base) {
    const int n1 = WF.n_sub + 1;
    const int nxb = s.nxc * s.nb, nyb = s.nyc * s.nbr;
    float L[NV], R[NV], v[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) L[t] = R[t] = 0.f;
    const bool xdir = T.xdir;
    const int lo = T.lo, hi = T.hi, l0 = T.l0;
    if constexpr (NV == 1) {
        // along a line the sampled DM point moves by a constant step: one FMA
        // per coordinate from the line's first pixel
        float x0, y0, x1, y1, sx, sy;
        if (xdir) {
            const float di = (float)(lo - ev.pi0), dj = (float)(l0 - ev.pj0);
            x0 = fmaf(ev.a00, dj, fmaf(ev.a01, di, ev.xo));
            y0 = fmaf(ev.a10, dj, fmaf(ev.a11, di, ev.yo));
            x1 = fmaf(ev.a00, dj + 1.f, fmaf(ev.a01, di, ev.xo));
            y1 = fmaf(ev.a10, dj + 1.f, fmaf(ev.a11, di, ev.yo));
            sx = ev.a01;
            sy = ev.a11;
        } else {
            const float di = (float)(l0 - ev.pi0), dj = (float)(lo - ev.pj0);
            x0 = fmaf(ev.a00, dj, fmaf(ev.a01, di, ev.xo));
            y0 = fmaf(ev.a10, dj, fmaf(ev.a11, di, ev.yo));
            x1 = fmaf(ev.a00, dj, fmaf(ev.a01, di + 1.f, ev.xo));
            y1 = fmaf(ev.a10, dj, fmaf(ev.a11, di + 1.f, ev.yo));
            sx = ev.a00;
            sy = ev.a10;
        }
        for (int rb = lo; rb <= hi; rb += 8) {
            if (rb != lo) pack = load_codes(T, n1, rb);
            const int cnt = min(8, hi - rb + 1);
            for (int q = 0; q < cnt; ++q) {
                const int r = rb + q;
                const float m = (float)(r - lo);
                const int code = (int)((pack >> (8 * q)) & 0xffull);
                if (T.use0 && (code & 3)) {
                    const int cls = (code >> 4) & 3;
                    float vv = 0.f;
                    if (cls == 1) vv = bil_xy(ev.win, ev.Wp, ev.Wf1, fmaf(sx, m, x0), fmaf(sy, m, y0));
                    else if (cls == 2) { if (xdir) ev.ring(r, l0, &vv); else ev.ring(l0, r, &vv); }
                    L[0] += (code & 1) ? vv : 0.f;
                    R[0] += (code & 2) ? vv : 0.f;
                }
                if (T.use1 && (code & 12)) {
                    const int cls = code >> 6;
                    float vv = 0.f;
                    if (cls == 1) vv = bil_xy(ev.win, ev.Wp, ev.Wf1, fmaf(sx, m, x1), fmaf(sy, m, y1));
                    else if (cls == 2) { if (xdir) ev.ring(r, l0 + 1, &vv); else ev.ring(l0 + 1, r, &vv); }
                    L[0] += (code & 4) ? vv : 0.f;
                    R[0] += (code & 8) ? vv : 0.f;
                }
            }
        }
    } else {
        for (int rb = lo; rb <= hi; rb += 8) {
            if (rb != lo) pack = load_codes(T, n1, rb);
            const int cnt = min(8, hi - rb + 1);
            for (int q = 0; q < cnt; ++q) {
                const int r = rb + q;
                const int code = (int)((pack >> (8 * q)) & 0xffull);
#pragma unroll 1
                for (int px = 0; px < 2; ++px) {
                    const int bits = (code >> (2 * px)) & 3;
                    if (!bits || !(px ? T.use1 : T.use0)) continue;
                    const int line = l0 + px;
                    if (xdir) ev.eval_cls(r, line, (code >> (4 + 2 * px)) & 3, v);
                    else ev.eval_cls(line, r, (code >> (4 + 2 * px)) & 3, v);
                    if (bits & 1)
#pragma unroll
                        for (int t = 0; t < NV; ++t) L[t] += v[t];
                    if (bits & 2)
#pragma unroll
                        for (int t = 0; t < NV; ++t) R[t] += v[t];
                }
            }
        }
    }
    float *lp, *rp;
    if (xdir) {
        lp = base + T.slot * NV;
        rp = base + NV * nxb + T.slot * NV;
    } else {
        lp = base + 2 * NV * nxb + T.slot * NV;
        rp = base + 2 * NV * nxb + NV * nyb + T.slot * NV;
    }
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        lp[t] = L[t];
        rp[t] = R[t];
    }
}

// Subaperture sums of one sensor (x block, then y block): add the telescoped
// boundary-line sums of every chunk to the pupil-edge sums already in S.
template <int NV>
__device__ __forceinline__ void finalize_sub(const ItemWfs &s, const DevWFS &WF, float *base, int q) {
    const int k = WF.k, CH = WF.CH;
    const int nsj = s.sj1 - s.sj0 + 1, nsub = (s.si1 - s.si0 + 1) * nsj;
    const int nxb = s.nxc * s.nb, nyb = s.nyc * s.nbr;
    float *S = base + NV * (2 * nxb + 2 * nyb);
    const int comp = q >= nsub ? 1 : 0, idx = q - comp * nsub;
    const int si = s.si0 + idx / nsj, sj = s.sj0 + idx % nsj;
    float v[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = S[q * NV + t];
    if (comp == 0) {
        const float *CBL = base, *CBR = base + NV * nxb;
        const int lo = max(si * k / CH, s.pi0 / CH), hi = min(((si + 1) * k - 1) / CH, s.pi1 / CH);
        for (int cid = lo; cid <= hi; ++cid) {
            const int c = cid - s.pi0 / CH;
#pragma unroll
            for (int t = 0; t < NV; ++t)
                v[t] += CBL[(c * s.nb + sj + 1 - s.sj0) * NV + t] - CBR[(c * s.nb + sj - s.sj0) * NV + t];
        }
    } else {
        const float *RBU = base + 2 * NV * nxb, *RBD = RBU + NV * nyb;
        const int lo = max(sj * k / CH, s.pj0 / CH), hi = min(((sj + 1) * k - 1) / CH, s.pj1 / CH);
        for (int cid = lo; cid <= hi; ++cid) {
            const int c = cid - s.pj0 / CH;
#pragma unroll
            for (int t = 0; t < NV; ++t)
                v[t] += RBU[(c * s.nbr + si + 1 - s.si0) * NV + t] - RBD[(c * s.nbr + si - s.si0) * NV + t];
        }
    }
#pragma unroll
    for (int t = 0; t < NV; ++t) S[q * NV + t] = v[t];
}

template <int MODE>
__global__ void __launch_bounds__(512, (MODE == MODE_FWD) ? 2 : 1)
    k_im(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs, int *__restrict__ counter,
         int *__restrict__ err, double *__restrict__ gp) {
    constexpr int NV = (MODE == MODE_FWD) ? 1 : 5;
    extern __shared__ __align__(128) unsigned char smem[];
    float *s_win = reinterpret_cast<float *>(smem);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + (size_t)g.max_win_floats * 4);
    ItemWfs *s_info = reinterpret_cast<ItemWfs *>(s_bar + 2);
    float *s_arena = reinterpret_cast<float *>(s_info + SYNIM_MAX_WFS);
    __shared__ int s_item, s_next, s_abort;
    __shared__ double s_gp[MODE == MODE_VJP ? SYNIM_MAX_PAIRS * 4 : 1];

    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
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
        if (tid == 0) {
            // claim the next actuator now and pull its window towards L2
            const int nx = atomicAdd(counter, 1);
            s_next = nx;
            if (nx < g.n_items) prefetch_window(g, nx);
        }
        for (int w = tid; w < g.n_wfs; w += nth) make_info<MODE, NV>(g, pairs, d, a, w, s_info[w], err);
        if (!mbar_wait_bounded(bar, phase)) {
            s_abort = 1;
            atomicOr(err, ERR_TIMEOUT);
        }
        __syncthreads();
        if (s_abort) break;
        phase ^= 1u;
        const int next_item = s_next;  // read before tid 0 can claim again
        const int ng = g.n_groups[d];
        for (int gi = 0; gi < ng; ++gi) {
            // telescoped boundary lines: the tasks of every sensor of the group
            // form one sequence dealt round-robin to the threads; each thread
            // loads the next task's line bytes before resampling the current one
            {
                auto find = [&](int gq, int &w, int &basew) -> bool {
                    while (true) {
                        if (w >= 0) {
                            if (gq < basew + s_info[w].ntask) return true;
                            basew += s_info[w].ntask;
                        }
                        do { ++w; } while (w < g.n_wfs && (s_info[w].group != gi || s_info[w].empty));
                        if (w >= g.n_wfs) return false;
                    }
                };
                int gq = tid, w = -1, basew = 0;
                if (find(gq, w, basew)) {
                    LineTask T = decode_task(g.wfs[w], s_info[w], gq - basew);
                    unsigned long long pack = load_codes(T, g.wfs[w].n_sub + 1, T.lo);
                    Eval<NV> ev;
                    ev.load(s_info[w], s_win, D.Wp, D.W, g.wfs[w].M);
                    int ev_w = w;
                    while (true) {
                        int gn = gq + nth, wn = w, bn = basew;
                        const bool more = find(gn, wn, bn);
                        LineTask Tn;
                        unsigned long long packn = 0ull;
                        if (more) {
                            Tn = decode_task(g.wfs[wn], s_info[wn], gn - bn);
                            packn = load_codes(Tn, g.wfs[wn].n_sub + 1, Tn.lo);
                        }
                        if (ev_w != w) {
                            ev.load(s_info[w], s_win, D.Wp, D.W, g.wfs[w].M);
                            ev_w = w;
                        }
                        run_task<NV>(g.wfs[w], s_info[w], T, pack, ev, s_arena + s_info[w].arena);
                        if (!more) break;
                        gq = gn; w = wn; basew = bn; T = Tn; pack = packn;
                    }
                }
            }
            // pupil-edge pixels: one warp per (sensor, subaperture row) writes the
            // edge sum of every subaperture of that row (zero where there is none);
            // only the entries on pixel rows inside the box are visited
            for (int rr = warp;; rr += nwarps) {
                int w = 0, acc = 0;
                for (; w < g.n_wfs; ++w) {
                    const ItemWfs &s = s_info[w];
                    if (s.group != gi || s.empty) continue;
                    const int nr = s.si1 - s.si0 + 1;
                    if (rr < acc + nr) break;
                    acc += nr;
                }
                if (w >= g.n_wfs) break;
                const ItemWfs &s = s_info[w];
                const DevWFS &WF = g.wfs[w];
                const int k = WF.k;
                const int si = s.si0 + rr - acc;
                const int nsj = s.sj1 - s.sj0 + 1, nsub = (s.si1 - s.si0 + 1) * nsj;
                float *S = s_arena + s.arena + NV * (2 * s.nxc * s.nb + 2 * s.nyc * s.nbr);
                const int row = (si - s.si0) * nsj;
                for (int q = lane; q < nsj * NV; q += 32) {
                    S[row * NV + q] = 0.f;
                    S[(nsub + row) * NV + q] = 0.f;
                }
                __syncwarp();
                const int ra = max(s.pi0, si * k) - si * k, rb = min(s.pi1, si * k + k - 1) - si * k;
                const int c1 = WF.irrc_row[si + 1];
                if (ra <= rb && c1 > WF.irrc_row[si]) {
                    Eval<NV> ev;
                    ev.load(s, s_win, D.Wp, D.W, WF.M);
                    for (int c = WF.irrc_row[si]; c < c1; ++c) {
                        const int sj = WF.irrc[c].x;
                        if (sj < s.sj0 || sj > s.sj1) continue;
                        const long sr = (long)(si * WF.n_sub + sj) * k;
                        const int e0 = WF.irr_sr[sr + ra], e1 = WF.irr_sr[sr + rb + 1];
                        float ax[NV], ay[NV], v[NV];
#pragma unroll
                        for (int t = 0; t < NV; ++t) ax[t] = ay[t] = 0.f;
                        for (int e = e0 + lane; e < e1; e += 32) {
                            const int pix = WF.irr_pix[e];
                            const int i = pix >> 16, j = pix & 0xffff;
                            if (j < s.pj0 || j > s.pj1) continue;
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
                            const int idx = row + sj - s.sj0;
#pragma unroll
                            for (int t = 0; t < NV; ++t) {
                                S[idx * NV + t] = ax[t];
                                S[(nsub + idx) * NV + t] = ay[t];
                            }
                        }
                    }
                }
                __syncwarp();
            }
            __syncthreads();
            if (gi == ng - 1 && tid == 0 && next_item < g.n_items) {
                // the window is no longer read: stage the next actuator's
                fence_proxy_async_smem();
                issue_window(g, next_item, s_win, bar);
            }
            // finalize the subaperture sums of every sensor of the group, and
            // stream zeros over every output column of the group (no loads)
            {
                int seq = 0;
                for (int w = 0; w < g.n_wfs; ++w) {
                    const ItemWfs &s = s_info[w];
                    if (s.group != gi || s.empty) continue;
                    const int nq = 2 * (s.si1 - s.si0 + 1) * (s.sj1 - s.sj0 + 1);
                    int q = tid - seq % nth;
                    if (q < 0) q += nth;
                    for (; q < nq; q += nth) finalize_sub<NV>(s, g.wfs[w], s_arena + s.arena, q);
                    seq += nq;
                }
                if (MODE != MODE_VJP) {
                    for (int w = 0; w < g.n_wfs; ++w) {
                        if (s_info[w].group != gi) continue;
                        const DevPair &P = pairs[d * g.n_wfs + w];
                        const int nv = g.wfs[w].nv, n2 = 2 * nv;
                        const int nout = (MODE == MODE_FWD) ? 1 : 5;
                        for (int t = 0; t < nout; ++t) {
                            float *dst = (t == 0) ? P.im : P.dim[t - 1];
                            if (!dst) continue;
                            dst += (size_t)a * n2;
                            if ((nv & 1) == 0) {
                                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                                for (int q = tid; q < n2 / 4; q += nth) reinterpret_cast<float4 *>(dst)[q] = z;
                            } else {
                                const float2 z = make_float2(0.f, 0.f);
                                for (int q = tid; q < nv; q += nth) reinterpret_cast<float2 *>(dst)[q] = z;
                            }
                        }
                    }
                }
            }
            __syncthreads();
            // the box subapertures' slopes: scattered stores over the zeroed
            // columns (MODE_FWD / MODE_TAN) or the VJP dot product
            {
                int seq = 0;
                for (int w = 0; w < g.n_wfs; ++w) {
                    const ItemWfs &s = s_info[w];
                    if (s.group != gi) continue;
                    const int pidx = d * g.n_wfs + w;
                    const DevPair &P = pairs[pidx];
                    if (MODE == MODE_VJP && !P.gim) continue;
                    const DevWFS &WF = g.wfs[w];
                    const int nv = WF.nv, n2 = 2 * nv;
                    const int nsj = s.sj1 - s.sj0 + 1, nsub = (s.si1 - s.si0 + 1) * nsj;
                    const int nq = s.empty ? 0 : 2 * nsub;
                    const float *S = s_arena + s.arena + NV * (2 * s.nxc * s.nb + 2 * s.nyc * s.nbr);
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    int q = tid - seq % nth;
                    if (q < 0) q += nth;
                    for (; q < nq; q += nth) {
                        const int comp = q >= nsub ? 1 : 0, idx = q - comp * nsub;
                        const int si = s.si0 + idx / nsj, sj = s.sj0 + idx % nsj;
                        const int row = WF.vidx[si * WF.n_sub + sj];
                        if (row < 0) continue;
                        const float f = WF.fac[row];
                        const size_t at = (size_t)a * n2 + comp * nv + row;
                        if (MODE == MODE_VJP) {
                            const float gv = P.gim[at];
#pragma unroll
                            for (int t = 0; t < 4; ++t) acc[t] = fmaf(gv, S[q * NV + t + 1] * f, acc[t]);
                        } else {
                            if (P.im) P.im[at] = S[q * NV] * f;
                            if (MODE == MODE_TAN)
#pragma unroll
                                for (int t = 0; t < 4; ++t)
                                    if (P.dim[t]) P.dim[t][at] = S[q * NV + t + 1] * f;
                        }
                    }
                    seq += nq;
                    if (MODE == MODE_VJP) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            float vsum = acc[t];
                            for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
                            if (lane == 0 && vsum != 0.f) atomicAdd(&s_gp[pidx * 4 + t], (double)vsum);
                        }
                    }
                }
            }
            __syncthreads();
        }
        item = next_item;
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
