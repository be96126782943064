// synim_kernels.cu -- sm_103a kernels of the synthetic interaction-matrix path.
//
// k_support / k_pack  (create time) scan each influence function for its
//                     support box and pack it into a zero-bordered window.
// k_pst_core / _codes (every call) edge-repair pixel classes per pair,
//                     Sec. 2.3 steps 1-2: the DM mask carried by the composite
//                     affine, strictly binarised at 0.999999 (decided in FP64,
//                     exactly as the definition), and the cross-dilated ring.
// k_im<MODE>          (every call) one launch over every (actuator, sensor)
//                     column of every DM (Sec. 4.2: all sensors in one pass);
//                     one warp per column, the columns of one actuator in
//                     consecutive warps of a CTA so that its packed window is
//                     fetched from HBM once and served to the others from L1.
//                     Box row by box row the warp resamples the IF at the
//                     boundary line pixels (Sec. 2.1), repairs ring pixels
//                     (Sec. 2.3), forms the telescoped boundary segments and
//                     the subaperture means of the central differences (Sec.
//                     2.2), and writes the column once (16-byte stores for the
//                     zero runs).  No warp ever waits for another.
// k_tele              (every call, telescoping-sum engine of Sec. 2.2) the same
//                     one-warp-per-column launch; a slope is the signed sum of
//                     the IF resampled at the half-pixel ends of the lit runs
//                     of its subaperture (create-time event tables), without
//                     pixel classes or edge repair.  A run end shared by two
//                     valid neighbours is resampled once and credited to both.
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

// win[a][r][c] = IF_a(wy0 + r - pad, wx0 + c - pad) for pad <= r, c < pad + W,
// zero elsewhere (a zero border of pad pixels).
__global__ void k_pack(const float *__restrict__ cube, int N, const int *__restrict__ org, int W,
                       int Wp, int stride, float *__restrict__ win, int pad) {
    const int a = blockIdx.x;
    const int wx0 = org[2 * a], wy0 = org[2 * a + 1];
    const float *img = cube + (size_t)a * N * N;
    float *dst = win + (size_t)a * stride;
    for (int idx = threadIdx.x; idx < stride; idx += blockDim.x) {
        float v = 0.f;
        const int r = idx / Wp, c = idx - r * Wp;
        if (idx < Wp * Wp && r >= pad && r < pad + W && c >= pad && c < pad + W) {
            const int x = wx0 + c - pad, y = wy0 + r - pad;
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
                        int stride, float *win, cudaStream_t s, int pad) {
    k_pack<<<n_act, 256, 0, s>>>(cube, N, org, W, Wp, stride, win, pad);
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
__device__ __forceinline__ int core_at(const DevPair &P, const uint8_t *__restrict__ mask,
                                       const uint8_t *__restrict__ mcls, int N, int i, int j) {
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
            const int c = mcls[(long)(iy + 1) * (N + 1) + (ix + 1)];
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
    return core;
}

// Four consecutive pixels (row-major over the M x M grid) per thread, stored
// as one 32-bit word where aligned.
__global__ void k_pst_core(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs) {
    const int p = blockIdx.y;
    const int d = p / g.n_wfs, w = p - d * g.n_wfs;
    const int M = g.wfs[w].M;
    const long MM = (long)M * M;
    const long q0 = 4 * ((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (q0 >= MM) return;
    const DevPair &P = pairs[p];
    uint8_t *pst = P.pst;
    if (!pst) return;
    const int N = g.dm[d].N;
    const uint8_t *mask = g.dm[d].mask, *mcls = g.dm[d].mcls;
    int c[4];
    // M * M < 2^31: 32-bit index arithmetic, the row advanced as j wraps
    int i = (int)q0 / M, j = (int)q0 - i * M;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        c[e] = 0;
        if (q0 + e < MM) c[e] = core_at(P, mask, mcls, N, i, j);
        if (++j == M) {
            j = 0;
            ++i;
        }
    }
    if (q0 + 3 < MM && (reinterpret_cast<uintptr_t>(pst + q0) & 3u) == 0) {
        *reinterpret_cast<uint32_t *>(pst + q0) = (uint32_t)c[0] | ((uint32_t)c[1] << 8) | ((uint32_t)c[2] << 16) |
                                                  ((uint32_t)c[3] << 24);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (q0 + e < MM) pst[q0 + e] = (uint8_t)c[e];
    }
}

// Class of a sensor pixel from the core map: 1 core, 2 ring (Sec. 2.3 step 2:
// a non-core pixel with a core 4-neighbour), 0 otherwise.
__device__ __forceinline__ int pixel_class(const uint8_t *__restrict__ pst, int M, int i, int j) {
    const long q = (long)i * M + j;
    // five independent byte loads (no short-circuit chain)
    const int c = pst[q];
    const int nb = (j + 1 < M ? pst[q + 1] : 0) | (j >= 1 ? pst[q - 1] : 0) | (i + 1 < M ? pst[q + M] : 0) |
                   (i >= 1 ? pst[q - M] : 0);
    return c ? 1 : (nb ? 2 : 0);
}

// The same class with the neighbour tests short-circuited (fewer loads where
// most pixels are core: the whole-grid class kernel).
__device__ __forceinline__ int pixel_class_sc(const uint8_t *__restrict__ pst, int M, int i, int j) {
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
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // 2 M (n_sub + 1) < 2^31
    if (idx >= 2 * M * n1) return;
    const DevPair &P = pairs[p];
    if (!P.pst) return;
    const int dir = idx >= M * n1 ? 1 : 0;
    const int r = idx - dir * M * n1;
    const int x = r / n1, b = r - x * n1;
    const int c0 = b * k - 1, c1 = b * k;
    int code;
    if (dir == 0) {
        code = WF.xcode[(long)b * M + x];
        const int k0 = (c0 >= 0) ? pixel_class_sc(P.pst, M, x, c0) : 0;
        const int k1 = (c1 < M) ? pixel_class_sc(P.pst, M, x, c1) : 0;
        P.xcc[r] = (uint8_t)(code | (k0 << 4) | (k1 << 6));
    } else {
        code = WF.ycode[(long)b * M + x];
        const int k0 = (c0 >= 0) ? pixel_class_sc(P.pst, M, c0, x) : 0;
        const int k1 = (c1 < M) ? pixel_class_sc(P.pst, M, c1, x) : 0;
        P.ycc[r] = (uint8_t)(code | (k0 << 4) | (k1 << 6));
    }
}

cudaError_t launch_pst(const Geo &g, const DevPair *pairs, int max_mm, int max_lines, cudaStream_t s) {
    dim3 grid((max_mm + 1023) / 1024, g.n_dm * g.n_wfs);
    k_pst_core<<<grid, 256, 0, s>>>(g, pairs);
    dim3 grid2((2 * max_lines + 255) / 256, g.n_dm * g.n_wfs);
    k_pst_codes<<<grid2, 256, 0, s>>>(g, pairs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Every call: boundary-segment weight boxes
// ---------------------------------------------------------------------------
// A boundary segment is the two pixel lines at a subaperture boundary (pixels
// b k - 1 and b k) over one subaperture row (x) or column (y).  Its
// telescoped sums (Sec. 2.2) A (credited to the subaperture before the
// boundary) and B (after) add the bilinear resamples (Sec. 2.1) of its core
// pixels, selected by the sensor's pupil bits.  A window origin is a whole DM
// pixel, so the fractional sample positions, the pixel classes (Sec. 2.3)
// and the bits belong to the (DM, sensor) pair, not to the actuator: A and B
// are dot products of one box of DM-pixel weights with any actuator's packed
// window.  k_kseg builds those boxes once per call; the IM kernel then reads
// BA x BC taps per segment instead of resampling 2 k pixels.  A ring pixel's
// repair reaches beyond the box: it is left out of the box and listed, and the
// IM kernel repairs it from its core neighbours.  Segments whose samples do not
// fit the pair's box are flagged KF_FALLBACK and keep the per-sample path.

// Shape code (ori << 8) | (BA << 4) | BC of one axis, or -1.  The samples of a
// segment are 2 pixels across by k along (x segments: along the sensor rows);
// their DM extents bound the taps per axis by floor(extent) + 3.  The box
// takes floor(extent + 0.9) + 2 (segments that need the last tap fall back)
// rounded up to a supported size.
int kseg_shape(const double A[4], int k, int axis) {
    const double jx = std::fabs(A[0]), ix = std::fabs(A[1]), jy = std::fabs(A[2]), iy = std::fabs(A[3]);
    const double dx = axis == 0 ? jx + (k - 1) * ix : ix + (k - 1) * jx;
    const double dy = axis == 0 ? jy + (k - 1) * iy : iy + (k - 1) * jy;
    const int ori = dy >= dx ? 0 : 1;                 // along the larger DM extent
    const double dl = ori ? dx : dy, dc = ori ? dy : dx;
    int BA = (int)std::floor(dl + 0.9) + 2, BC = (int)std::floor(dc + 0.9) + 2;
    if (BA <= 4) BA = 4;
    else if (BA <= 6) BA = 6;
    else if (BA <= 8) BA = 8;
    else if (BA > KBA_MAX) return -1;
    if (BC <= 3) BC = 3;
    else if (BC > KBC_MAX) return -1;
    return (ori << 8) | (BA << 4) | BC;
}

__global__ void __launch_bounds__(128) k_kseg(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs) {
    __shared__ float acc[128][2 * KTAPS + 1];
    const int p = blockIdx.y;
    const DevPair &P = pairs[p];
    if (!P.kf || (int)blockIdx.z >= P.kcomp) return;
    const DevWFS &WF = g.wfs[p % g.n_wfs];
    const int n = WF.n_sub, n1 = n + 1, k = WF.k;
    const int nseg = n * n1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * nseg) return;
    const int ax = idx >= nseg ? 1 : 0, sid = idx - ax * nseg;
    int row, b;   // x: subaperture row, boundary (sid = row n1 + b); y: boundary, subaperture column (sid = b n + row)
    if (ax == 0) { row = sid / n1; b = sid - row * n1; }
    else { b = sid / n; row = sid - b * n; }
    const uint8_t *cc = (ax ? P.ycc : P.xcc) + b;    // byte of line pixel pair u at cc[u n1]
    const int shape = P.kshape[ax];
    const int ori = shape >> 8, BA = (shape >> 4) & 15, BC = shape & 15;
    const int ex = ori ? BA : BC, ey = ori ? BC : BA;  // box extents along DM x and y
    const int u0 = row * k, l0 = b * k - 1;
    // sample (q, t) = line pixel t of pair u0 + q: sensor pixel (i, j)
    auto pix = [&](int q, int t, int &i, int &j) {
        if (ax == 0) { i = u0 + q; j = l0 + t; }
        else { i = l0 + t; j = u0 + q; }
    };
    int i, j;
    pix(0, 0, i, j);
    const float xf = fmaf(P.Ahi[0], (float)j, fmaf(P.Ahi[1], (float)i, P.bhi[0]));
    const float yf = fmaf(P.Ahi[2], (float)j, fmaf(P.Ahi[3], (float)i, P.bhi[1]));
    int flags = 0, ring = 0;
    bool any = false, asym = false;
    int ox = 0, oy = 0, cx0 = INT_MAX, cx1 = INT_MIN, cy0 = INT_MAX, cy1 = INT_MIN;
    int qa = KF_MAX_K, qb = -1, ta = 1, tb = 0;   // rectangle of the core samples with stencil bits
    // the segment's class bytes, loaded together (k <= KF_MAX_K)
    int cb[KF_MAX_K];
#pragma unroll
    for (int q = 0; q < KF_MAX_K; ++q) cb[q] = q < k ? cc[(long)(u0 + q) * n1] : 0;
    if (!(fabsf(xf) < 1e5f && fabsf(yf) < 1e5f)) {
        flags = KF_FALLBACK;
    } else {
        ox = (int)floorf(xf) - 1;
        oy = (int)floorf(yf) - 1;
#pragma unroll
        for (int q = 0; q < KF_MAX_K; ++q) {
            if (q >= k) break;
            const int c = cb[q];
            for (int t = 0; t < 2; ++t) {
                const int cl = (c >> (4 + 2 * t)) & 3;
                const int ba = c & (t ? 4 : 1), bb = c & (t ? 8 : 2);
                if (!(ba || bb) || cl == 0) continue;
                if (cl == 2) {   // repaired by the IM kernel from its core neighbours
                    ring |= 1 << (2 * q + t);
                    continue;
                }
                qa = min(qa, q); qb = max(qb, q); ta = min(ta, t); tb = max(tb, t);
                any = true;
                if ((ba != 0) != (bb != 0)) asym = true;
            }
        }
        // the map is affine: the extreme cells of the core samples lie at the
        // corners of their (q, t) rectangle (the second pass checks each sample)
        if (any)
            for (int e = 0; e < 4; ++e) {
                pix((e & 1) ? qb : qa, (e & 2) ? tb : ta, i, j);
                const float xl = exact_affine(P.Ahi[0], P.Alo[0], P.Ahi[1], P.Alo[1], P.bhi[0], P.blo[0], j, i, ox);
                const float yl = exact_affine(P.Ahi[2], P.Alo[2], P.Ahi[3], P.Alo[3], P.bhi[1], P.blo[1], j, i, oy);
                const int cx = (int)floorf(xl), cy = (int)floorf(yl);
                cx0 = min(cx0, cx); cx1 = max(cx1, cx); cy0 = min(cy0, cy); cy1 = max(cy1, cy);
            }
    }
    int gx = 0, gy = 0;
    if (!(flags & KF_FALLBACK) && any) {
        gx = ox + cx0;
        gy = oy + cy0;
        if (cx1 - cx0 + 2 > ex || cy1 - cy0 + 2 > ey || gx < -2048 || gx > 2047 || gy < -2048 || gy > 2047)
            flags |= KF_FALLBACK;
    }
    if (!any) flags |= KF_NOCORE;
    if (ring && !(flags & KF_FALLBACK)) {
        flags |= KF_RING;
        if (blockIdx.z == 0) P.kring[ax][sid] = ring;
    }
    if (!(flags & (KF_FALLBACK | KF_NOCORE))) {
        if (asym) flags |= KF_ASYM;
        float *wa = acc[threadIdx.x], *wb = wa + KTAPS;
        bool overflow = false;
        // component 0: the resampled value; 1..4 (P.kcomp = 5): its
        // derivatives with respect to p_k through the sample position, the
        // pixel classes held fixed (d phi = gx dx_k + gy dy_k, with gx, gy the
        // bilinear cell's differences and (dx_k, dy_k) = d(A, b)/dp_k (j, i))
        {
        const int comp = blockIdx.z;   // one component per thread (grid z)
        float dA[4] = {0.f, 0.f, 0.f, 0.f}, db[2] = {0.f, 0.f};
        if (comp > 0)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                dA[e] = (float)P.dA[4 * (comp - 1) + e];
                if (e < 2) db[e] = (float)P.db[2 * (comp - 1) + e];
            }
        for (int q = 0; q < 2 * KTAPS; ++q) wa[q] = 0.f;
#pragma unroll
        for (int q = 0; q < KF_MAX_K; ++q) {
            if (q >= k) break;
            const int c = cb[q];
            for (int t = 0; t < 2; ++t) {
                const int cl = (c >> (4 + 2 * t)) & 3;
                const int ba = c & (t ? 4 : 1), bb = c & (t ? 8 : 2);
                if (!(ba || bb) || cl != 1) continue;
                pix(q, t, i, j);
                // the same local coordinates as the first pass, so the cells agree with its extents
                const float xl = exact_affine(P.Ahi[0], P.Alo[0], P.Ahi[1], P.Alo[1], P.bhi[0], P.blo[0], j, i, ox);
                const float yl = exact_affine(P.Ahi[2], P.Alo[2], P.Ahi[3], P.Alo[3], P.bhi[1], P.blo[1], j, i, oy);
                const float fx0 = floorf(xl), fy0 = floorf(yl);
                const int cx = (int)fx0 - cx0, cy = (int)fy0 - cy0;
                if (cx < 0 || cy < 0 || cx + 1 >= ex || cy + 1 >= ey) {
                    overflow = true;   // a rounding past the corners' cells: per-sample path
                    continue;
                }
                const float fx = xl - fx0, fy = yl - fy0, hx = 1.f - fx, hy = 1.f - fy;
                float wq[4];
                if (comp == 0) {
                    wq[0] = hx * hy; wq[1] = fx * hy; wq[2] = hx * fy; wq[3] = fx * fy;
                } else {
                    const float dx = fmaf(dA[0], (float)j, fmaf(dA[1], (float)i, db[0]));
                    const float dy = fmaf(dA[2], (float)j, fmaf(dA[3], (float)i, db[1]));
                    wq[0] = -hy * dx - hx * dy;
                    wq[1] = hy * dx - fx * dy;
                    wq[2] = -fy * dx + hx * dy;
                    wq[3] = fy * dx + fx * dy;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int tx = cx + (e & 1), ty = cy + (e >> 1);
                    const int tap = ori ? tx * KBC_MAX + ty : ty * KBC_MAX + tx;
                    if (ba) wa[tap] += wq[e];
                    if (bb) wb[tap] += wq[e];
                }
            }
        }
        if (overflow) {
            flags |= KF_FALLBACK;
        } else {
            float *ka = P.kw[ax] + sid + (long)comp * KTAPS * KPS, *kb = P.kwb[ax] + sid + (long)comp * KTAPS * KPS;
            for (int q = 0; q < KTAPS; ++q) ka[(long)q * KPS] = wa[q];
            if (asym)
                for (int q = 0; q < KTAPS; ++q) kb[(long)q * KPS] = wb[q];
        }
        }
    }
    if (blockIdx.z == 0) P.korg[ax][sid] = (gx & 0xfff) | ((gy & 0xfff) << 12) | (flags << 24);
}

cudaError_t launch_kseg(const Geo &g, const DevPair *pairs, int max_seg, int ncomp, cudaStream_t s) {
    if (max_seg <= 0) return cudaSuccess;
    dim3 grid((2 * max_seg + 127) / 128, g.n_dm * g.n_wfs, ncomp);
    k_kseg<<<grid, 128, 0, s>>>(g, pairs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The IM kernel
// ---------------------------------------------------------------------------
// Per (actuator, sensor): the pixel box where the resampled, repaired IF can
// be non-zero, the subaperture box whose slopes can be non-zero, and the
// local coordinates of the box origin in the packed window.
struct ItemWfs {
    int pi0, pi1, pj0, pj1;  // pixel box (inclusive)
    int si0, si1, sj0, sj1;  // subaperture box (inclusive)
    int nsj, nsub;           // box width and size in subapertures
    int empty;
    float xo, yo;            // padded-window coordinates of pixel (pi0, pj0)
    float a00, a01, a10, a11;
    float dxo[4], dyo[4], da[16];  // tangents of the coordinates (MODE_TAN / MODE_VJP)
    const uint8_t *pst, *xcc, *ycc;
};

template <int NV>
struct Eval {
    static constexpr int NT = (NV == 5) ? 4 : 1;  // tangent parameters held
    const float *win;
    const uint8_t *pst;
    int Wp, M, pi0, pj0;
    float xlo, xhi, xo, yo, a00, a01, a10, a11;   // window data at padded coordinates (xlo, xhi)
    float dxo[NT], dyo[NT], da[4 * NT];
#ifdef SYNIM_DEBUG_BOUNDS
    int *err;   // the context's error flag
    long wn;    // floats of this actuator's packed window
#endif

    // w: the actuator's packed window, pitch wp, data W x W after a zero border of pad pixels
    __device__ __forceinline__ void load(const ItemWfs &s, const float *w, int wp, int W, int m, int pad = 1) {
        win = w; pst = s.pst; Wp = wp; M = m; pi0 = s.pi0; pj0 = s.pj0;
        xlo = (float)(pad - 1); xhi = (float)(W + pad); xo = s.xo; yo = s.yo;
        a00 = s.a00; a01 = s.a01; a10 = s.a10; a11 = s.a11;
        if (NV == 5) {
#pragma unroll
            for (int k = 0; k < 4; ++k) { dxo[k] = s.dxo[k]; dyo[k] = s.dyo[k]; }
#pragma unroll
            for (int k = 0; k < 16; ++k) da[k] = s.da[k];
        }
    }

    // Bilinear resample of the packed window at sensor pixel (i, j) (Sec. 2.1);
    // v[0] = phi, v[1..4] = d phi / d p_k (chain rule through the floor cell).
    __device__ __forceinline__ void bil(int i, int j, float *v) const {
        const float di = (float)(i - pi0), dj = (float)(j - pj0);
        const float x = fmaf(a00, dj, fmaf(a01, di, xo));
        const float y = fmaf(a10, dj, fmaf(a11, di, yo));
        if (!(x > xlo && x < xhi && y > xlo && y < xhi)) {
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = 0.f;
            return;
        }
        const float fx0 = floorf(x), fy0 = floorf(y);
        const int ix = (int)fx0, iy = (int)fy0;
        const float fx = x - fx0, fy = y - fy0;
        if (!SYNIM_IDX_OK(ix >= 0 && iy >= 0 && (long)iy * Wp + ix + Wp + 1 < wn, err)) {
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = 0.f;
            return;
        }
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

    // Bilinear value at padded-window coordinates (x, y) (no tangents).
    __device__ __forceinline__ float bil_at(float x, float y) const {
        if (!(x > xlo && x < xhi && y > xlo && y < xhi)) return 0.f;
        const float fx0 = floorf(x), fy0 = floorf(y);
        const float fx = x - fx0, fy = y - fy0;
        if (!SYNIM_IDX_OK(fx0 >= 0.f && fy0 >= 0.f && (long)fy0 * Wp + (long)fx0 + Wp + 1 < wn, err)) return 0.f;
        const float *q = win + (int)fy0 * Wp + (int)fx0;
        const float v00 = q[0], v10 = q[1], v01 = q[Wp], v11 = q[Wp + 1];
        const float top = fmaf(fx, v10 - v00, v00), bot = fmaf(fx, v11 - v01, v01);
        return fmaf(fy, bot - top, top);
    }

    // Edge repair step 3 (Sec. 2.3) at a ring pixel: mean over the valid
    // cardinal directions of 2 P1 - P2 (or P1); P1, P2 must be strict core.
    __device__ __forceinline__ void ring(int i, int j, float *v) const {
        float acc[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) acc[t] = 0.f;
        int n = 0;
#pragma unroll 1
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

    // acc += wgt * (repaired phase and tangents at (i, j) of class c: 0 zero,
    // 1 core, 2 ring).
    __device__ __forceinline__ void add(int i, int j, int c, float wgt, float *acc) const {
        if (c == 0) return;
        float v[NV];
        if (c == 1) bil(i, j, v);
        else ring(i, j, v);
#pragma unroll
        for (int t = 0; t < NV; ++t) acc[t] = fmaf(wgt, v[t], acc[t]);
    }
};

__device__ __forceinline__ void decode_item(const Geo &g, int item, int &d, int &a) {
    int pos = 0;
    while (pos + 1 < g.n_dm && item >= g.order_start[pos + 1]) ++pos;
    d = g.order_dm[pos];
    a = item - g.order_start[pos];
}

template <int MODE>
__device__ __forceinline__ bool pair_active(const DevPair &P) {
    if (MODE == MODE_FWD) return P.im != nullptr;
    if (MODE == MODE_TAN)
        return P.im || P.dim[0] || P.dim[1] || P.dim[2] || P.dim[3];
    return P.gim != nullptr;
}

// Pixel and subaperture boxes of actuator a on sensor w, local coordinates.
// pad: zero border of the window the column reads (the local coordinates xo,
// yo are relative to DM pixel (wx0 - pad, wy0 - pad)).
template <int MODE, int NV>
__device__ void make_info(const Geo &g, const DevPair *__restrict__ pairs, int d, int a, int w,
                          ItemWfs &s, int *err, int pad = 1) {
    const DevPair &P = pairs[d * g.n_wfs + w];
    const DevWFS &WF = g.wfs[w];
    const DevDM &D = g.dm[d];
    const int M = WF.M, k = WF.k;
    s.pst = P.pst;
    s.xcc = P.xcc;
    s.ycc = P.ycc;
    s.empty = 1;
    s.nsub = 0;
    s.nsj = 1;
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
    const int nsj = sj1 - sj0 + 1, nsub = (si1 - si0 + 1) * nsj;
    (void)err;
    s.empty = 0;
    s.pi0 = pi0; s.pi1 = pi1; s.pj0 = pj0; s.pj1 = pj1;
    s.si0 = si0; s.si1 = si1; s.sj0 = sj0; s.sj1 = sj1;
    s.nsj = nsj;
    s.nsub = nsub;
    s.xo = exact_affine(P.Ahi[0], P.Alo[0], P.Ahi[1], P.Alo[1], P.bhi[0], P.blo[0], pj0, pi0, wx0 - pad);
    s.yo = exact_affine(P.Ahi[2], P.Alo[2], P.Ahi[3], P.Alo[3], P.bhi[1], P.blo[1], pj0, pi0, wy0 - pad);
    s.a00 = P.Ahi[0]; s.a01 = P.Ahi[1]; s.a10 = P.Ahi[2]; s.a11 = P.Ahi[3];
    if (NV == 5) {
        for (int q = 0; q < 4; ++q) {
            s.dxo[q] = (float)(P.dA[4 * q + 0] * pj0 + P.dA[4 * q + 1] * pi0 + P.db[2 * q + 0]);
            s.dyo[q] = (float)(P.dA[4 * q + 2] * pj0 + P.dA[4 * q + 3] * pi0 + P.db[2 * q + 1]);
        }
        for (int q = 0; q < 16; ++q) s.da[q] = (float)P.dA[q];
    }
}

// One boundary segment (Sec. 2.2, telescoped): the two pixel lines at
// boundary b (pixels b k - 1 and b k) over one subaperture row (x) or column
// (y), restricted to the pixel box.  A collects their contributions to the
// subaperture before the boundary (bits 0 and 2 of the boundary byte), B to
// the one after (bits 1 and 3); the slope of subaperture s along x is then
// A(b = sj + 1) - B(b = sj) plus its pupil-edge pixels.
struct SegRows {
    int ua, ub, l0, inmask, b;
    const uint8_t *cc;
};

__device__ __forceinline__ SegRows seg_rows(const DevWFS &WF, const ItemWfs &s, int axis, int b, int sq) {
    const int k = WF.k;
    SegRows r;
    const int u0 = sq * k;
    r.ua = max(u0, axis ? s.pj0 : s.pi0);
    r.ub = min(u0 + k - 1, axis ? s.pj1 : s.pi1);
    r.l0 = b * k - 1;
    const int c0 = axis ? s.pi0 : s.pj0, c1 = axis ? s.pi1 : s.pj1;
    r.inmask = ((r.l0 >= c0 && r.l0 <= c1) ? 1 : 0) | ((r.l0 + 1 >= c0 && r.l0 + 1 <= c1) ? 2 : 0);
    r.cc = (axis ? s.ycc : s.xcc) + b;
    r.b = b;
    return r;
}

// This lane's share of a segment: pixel rows ua + lane0, ua + lane0 + lstep, ...
template <int NV>
__device__ __forceinline__ void seg_compute(const DevWFS &WF, const SegRows &r, const Eval<NV> &ev, int axis,
                                            int lane0, int lstep, float *A, float *B) {
    if (!r.inmask) return;
    const int n1 = WF.n_sub + 1, l0 = r.l0, inmask = r.inmask;
    // line bytes [u][b]: rows ua .. ub of the sensor, boundary b <= n_sub;
    // line pixels l0, l0 + 1 inside the sensor where their class is read
    if (!SYNIM_IDX_OK(r.ua >= 0 && r.ub < WF.M && r.b >= 0 && r.b < n1 && l0 >= -1 && l0 + 1 <= WF.M, ev.err))
        return;
    const int u0 = r.ua + lane0;
    if (u0 > r.ub) return;
    const uint8_t *cp = r.cc + (long)u0 * n1;
    const int cstep = lstep * n1;
    if constexpr (NV == 1) {
        // the sampled DM points move by a constant step along the line; the
        // second line pixel is one sensor pixel across
        const float di = (float)((axis ? l0 : u0) - ev.pi0), dj = (float)((axis ? u0 : l0) - ev.pj0);
        const float x0 = fmaf(ev.a00, dj, fmaf(ev.a01, di, ev.xo));
        const float y0 = fmaf(ev.a10, dj, fmaf(ev.a11, di, ev.yo));
        // lstep is a power of two: the step is exact, each point one rounding
        const float sx = (float)lstep * (axis ? ev.a00 : ev.a01), sy = (float)lstep * (axis ? ev.a10 : ev.a11);
        const float ox = axis ? ev.a01 : ev.a00, oy = axis ? ev.a11 : ev.a10;
        float qf = 0.f;
        // the next pixel pair's byte is loaded before this one's resamples
        int c_next = __ldg(cp);
        for (int u = u0; u <= r.ub; u += lstep, qf += 1.f, cp += cstep) {
            const float x = fmaf(qf, sx, x0), y = fmaf(qf, sy, y0);
            const int c = c_next;
            if (u + lstep <= r.ub) c_next = __ldg(cp + cstep);
            const int cl0 = (inmask & 1) ? (c >> 4) & 3 : 0, cl1 = (inmask & 2) ? (c >> 6) & 3 : 0;
            float v0, v1;
            if (cl0 == 2 || cl1 == 2) {
                float t0[1] = {0.f}, t1[1] = {0.f};
                if (cl0 == 1) ev.bil(axis ? l0 : u, axis ? u : l0, t0);
                else if (cl0 == 2) ev.ring(axis ? l0 : u, axis ? u : l0, t0);
                if (cl1 == 1) ev.bil(axis ? l0 + 1 : u, axis ? u : l0 + 1, t1);
                else if (cl1 == 2) ev.ring(axis ? l0 + 1 : u, axis ? u : l0 + 1, t1);
                v0 = t0[0];
                v1 = t1[0];
            } else {
                v0 = cl0 ? ev.bil_at(x, y) : 0.f;
                v1 = cl1 ? ev.bil_at(x + ox, y + oy) : 0.f;
            }
            A[0] += ((c & 1) ? v0 : 0.f) + ((c & 4) ? v1 : 0.f);
            B[0] += ((c & 2) ? v0 : 0.f) + ((c & 8) ? v1 : 0.f);
        }
    } else {
        for (int u = u0; u <= r.ub; u += lstep, cp += cstep) {
            const int c = __ldg(cp);
            const int cl0 = (inmask & 1) ? (c >> 4) & 3 : 0, cl1 = (inmask & 2) ? (c >> 6) & 3 : 0;
            const float wa0 = (c & 1) ? 1.f : 0.f, wb0 = (c & 2) ? 1.f : 0.f;
            const float wa1 = (c & 4) ? 1.f : 0.f, wb1 = (c & 8) ? 1.f : 0.f;
            float v0[NV], v1[NV];
            if (cl0 == 2 || cl1 == 2) {
#pragma unroll
                for (int t = 0; t < NV; ++t) v0[t] = v1[t] = 0.f;
                if (cl0 == 1) ev.bil(axis ? l0 : u, axis ? u : l0, v0);
                else if (cl0 == 2) ev.ring(axis ? l0 : u, axis ? u : l0, v0);
                if (cl1 == 1) ev.bil(axis ? l0 + 1 : u, axis ? u : l0 + 1, v1);
                else if (cl1 == 2) ev.ring(axis ? l0 + 1 : u, axis ? u : l0 + 1, v1);
            } else {
                // both pixels core or zero: two independent gathers, zero
                // weight for a zero-class pixel
                ev.bil(axis ? l0 : u, axis ? u : l0, v0);
                ev.bil(axis ? l0 + 1 : u, axis ? u : l0 + 1, v1);
                if (cl0 == 0)
#pragma unroll
                    for (int t = 0; t < NV; ++t) v0[t] = 0.f;
                if (cl1 == 0)
#pragma unroll
                    for (int t = 0; t < NV; ++t) v1[t] = 0.f;
            }
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                A[t] = fmaf(wa0, v0[t], fmaf(wa1, v1[t], A[t]));
                B[t] = fmaf(wb0, v0[t], fmaf(wb1, v1[t], B[t]));
            }
        }
    }
}

// Pupil-edge pixels of subaperture (si, sj) inside the pixel box, both axes
// at once: ax += wx(q) phi(q), ay += wy(q) phi(q); the warp's lanes split the
// entries (lane0, lstep) and the caller reduces.
template <int NV>
__device__ __forceinline__ void edge_sum(const DevWFS &WF, const ItemWfs &s, const Eval<NV> &ev, int si, int sj,
                                         int lane0, int lstep, float *ax, float *ay) {
    const int k = WF.k;
    const int ra = max(si * k, s.pi0), rb = min(si * k + k - 1, s.pi1);
    if (ra > rb) return;
    const long sr = (long)(si * WF.n_sub + sj) * k - (long)si * k;
    if (!SYNIM_IDX_OK(si >= 0 && sj >= 0 && si < WF.n_sub && sj < WF.n_sub && sr + ra >= 0 &&
                      sr + rb + 1 <= (long)WF.n_sub * WF.n_sub * k, ev.err))
        return;
    const int e0 = WF.irr_sr[sr + ra], e1 = WF.irr_sr[sr + rb + 1];
    if (!SYNIM_IDX_OK(e0 >= 0 && e1 <= WF.n_irr, ev.err)) return;
    for (int e = e0 + lane0; e < e1; e += lstep) {
        const int pix = WF.irr_pix[e];
        const int i = pix >> 16, j = pix & 0xffff;
        if (j < s.pj0 || j > s.pj1) continue;
        if (!SYNIM_IDX_OK(i >= 0 && i < WF.M && j < WF.M, ev.err)) continue;
        const float wx = WF.irr_w[2 * e], wy = WF.irr_w[2 * e + 1];
        float v[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) v[t] = 0.f;
        const int c = pixel_class(s.pst, WF.M, i, j);
        if constexpr (NV == 1) {
            // resample while the class loads; keep it for a core pixel
            float b1[1];
            ev.bil(i, j, b1);
            if (c == 1) v[0] = b1[0];
            else if (c == 2) ev.ring(i, j, v);
        } else {
            if (c == 1) ev.bil(i, j, v);
            else if (c == 2) ev.ring(i, j, v);
        }
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            ax[t] = fmaf(wx, v[t], ax[t]);
            ay[t] = fmaf(wy, v[t], ay[t]);
        }
    }
}

// The same sums for large subapertures (k > 32) from the create-time tiles:
// only the 16 x 16 pixel tiles that the pixel box overlaps are read, their
// entries spread over the lanes (entries outside the box are skipped, as in
// edge_sum).  Each lane accumulates its entries in a fixed order.
template <int NV>
__device__ __forceinline__ void edge_sum_tiles(const DevWFS &WF, const ItemWfs &s, const Eval<NV> &ev, int si,
                                               int sj, int lane, float *ax, float *ay) {
    const int k = WF.k, T = WF.tl_n;
    const int i0 = max(si * k, s.pi0), i1 = min(si * k + k - 1, s.pi1);
    const int j0 = max(sj * k, s.pj0), j1 = min(sj * k + k - 1, s.pj1);
    if (i0 > i1 || j0 > j1) return;
    const int ti0 = (i0 - si * k) >> 4, ti1 = (i1 - si * k) >> 4;
    const int tj0 = (j0 - sj * k) >> 4, tj1 = (j1 - sj * k) >> 4;
    const int ntj = tj1 - tj0 + 1, ntiles = (ti1 - ti0 + 1) * ntj;
    const int base = (si * WF.n_sub + sj) * T * T;
    for (int g0 = 0; g0 < ntiles; g0 += 32) {
        const int tq = g0 + lane;
        int st = 0, cnt = 0;
        if (tq < ntiles) {
            const int a = tq / ntj, b = tq - a * ntj;
            const int tile = base + (ti0 + a) * T + tj0 + b;
            if (SYNIM_IDX_OK(tile >= 0 && tile < WF.n_sub * WF.n_sub * T * T, ev.err)) {
                st = WF.tl_start[tile];
                cnt = WF.tl_start[tile + 1] - st;
            }
        }
        int pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        const int total = __shfl_sync(0xffffffffu, pre, 31), excl = pre - cnt;
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int jj = e0 + lane;
            int own = 0;   // the last lane whose first entry is at or before jj
#pragma unroll
            for (int st2 = 16; st2 > 0; st2 >>= 1)
                if (__shfl_sync(0xffffffffu, excl, own + st2) <= jj) own += st2;
            const int ost = __shfl_sync(0xffffffffu, st, own), oex = __shfl_sync(0xffffffffu, excl, own);
            if (jj >= total) continue;
            const int e = ost + (jj - oex);
            if (!SYNIM_IDX_OK(e >= 0 && e < WF.n_irr, ev.err)) continue;
            const int pix = WF.tl_pix[e];
            const int i = pix >> 16, j = pix & 0xffff;
            if (i < i0 || i > i1 || j < j0 || j > j1) continue;
            const float wx = WF.tl_w[2 * e], wy = WF.tl_w[2 * e + 1];
            float v[NV];
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = 0.f;
            const int c = pixel_class(s.pst, WF.M, i, j);
            if (c == 1) ev.bil(i, j, v);
            else if (c == 2) ev.ring(i, j, v);
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                ax[t] = fmaf(wx, v[t], ax[t]);
                ay[t] = fmaf(wy, v[t], ay[t]);
            }
        }
    }
}

// Zero rows [r0, r1) of a 16-byte-aligned column: lanes store the unaligned
// head and tail, lane 0 issues bulk copies (cp.async.bulk, at most 4 KB each)
// of the CTA's shared zero buffer over the aligned middle.
constexpr int kZeroFloats = 1024;
__shared__ __align__(128) float4 s_zero[kZeroFloats / 4];   // zeroed by k_im at entry

__device__ __forceinline__ void bulk_zero(float *col, int r0, int r1, int lane) {
    if (r0 >= r1) return;
    const int h = min(r1, (r0 + 3) & ~3), t = max(h, r1 & ~3);
    if (lane < h - r0) col[r0 + lane] = 0.f;
    if (lane < r1 - t) col[t + lane] = 0.f;
    if (lane == 0 && h < t) {
        const uint32_t zsrc = (uint32_t)__cvta_generic_to_shared(s_zero);
        for (int q = h; q < t; q += kZeroFloats) {
            const int n = min(kZeroFloats, t - q) * 4;
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(col + q), "r"(zsrc), "r"(n)
                         : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
}

// Zero rows [r0, r1) of one output column (16-byte stores where aligned).
__device__ __forceinline__ void zero_rows(float *col, int r0, int r1, bool vec4, int lane) {
    if (r0 >= r1) return;
    if (!vec4) {
        for (int r = r0 + lane; r < r1; r += 32) col[r] = 0.f;
        return;
    }
    const int h = min(r1, (r0 + 3) & ~3), t = max(h, r1 & ~3);
    if (lane < h - r0) col[r0 + lane] = 0.f;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int c = h / 4 + lane; c < t / 4; c += 32) reinterpret_cast<float4 *>(col)[c] = z;
    if (lane < r1 - t) col[t + lane] = 0.f;
}

// Boundary segments of one box row (x, boundaries sj0 .. sj1 + 1 over the
// subaperture row si) or one row boundary (y, boundary b over the box's
// subaperture columns), warp-cooperative: groups of L lanes share a segment
// and split its pixel rows / columns, then reduce (fixed butterfly order).
// seg[(q) * 2 NV + v] = A, seg[(q) * 2 NV + NV + v] = B of the q-th segment.
template <int NV>
__device__ __forceinline__ void warp_segments(const DevWFS &WF, const ItemWfs &s, const Eval<NV> &ev, int axis,
                                              int fixed, int first, int count, float *seg, int lane, int lanes) {
    // lanes per segment: a whole warp for large k, else the tuned or default count
    const int L = (WF.k > 32) ? 32 : (lanes > 0 ? lanes : (WF.k > 16 ? 8 : 4));
    const int per = 32 / L;
    const int grp = lane / L, q = lane - grp * L;
    // x: boundary first + idx over subaperture row `fixed`; y: boundary
    // `fixed` over subaperture column first + idx
    for (int base = 0; base < count; base += per) {
        const int idx = base + grp;
        float A[NV], B[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) A[v] = B[v] = 0.f;
        if (idx < count) {
            const SegRows r = seg_rows(WF, s, axis, axis ? fixed : first + idx, axis ? first + idx : fixed);
            seg_compute<NV>(WF, r, ev, axis, q, L, A, B);
        }
        for (int o = L >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                A[v] += __shfl_xor_sync(0xffffffffu, A[v], o);
                B[v] += __shfl_xor_sync(0xffffffffu, B[v], o);
            }
        if (q == 0 && idx < count)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                seg[(size_t)idx * 2 * NV + v] = A[v];
                seg[(size_t)idx * 2 * NV + NV + v] = B[v];
            }
    }
}

// ---------------------------------------------------------------------------
// IM columns from the boundary-segment weight boxes
// ---------------------------------------------------------------------------
// t / n for 0 <= t < 2^20 and 0 < n, from inv = 1 / n (one correction step).
__device__ __forceinline__ int fast_div(int t, float inv, int n) {
    int q = (int)(((float)t + 0.5f) * inv);
    if (q * n > t) --q;
    else if ((q + 1) * n <= t) ++q;
    return q;
}

// NC components per segment: the value (q = 0) and, for tangents, its
// derivatives with respect to the four misregistration parameters (q = 1..4),
// each with its own weight planes starting at plane q KTAPS.
// A[q] = sum over the box of kw[q][tap] * window, B[q] likewise with kwb
// (TWO) or A[q].  wb: the window at the box origin; ka / kb: tap 0 of the
// segment's planes.
template <int BA, int BC, int ORI, bool TWO, int NC>
__device__ __forceinline__ void kf_dot(const float *__restrict__ wb, int Wp, const float *__restrict__ ka,
                                       const float *__restrict__ kb, float *A, float *B) {
    float sa[NC], sb[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) sa[q] = sb[q] = 0.f;
    if constexpr (ORI == 0) {   // along the window's rows (stride Wp), across its columns
#pragma unroll
        for (int a = 0; a < BA; ++a) {
            const float *wr = wb + a * Wp;
#pragma unroll
            for (int c = 0; c < BC; ++c) {
                const float v = __ldg(wr + c);
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    const long off = (long)(q * KTAPS + a * KBC_MAX + c) * KPS;
                    sa[q] = fmaf(__ldg(ka + off), v, sa[q]);
                    if (TWO) sb[q] = fmaf(__ldg(kb + off), v, sb[q]);
                }
            }
        }
    } else {                    // along the window's columns, across its rows
#pragma unroll
        for (int c = 0; c < BC; ++c) {
            const float *wr = wb + c * Wp;
#pragma unroll
            for (int a = 0; a < BA; ++a) {
                const float v = __ldg(wr + a);
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    const long off = (long)(q * KTAPS + a * KBC_MAX + c) * KPS;
                    sa[q] = fmaf(__ldg(ka + off), v, sa[q]);
                    if (TWO) sb[q] = fmaf(__ldg(kb + off), v, sb[q]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        A[q] = sa[q];
        B[q] = TWO ? sb[q] : sa[q];
    }
}

template <int ORI, bool TWO, int NC>
__device__ __forceinline__ void kf_dot_ba(int BA, int BC, const float *wb, int Wp, const float *ka,
                                          const float *kb, float *A, float *B) {
#define SYNIM_KF(ba, bc) \
    if (BA == ba && BC == bc) { kf_dot<ba, bc, ORI, TWO, NC>(wb, Wp, ka, kb, A, B); return; }
    SYNIM_KF(9, 3) SYNIM_KF(8, 3) SYNIM_KF(10, 3) SYNIM_KF(6, 3) SYNIM_KF(4, 3)
    SYNIM_KF(9, 4) SYNIM_KF(8, 4) SYNIM_KF(10, 4) SYNIM_KF(6, 4) SYNIM_KF(4, 4)
#undef SYNIM_KF
#pragma unroll
    for (int q = 0; q < NC; ++q) A[q] = B[q] = 0.f;
}

// One pass over cnt segments of axis ax: t = r ncol + c is x segment
// (row0 + r, boundary col0 + c) or y segment (boundary row0 + r, column col0
// + c); out[2 NC t + q] = A[q], out[2 NC t + NC + q] = B[q].  Lanes take one
// segment each; flagged segments are resampled pixel by pixel afterwards by
// the whole warp.  rbuf: 64 NC floats of the warp's buffer for the ring pixels.
template <int NC>
__device__ void kf_pass(const DevWFS &WF, const DevPair &P, const ItemWfs &s, const Eval<NC> &ev,
                        const float *__restrict__ win, int Wp, int W, int wx0, int wy0, int ax, int row0,
                        int ncol, int col0, int cnt, float *out, float *rbuf, int lane, int *err) {
    const int n = WF.n_sub, n1 = n + 1;
    const int shape = P.kshape[ax];
    const int ori = shape >> 8, BA = (shape >> 4) & 15, BC = shape & 15;
    const int ex = ori ? BA : BC, ey = ori ? BC : BA;
    const int *__restrict__ org = P.korg[ax];
    const float *kwa = P.kw[ax], *kwb = P.kwb[ax];
    const int lx0 = wx0 - KPAD, ly0 = wy0 - KPAD;
    const float inv = 1.f / (float)ncol;
    (void)err;
    for (int base = 0; base < cnt; base += 32) {
        const int t = base + lane;
        int sid = 0, fl = 0;
        bool act = false, fb = false;
        const float *wb = win;
        if (t < cnt) {
            const int r = fast_div(t, inv, ncol), c = t - r * ncol;
            sid = ax ? (row0 + r) * n + (col0 + c) : (row0 + r) * n1 + (col0 + c);
            const int word = __ldg(org + sid);
            fl = (int)((unsigned)word >> 24);
            const int gx = (word << 20) >> 20, gy = (word << 8) >> 20;
            const int lx = gx - lx0, ly = gy - ly0;
            // the box touches the window's data (padded coordinates [KPAD, KPAD + W))
            const bool hit = lx + ex > KPAD && lx < KPAD + W && ly + ey > KPAD && ly < KPAD + W;
            if (fl & KF_FALLBACK) {
                fb = true;
            } else if (!(fl & KF_NOCORE) && hit &&
                       SYNIM_IDX_OK(lx >= 0 && ly >= 0 && (long)(ly + ey - 1) * Wp + lx + ex - 1 < ev.wn, err)) {
                act = true;
                wb = win + ly * Wp + lx;
            }
        }
        const bool two = __any_sync(0xffffffffu, act && (fl & KF_ASYM));
        float A[NC], B[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) A[q] = B[q] = 0.f;
        if (act) {
            if (ori == 0) {
                if (two) kf_dot_ba<0, true, NC>(BA, BC, wb, Wp, kwa + sid, kwb + sid, A, B);
                else kf_dot_ba<0, false, NC>(BA, BC, wb, Wp, kwa + sid, kwb + sid, A, B);
            } else {
                if (two) kf_dot_ba<1, true, NC>(BA, BC, wb, Wp, kwa + sid, kwb + sid, A, B);
                else kf_dot_ba<1, false, NC>(BA, BC, wb, Wp, kwa + sid, kwb + sid, A, B);
            }
            if (!(fl & KF_ASYM))   // kwb holds only the asymmetric segments' weights
#pragma unroll
                for (int q = 0; q < NC; ++q) B[q] = A[q];
        }
        // ring pixels of the pass's segments (Sec. 2.3 step 3) with their
        // stencil bits, spread over the lanes: the j-th one is repaired by lane
        // j % 32 into rbuf, then each segment's lane adds its own in order
        const int rm = (t < cnt && (fl & KF_RING)) ? __ldg(P.kring[ax] + sid) : 0;
        const int nr = __popc(rm);
        if (__any_sync(0xffffffffu, rm != 0)) {
        int pre = nr;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        const int total = __shfl_sync(0xffffffffu, pre, 31), excl = pre - nr;
        for (int j0 = 0; j0 < total; j0 += 32) {
            const int j = j0 + lane;
            int own = 0;   // the last lane whose first ring pixel is at or before j
#pragma unroll
            for (int st = 16; st > 0; st >>= 1)
                if (__shfl_sync(0xffffffffu, excl, own + st) <= j) own += st;
            const int orm = __shfl_sync(0xffffffffu, rm, own), oex = __shfl_sync(0xffffffffu, excl, own);
            float v[NC];
            bool ba = false, bb = false;
#pragma unroll
            for (int q = 0; q < NC; ++q) v[q] = 0.f;
            if (j < total) {
                int mm = orm;
                for (int q = j - oex; q > 0; --q) mm &= mm - 1;
                const int bit = __ffs(mm) - 1, q = bit >> 1, tt = bit & 1;
                const int to = base + own, r = fast_div(to, inv, ncol), c = to - r * ncol;
                const int sq = ax ? col0 + c : row0 + r, b = ax ? row0 + r : col0 + c;
                const int u0 = sq * WF.k, l0 = b * WF.k - 1;
                const int cb = __ldg((ax ? P.ycc : P.xcc) + b + (long)(u0 + q) * n1);
                ev.ring(ax ? l0 + tt : u0 + q, ax ? u0 + q : l0 + tt, v);
                ba = (cb & (tt ? 4 : 1)) != 0;
                bb = (cb & (tt ? 8 : 2)) != 0;
            }
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                rbuf[2 * NC * lane + q] = ba ? v[q] : 0.f;
                rbuf[2 * NC * lane + NC + q] = bb ? v[q] : 0.f;
            }
            __syncwarp();
            const int q1 = min(excl + nr, j0 + 32);
            for (int qq = max(excl, j0); qq < q1; ++qq)
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    A[q] += rbuf[2 * NC * (qq - j0) + q];
                    B[q] += rbuf[2 * NC * (qq - j0) + NC + q];
                }
            __syncwarp();
        }
        }
        if (t < cnt && !fb)
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                out[2 * NC * t + q] = A[q];
                out[2 * NC * t + NC + q] = B[q];
            }
        unsigned m = __ballot_sync(0xffffffffu, fb);
        while (m) {
            const int tt = base + __ffs(m) - 1;
            m &= m - 1;
            const int r = fast_div(tt, inv, ncol), c = tt - r * ncol;
            const SegRows sr = ax ? seg_rows(WF, s, 1, row0 + r, col0 + c) : seg_rows(WF, s, 0, col0 + c, row0 + r);
            float fa[NC], fbv[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) fa[q] = fbv[q] = 0.f;
            seg_compute<NC>(WF, sr, ev, ax, lane, 32, fa, fbv);
#pragma unroll
            for (int q = 0; q < NC; ++q)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    fa[q] += __shfl_xor_sync(0xffffffffu, fa[q], o);
                    fbv[q] += __shfl_xor_sync(0xffffffffu, fbv[q], o);
                }
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    out[2 * NC * tt + q] = fa[q];
                    out[2 * NC * tt + NC + q] = fbv[q];
                }
        }
    }
}

// One IM column from the weight boxes (forward: the IM; tangents: the IM and
// its four derivatives; adjoint: the cotangent dot products).  The same column
// as warp_column: zeros outside the rows of the subaperture box; then, in
// chunks of R box rows, every x segment of the chunk's rows and every y
// segment of the boundaries below them (the boundary above carried), the
// pupil-edge sums of the chunk's box subapertures, and one in-order pass over
// the chunk's valid rows (slopes in the box, zeros elsewhere).  Buffer
// (floats, NC components per value): X [R][nsj + 1][2][NC], Y [R + 1][nsj][2][NC],
// E [R][nsj][2][NC], then 64 NC for the ring pixels.
template <int MODE>
__device__ __forceinline__ void warp_column_kf(const Geo &g, const DevPair *__restrict__ pairs, int d, int a,
                                               int w, float *wbuf, int cap, int lane, int *err, double *gp,
                                               long unit) {
    constexpr int NC = (MODE == MODE_FWD) ? 1 : 5;
    constexpr int NOUT = (MODE == MODE_FWD) ? 1 : (MODE == MODE_TAN ? 5 : 0);
    constexpr int S = 2 * NC;   // floats per segment or subaperture sum
    const DevPair &P = pairs[d * g.n_wfs + w];
    const DevWFS &WF = g.wfs[w];
    const DevDM &D = g.dm[d];
    __shared__ ItemWfs s_item[8];
    ItemWfs &s = s_item[threadIdx.x >> 5];
    __syncwarp();
    make_info<MODE, NC>(g, pairs, d, a, w, s, err, KPAD);
    __syncwarp();
    const int nv = WF.nv, n2 = 2 * nv;
    const int nsj = s.empty ? 0 : s.nsj;
    // at least one box row: X, two Y rows and E, and the ring buffer
    if (!s.empty && S * (4 * nsj + 1) + 64 * NC > cap) {
        if (lane == 0) atomicOr(err, ERR_ARENA);
        s.empty = 1;
    }
    if (!s.empty && !SYNIM_IDX_OK(s.si0 >= 0 && s.si1 < WF.n_sub && s.sj0 >= 0 && s.sj1 < WF.n_sub, err)) return;
    const int vr0 = s.empty ? 0 : WF.vrow[s.si0], vr1 = s.empty ? 0 : WF.vrow[s.si1 + 1];
    if (!SYNIM_IDX_OK(0 <= vr0 && vr0 <= vr1 && vr1 <= nv, err)) return;
    float *cols[NOUT > 0 ? NOUT : 1];
    if constexpr (MODE != MODE_VJP) {
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            float *base = (o == 0) ? P.im : P.dim[o - 1];
            cols[o] = base ? base + (size_t)a * n2 : nullptr;
            if (!cols[o]) continue;
            if (P.vec4) {
                bulk_zero(cols[o], 0, vr0, lane);
                bulk_zero(cols[o], vr1, nv + vr0, lane);
                bulk_zero(cols[o], nv + vr1, n2, lane);
            } else {
                zero_rows(cols[o], 0, vr0, false, lane);
                zero_rows(cols[o], vr1, nv + vr0, false, lane);
                zero_rows(cols[o], nv + vr1, n2, false, lane);
            }
        }
    }
    float gacc[4] = {0.f, 0.f, 0.f, 0.f};
    const float *G = (MODE == MODE_VJP) ? P.gim + (size_t)a * n2 : nullptr;
    if (!s.empty) {
    const float *win = D.winK + (size_t)a * D.strideK;
    const int wx0 = D.org[2 * a], wy0 = D.org[2 * a + 1];
    Eval<NC> ev;
    ev.load(s, win, D.WpK, D.W, WF.M, KPAD);
#ifdef SYNIM_DEBUG_BOUNDS
    ev.err = err;
    ev.wn = D.strideK;
#endif
    const int nrows = s.si1 - s.si0 + 1;
    // chunk rows: X, Y and E of R rows plus the carried Y row
    const int R = max(1, min(nrows, ((cap - 64 * NC) / S - nsj) / (3 * nsj + 1)));
    float *rbuf = wbuf + cap - 64 * NC;
    float *X = wbuf;
    float *Y = X + (size_t)R * (nsj + 1) * S;
    float *E = Y + (size_t)(R + 1) * nsj * S;
    for (int r0 = s.si0; r0 <= s.si1; r0 += R) {
        const int Rc = min(R, s.si1 - r0 + 1), nb = Rc * nsj;
        kf_pass<NC>(WF, P, s, ev, win, D.WpK, D.W, wx0, wy0, 0, r0, nsj + 1, s.sj0, Rc * (nsj + 1), X, rbuf, lane,
                    err);
        // the y boundaries below the chunk's rows; the first chunk also takes
        // the one above the box (later chunks carry it)
        if (r0 == s.si0)
            kf_pass<NC>(WF, P, s, ev, win, D.WpK, D.W, wx0, wy0, 1, r0, nsj, s.sj0, nb + nsj, Y, rbuf, lane, err);
        else
            kf_pass<NC>(WF, P, s, ev, win, D.WpK, D.W, wx0, wy0, 1, r0 + 1, nsj, s.sj0, nb, Y + (size_t)nsj * S, rbuf,
                        lane, err);
        // pupil-edge sums of the chunk's box subapertures that have edge
        // pixels: four at a time, eight lanes each (both axes from one
        // resample per pixel, fixed butterfly order within the group)
        const float inv_nsj = 1.f / (float)nsj;
        for (int t0 = 0; t0 < nb; t0 += 32) {
            const int t = t0 + lane;
            bool has = false;
            if (t < nb) {
                const int q = fast_div(t, inv_nsj, nsj), c = t - q * nsj;
                const int qq = (r0 + q) * WF.n_sub + s.sj0 + c;
                has = WF.irr_sub[qq + 1] > WF.irr_sub[qq];
                if (!has)
#pragma unroll
                    for (int v = 0; v < S; ++v) E[(size_t)S * t + v] = 0.f;
            }
            unsigned m = __ballot_sync(0xffffffffu, has);
            const int grp = lane >> 3, gl = lane & 7;
            while (m) {
                // the group's subaperture: the grp-th lowest remaining one
                unsigned mm = m;
                for (int g2 = 0; g2 < grp && mm; ++g2) mm &= mm - 1;
                for (int g2 = 0; g2 < 4 && m; ++g2) m &= m - 1;
                const int tt = mm ? t0 + __ffs(mm) - 1 : -1;
                float ax_[NC], ay_[NC];
#pragma unroll
                for (int v = 0; v < NC; ++v) ax_[v] = ay_[v] = 0.f;
                if (tt >= 0) {
                    const int q = fast_div(tt, inv_nsj, nsj), c = tt - q * nsj;
                    edge_sum<NC>(WF, s, ev, r0 + q, s.sj0 + c, gl, 8, ax_, ay_);
                }
#pragma unroll
                for (int v = 0; v < NC; ++v)
#pragma unroll
                    for (int o = 4; o > 0; o >>= 1) {
                        ax_[v] += __shfl_xor_sync(0xffffffffu, ax_[v], o);
                        ay_[v] += __shfl_xor_sync(0xffffffffu, ay_[v], o);
                    }
                if (gl == 0 && tt >= 0)
#pragma unroll
                    for (int v = 0; v < NC; ++v) {
                        E[(size_t)S * tt + v] = ax_[v];
                        E[(size_t)S * tt + NC + v] = ay_[v];
                    }
            }
        }
        __syncwarp();
        // every valid row of the chunk's subaperture rows, in order: the
        // slope of a box subaperture (segment differences plus pupil-edge
        // sums, times slope_scale / (2 dw lit)), zero for the others; or the
        // adjoint's dot products of the tangents with the cotangent
        const int ra = WF.vrow[r0], rb = WF.vrow[r0 + Rc];
        if (!SYNIM_IDX_OK(0 <= ra && ra <= rb && rb <= nv, err)) return;
#pragma unroll 2
        for (int r = ra + lane; r < rb; r += 32) {
            const int vs = __ldg(WF.vsub + r);
            const int q = (vs >> 16) - r0, c = (vs & 0xffff) - s.sj0;
            float vx[NC], vy[NC];
#pragma unroll
            for (int v = 0; v < NC; ++v) vx[v] = vy[v] = 0.f;
            const bool inbox = c >= 0 && c < nsj;
            if (inbox) {
                const float f = __ldg(WF.fac + r);
                const float *segx = X + ((size_t)q * (nsj + 1) + c) * S;
                const float *sy0 = Y + ((size_t)q * nsj + c) * S, *sy1 = sy0 + (size_t)nsj * S;
                const float *eq = E + ((size_t)q * nsj + c) * S;
#pragma unroll
                for (int v = 0; v < NC; ++v) {
                    vx[v] = (segx[S + v] - segx[NC + v] + eq[v]) * f;
                    vy[v] = (sy1[v] - sy0[NC + v] + eq[NC + v]) * f;
                }
            }
            if constexpr (MODE == MODE_VJP) {
                if (inbox) {
                    const float gx = G[r], gy = G[nv + r];
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) gacc[k2] = fmaf(gx, vx[1 + k2], fmaf(gy, vy[1 + k2], gacc[k2]));
                }
            } else {
#pragma unroll
                for (int o = 0; o < NOUT; ++o)
                    if (cols[o]) {
                        cols[o][r] = vx[o];
                        cols[o][nv + r] = vy[o];
                    }
            }
        }
        __syncwarp();
        // carry the last boundary row of the chunk
        for (int c = lane; c < nsj * S; c += 32) Y[c] = Y[(size_t)Rc * nsj * S + c];
        __syncwarp();
    }
    }
    if constexpr (MODE == MODE_VJP) {
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            float vsum = gacc[k2];
            for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
            // this column's own slot: summed per pair in a fixed order by
            // k_vjp_reduce, so the result is reproducible
            if (lane == 0) gp[4 * unit + k2] = (double)vsum;
        }
    } else {
        (void)gp;
        (void)unit;
        (void)G;
    }
}

// One IM column (actuator a of DM d on sensor w) by one warp: zeros outside
// the rows of the subaperture box, and, box row by box row, the boundary
// segments, the slopes (segment differences plus pupil-edge pixels, times
// slope_scale / (2 dw lit)) and their stores; or the cotangent dot products.
template <int MODE, int NV>
__device__ __forceinline__ void warp_column(const Geo &g, const DevPair *__restrict__ pairs, int d, int a, int w,
                                            float *wbuf, int cap, int lane, int *err, double *gp, long unit) {
    const int pidx = d * g.n_wfs + w;
    const DevPair &P = pairs[pidx];
    if (!pair_active<MODE>(P)) return;
    if (P.kf) {   // a weight-box column: k_imk's
        if (lane == 0) atomicOr(err, ERR_ARENA);
        return;
    }
    const DevWFS &WF = g.wfs[w];
    const DevDM &D = g.dm[d];
    // The column's pixel and subaperture boxes live in shared memory, one
    // record per warp (every lane writes the same values), so that they take
    // no registers across the segment loops: at the forward kernel's
    // 64-register cap this removed its spills (1.226 -> 1.183 ms, MCAO).
    __shared__ ItemWfs s_item[8];
    ItemWfs &s = s_item[threadIdx.x >> 5];
    __syncwarp();   // every lane is done with the previous column's record
    make_info<MODE, NV>(g, pairs, d, a, w, s, err);
    __syncwarp();
    const int nv = WF.nv, n2 = 2 * nv;
    const int nsj = s.empty ? 0 : s.nsj;
    if (!s.empty && NV * 2 * (4 * nsj + 1) > cap) {
        if (lane == 0) atomicOr(err, ERR_ARENA);
        s.empty = 1;
    }
    const bool vec4 = P.vec4 != 0;
    if (!s.empty && !SYNIM_IDX_OK(s.si0 >= 0 && s.si1 < WF.n_sub && s.sj0 >= 0 && s.sj1 < WF.n_sub, err))
        return;
    const int vr0 = s.empty ? 0 : WF.vrow[s.si0], vr1 = s.empty ? 0 : WF.vrow[s.si1 + 1];
    if (!SYNIM_IDX_OK(0 <= vr0 && vr0 <= vr1 && vr1 <= nv, err)) return;
    constexpr int NOUT = (MODE == MODE_FWD) ? 1 : (MODE == MODE_TAN ? 5 : 0);
    float *cols[NOUT > 0 ? NOUT : 1];
    if (MODE != MODE_VJP) {
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            float *base = (o == 0) ? P.im : P.dim[o - 1];
            cols[o] = base ? base + (size_t)a * n2 : nullptr;
            if (!cols[o]) continue;
            if (vec4) {
                bulk_zero(cols[o], 0, vr0, lane);
                bulk_zero(cols[o], vr1, nv + vr0, lane);
                bulk_zero(cols[o], nv + vr1, n2, lane);
            } else {
                zero_rows(cols[o], 0, vr0, false, lane);
                zero_rows(cols[o], vr1, nv + vr0, false, lane);
                zero_rows(cols[o], nv + vr1, n2, false, lane);
            }
        }
    }
    if (s.empty) return;
    const float *G = (MODE == MODE_VJP) ? P.gim + (size_t)a * n2 : nullptr;
    float gacc[4] = {0.f, 0.f, 0.f, 0.f};
    Eval<NV> ev;
    ev.load(s, D.win + (size_t)a * D.win_stride, D.Wp, D.W, WF.M);
#ifdef SYNIM_DEBUG_BOUNDS
    ev.err = err;
    ev.wn = D.win_stride;
#endif
    float *segx = wbuf;                                // [nsj + 1][2][NV]
    float *sy0 = wbuf + (size_t)(nsj + 1) * 2 * NV;    // row boundary above the row: [nsj][2][NV]
    float *sy1 = sy0 + (size_t)nsj * 2 * NV;           // row boundary below it
    warp_segments<NV>(WF, s, ev, 1, s.si0, s.sj0, nsj, sy0, lane, g.seg_lanes);
    for (int si = s.si0; si <= s.si1; ++si) {
        warp_segments<NV>(WF, s, ev, 0, si, s.sj0, nsj + 1, segx, lane, g.seg_lanes);
        warp_segments<NV>(WF, s, ev, 1, si + 1, s.sj0, nsj, sy1, lane, g.seg_lanes);
        __syncwarp();
        // pupil-edge sums of the row's box subapertures that have edge pixels
        // (the whole warp on each, both axes from one resample per pixel)
        float *eb = wbuf + (size_t)(3 * nsj + 1) * 2 * NV;   // [nsj][2][NV], after both y rows
        for (int c0 = 0; c0 < nsj; c0 += 32) {
            // which of the next 32 box subapertures have edge pixels (one load each)
            const int cl = c0 + lane;
            bool has = false;
            if (cl < nsj) {
                const int q = si * WF.n_sub + s.sj0 + cl;
                has = WF.irr_sub[q + 1] > WF.irr_sub[q];
                if (!has)
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        eb[(size_t)cl * 2 * NV + v] = 0.f;
                        eb[(size_t)cl * 2 * NV + NV + v] = 0.f;
                    }
            }
            unsigned m = __ballot_sync(0xffffffffu, has);
            while (m) {
                const int c = c0 + __ffs(m) - 1;
                m &= m - 1;
                float ax[NV], ay[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) ax[v] = ay[v] = 0.f;
                if (WF.tl_n > 0) edge_sum_tiles<NV>(WF, s, ev, si, s.sj0 + c, lane, ax, ay);
                else edge_sum<NV>(WF, s, ev, si, s.sj0 + c, lane, 32, ax, ay);
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        ax[v] += __shfl_xor_sync(0xffffffffu, ax[v], o);
                        ay[v] += __shfl_xor_sync(0xffffffffu, ay[v], o);
                    }
                if (lane == 0)
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        eb[(size_t)c * 2 * NV + v] = ax[v];
                        eb[(size_t)c * 2 * NV + NV + v] = ay[v];
                    }
            }
        }
        __syncwarp();
        // slopes of the box subapertures (one lane each), zeros for the
        // row's other valid subapertures: rows [vrow[si], vrow[si + 1])
        int rlo = INT_MAX, rhi = -1;
        for (int c = lane; c < nsj; c += 32) {
            const int sj = s.sj0 + c;
            const int r = WF.vidx[si * WF.n_sub + sj];
            if (r < 0) continue;
            if (!SYNIM_IDX_OK(r < nv, err)) continue;
            rlo = min(rlo, r);
            rhi = max(rhi, r);
            float vx[NV], vy[NV];
            const float f = WF.fac[r];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                vx[v] = (segx[(size_t)(c + 1) * 2 * NV + v] - segx[(size_t)c * 2 * NV + NV + v] +
                         eb[(size_t)c * 2 * NV + v]) * f;
                vy[v] = (sy1[(size_t)c * 2 * NV + v] - sy0[(size_t)c * 2 * NV + NV + v] +
                         eb[(size_t)c * 2 * NV + NV + v]) * f;
            }
            if constexpr (MODE == MODE_VJP) {
                const float gx = G[r], gy = G[nv + r];
#pragma unroll
                for (int k2 = 0; k2 < 4; ++k2) gacc[k2] = fmaf(gx, vx[1 + k2], fmaf(gy, vy[1 + k2], gacc[k2]));
            } else {
#pragma unroll
                for (int o = 0; o < NOUT; ++o)
                    if (cols[o]) {
                        cols[o][r] = vx[o];
                        cols[o][nv + r] = vy[o];
                    }
            }
        }
        if constexpr (MODE != MODE_VJP) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                rlo = min(rlo, __shfl_xor_sync(0xffffffffu, rlo, o));
                rhi = max(rhi, __shfl_xor_sync(0xffffffffu, rhi, o));
            }
            const int ra = WF.vrow[si], rb = WF.vrow[si + 1];
            const int za = rhi < 0 ? rb : rlo, zb = rhi < 0 ? rb : rhi + 1;   // box rows: [za, zb)
#pragma unroll
            for (int o = 0; o < NOUT; ++o)
                if (cols[o]) {
                    zero_rows(cols[o], ra, za, false, lane);
                    zero_rows(cols[o], zb, rb, false, lane);
                    zero_rows(cols[o], nv + ra, nv + za, false, lane);
                    zero_rows(cols[o], nv + zb, nv + rb, false, lane);
                }
        }
        __syncwarp();
        float *t = sy0;
        sy0 = sy1;
        sy1 = t;
    }
    if (MODE == MODE_VJP) {
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            float vsum = gacc[k2];
            for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
            // this column's own slot (the caller zeroed it): summed per pair
            // in a fixed order by k_vjp_reduce, so the result is reproducible
            if (lane == 0) gp[4 * unit + k2] = (double)vsum;
        }
    }
}

// One warp per (actuator, sensor) column, the columns of one actuator in
// consecutive warps so that they share its window through L1.  Warps never
// wait for one another.  The long zero runs of a column are bulk copies of a
// shared zero buffer (TMA engine), which each issuing lane waits to have been
// read before the CTA exits.
template <int MODE>
__global__ void __launch_bounds__(256, (MODE == MODE_FWD) ? 4 : 2)
k_im(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs, int *__restrict__ err,
     double *__restrict__ gp) {
    constexpr int NV = (MODE == MODE_FWD) ? 1 : 5;
    extern __shared__ __align__(16) float smem_f[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float *wbuf = smem_f + (size_t)warp * g.seg_floats;
    if constexpr (MODE != MODE_VJP) {
        for (int q = threadIdx.x; q < kZeroFloats / 4; q += blockDim.x) s_zero[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic zeros -> bulk-copy reads
        __syncthreads();
    }
    const long n_units = (long)g.n_items * g.n_wfs;
    for (long u = (long)blockIdx.x * nw + warp; u < n_units; u += (long)gridDim.x * nw) {
        const int item = (int)(u / g.n_wfs), w = (int)(u - (long)item * g.n_wfs);
        int d, a;
        decode_item(g, item, d, a);
        if (MODE == MODE_VJP && lane < 4) gp[4 * u + lane] = 0.0;   // columns that return early add nothing
        warp_column<MODE, NV>(g, pairs, d, a, w, wbuf, g.seg_floats, lane, err, gp, u);
    }
    // the zero buffer must outlive the bulk copies that read it
    if (MODE != MODE_VJP && lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// The telescoping-sum engine (Sec. 2.2)
// ---------------------------------------------------------------------------
// Sums over one subaperture's events of sign * phi(edge point), this
// lane's share (events e0 + q, e0 + q + L, ..., four loads in flight):
// acc.x / acc.y the subaperture's own x / y sums, acc.z / acc.w the +phi
// credited to its left / upper neighbour by shared run ends.  The edge point's offset from the
// box origin (pi0, pj0) is exact in FP32 (half-integers below 2^13).
__device__ __forceinline__ void tele_events(const int *__restrict__ ev, int e0, int e1, const Eval<1> &E,
                                            int bi, int bj, int q, int L, float4 &acc) {
    constexpr int U = 4;   // events loaded ahead of their interpolation
    for (int e = e0 + q; e < e1; e += U * L) {
        int cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) cc[u] = (e + u * L < e1) ? __ldg(ev + e + u * L) : 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = cc[u];
            const float di = 0.5f * (float)(((c >> 16) & 0x7fff) - bi);
            const float dj = 0.5f * (float)((c & 0x3fff) - bj);
            const float x = fmaf(E.a00, dj, fmaf(E.a01, di, E.xo));
            const float y = fmaf(E.a10, dj, fmaf(E.a11, di, E.yo));
            const float phi = (e + u * L < e1) ? E.bil_at(x, y) : 0.f;
            const float v = (c < 0) ? phi : -phi;
            const float cr = (c & 0x4000) ? phi : 0.f;
            if (c & 0x8000) {
                acc.y += v;
                acc.w += cr;
            } else {
                acc.x += v;
                acc.z += cr;
            }
        }
    }
}

// One telescoping-sum IM column by one warp: zeros outside the valid rows
// of the subaperture box and in each box row's gaps (valid subapertures left
// or right of the box), then chunk by chunk of box rows: per box
// subaperture (groups of L lanes over the whole chunk, fixed butterfly
// order) the own sums and the credits to its left and upper neighbours, kept
// in shared memory with the previous chunk's last row; the x slopes (own +
// the right neighbour's credit) and the y slopes of the rows above (own +
// the lower neighbour's credit) times slope_scale / (dw lit).  A neighbour outside the box contributes nothing:
// its shared points lie beyond the pixel box, where the IF is zero.  Every
// phase value is one bilinear sample of the packed window; there is no
// pixel-class map and no edge repair.
__device__ __forceinline__ void tele_column(const Geo &g, const DevTele &T, const DevPair *__restrict__ pairs,
                                            int d, int a, int w, float4 *wbuf, int cap4, int lane, int *err) {
    const DevPair &P = pairs[d * g.n_wfs + w];
    if (!P.im) return;
    const DevWFS &WF = g.wfs[w];
    const DevDM &D = g.dm[d];
    ItemWfs s;
    make_info<MODE_FWD, 1>(g, pairs, d, a, w, s, nullptr);
    const int nv = WF.nv, n2 = 2 * nv;
    float *col = P.im + (size_t)a * n2;
    if (!s.empty && 2 * s.nsj > cap4) {   // the buffer holds at least two rows of n_sub: not reached
        if (lane == 0) atomicOr(err, ERR_ARENA);
        s.empty = 1;
    }
    if (!s.empty && !SYNIM_IDX_OK(s.si0 >= 0 && s.si1 < WF.n_sub && s.sj0 >= 0 && s.sj1 < WF.n_sub &&
                                  (long)(2 * s.nsj) <= cap4, err))
        return;
    const int vr0 = s.empty ? 0 : WF.vrow[s.si0], vr1 = s.empty ? 0 : WF.vrow[s.si1 + 1];
    if (!SYNIM_IDX_OK(0 <= vr0 && vr0 <= vr1 && vr1 <= nv, err)) return;
    if (P.vec4) {
        bulk_zero(col, 0, vr0, lane);
        bulk_zero(col, vr1, nv + vr0, lane);
        bulk_zero(col, nv + vr1, n2, lane);
    } else {
        zero_rows(col, 0, vr0, false, lane);
        zero_rows(col, vr1, nv + vr0, false, lane);
        zero_rows(col, nv + vr1, n2, false, lane);
    }
    if (s.empty) return;
    const int n1 = WF.n_sub + 1;
    for (int si = s.si0; si <= s.si1; ++si) {
        const int ra = WF.vrow[si], rb = WF.vrow[si + 1];
        const int za = T.vfirst[si * n1 + s.sj0], zb = T.vfirst[si * n1 + s.sj1 + 1];
        zero_rows(col, ra, za, false, lane);
        zero_rows(col, zb, rb, false, lane);
        zero_rows(col, nv + ra, nv + za, false, lane);
        zero_rows(col, nv + zb, nv + rb, false, lane);
    }
    Eval<1> E;
    E.load(s, D.win + (size_t)a * D.win_stride, D.Wp, D.W, WF.M);
#ifdef SYNIM_DEBUG_BOUNDS
    E.err = err;
    E.wn = D.win_stride;
#endif
    const int L = T.lanes, per = 32 / L, grp = lane / L, q = lane - grp * L;
    const int bi = 2 * s.pi0 + 1, bj = 2 * s.pj0 + 1;
    const int nsj = s.nsj, n = WF.n_sub;
    // chunks of R box rows: buffer row 0 carries the previous chunk's last row
    const int R = max(1, cap4 / nsj - 1);
    for (int sc = s.si0; sc <= s.si1; sc += R) {
        const int Rc = min(R, s.si1 - sc + 1), nb = Rc * nsj;
        const int *vchunk = WF.vidx + sc * n + s.sj0;
        for (int base = 0; base < nb; base += per) {
            const int t = base + grp;
            int r = -1;
            if (t < nb) {
                const int ri = t / nsj;
                r = vchunk[ri * n + (t - ri * nsj)];
            }
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r >= 0 && SYNIM_IDX_OK(r < nv && T.es[r] >= 0 && T.es[r + 1] <= T.n_ev, err))
                tele_events(T.ev, T.es[r], T.es[r + 1], E, bi, bj, q, L, acc);
            for (int o = L >> 1; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
                acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
            }
            if (q == 0 && t < nb && SYNIM_IDX_OK(nsj + t < cap4, err)) wbuf[nsj + t] = acc;
        }
        __syncwarp();
        // x slopes of the chunk's rows, y slopes of the rows above them
        for (int t = lane; t < nb; t += 32) {
            const int ri = t / nsj, c = t - ri * nsj;
            const float4 me = wbuf[nsj + t];
            const int r = vchunk[ri * n + c];
            if (r >= 0 && SYNIM_IDX_OK(r < nv, err))
                col[r] = (me.x + (c + 1 < nsj ? wbuf[nsj + t + 1].z : 0.f)) * T.fac[r];
            if (sc + ri > s.si0) {
                const int rp = vchunk[(ri - 1) * n + c];
                if (rp >= 0 && SYNIM_IDX_OK(rp < nv, err)) col[nv + rp] = (wbuf[t].y + me.w) * T.fac[rp];
            }
        }
        __syncwarp();
        for (int c = lane; c < nsj; c += 32) wbuf[c] = wbuf[nb + c];   // carry the last row
        __syncwarp();
    }
    // y slopes of the last box row (its lower neighbours lie outside the box)
    const int *vlast = WF.vidx + s.si1 * n + s.sj0;
    for (int c = lane; c < nsj; c += 32) {
        const int rp = vlast[c];
        if (rp >= 0 && SYNIM_IDX_OK(rp < nv, err)) col[nv + rp] = wbuf[c].y * T.fac[rp];
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256)
k_tele(const __grid_constant__ Geo g, const __grid_constant__ TeleSet t, const DevPair *__restrict__ pairs,
       int cap4, int *__restrict__ err) {
    extern __shared__ __align__(16) float4 tele_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = threadIdx.x; q < kZeroFloats / 4; q += blockDim.x) s_zero[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic zeros -> bulk-copy reads
    __syncthreads();
    float4 *wbuf = tele_smem + (size_t)warp * cap4;
    const long n_units = (long)g.n_items * g.n_wfs;
    for (long u = (long)blockIdx.x * nw + warp; u < n_units; u += (long)gridDim.x * nw) {
        const int item = (int)(u / g.n_wfs), w = (int)(u - (long)item * g.n_wfs);
        int d, a;
        decode_item(g, item, d, a);
        tele_column(g, t.w[w], pairs, d, a, w, wbuf, cap4, lane, err);
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Every IM column of a mode when some pair has boundary-segment weight boxes:
// one warp per column as in k_im, the weight boxes for those pairs (kf) and
// k_im's per-sample path for the others, all in one launch.  Within each DM
// the actuators' columns on the sensors with subapertures of at most 32
// pixels come first, then those on the others, so that a CTA's warps take
// one kind of column (and no warp idles behind a costlier neighbour).
template <int MODE>
__global__ void __launch_bounds__(256, (MODE == MODE_FWD) ? 3 : 2)
k_imk(const __grid_constant__ Geo g, const DevPair *__restrict__ pairs, int *__restrict__ err,
      double *__restrict__ gp) {
    constexpr int NV = (MODE == MODE_FWD) ? 1 : 5;
    extern __shared__ __align__(16) float smem_f[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float *wbuf = smem_f + (size_t)warp * g.seg_floats;
    if constexpr (MODE != MODE_VJP) {
        for (int q = threadIdx.x; q < kZeroFloats / 4; q += blockDim.x) s_zero[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic zeros -> bulk-copy reads
        __syncthreads();
    }
    const long n_units = (long)g.n_items * g.n_wfs;
    for (long u = (long)blockIdx.x * nw + warp; u < n_units; u += (long)gridDim.x * nw) {
        int pos = 0;
        while (pos + 1 < g.n_dm && u >= (long)g.order_start[pos + 1] * g.n_wfs) ++pos;
        const int n_act = g.order_start[pos + 1] - g.order_start[pos];
        const int na = g.n_wfs_a, nb = g.n_wfs - na;
        long r = u - (long)g.order_start[pos] * g.n_wfs;
        int a, w;
        if (r < (long)n_act * na) {
            a = (int)(r / na);
            w = g.wfs_order[r - (long)a * na];
        } else {
            r -= (long)n_act * na;
            a = (int)(r / nb);
            w = g.wfs_order[na + (r - (long)a * nb)];
        }
        const int d = g.order_dm[pos];
        // the adjoint's partials are indexed by the natural column order
        const long unit = (long)(g.order_start[pos] + a) * g.n_wfs + w;
        if (MODE == MODE_VJP && lane < 4) gp[4 * unit + lane] = 0.0;   // columns that return early add nothing
        const DevPair &P = pairs[d * g.n_wfs + w];
        if (!pair_active<MODE>(P)) continue;
        if (P.kf) warp_column_kf<MODE>(g, pairs, d, a, w, wbuf, g.seg_floats, lane, err, gp, unit);
        else warp_column<MODE, NV>(g, pairs, d, a, w, wbuf, g.seg_floats, lane, err, gp, unit);
    }
    if (MODE != MODE_VJP && lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

size_t tele_smem_bytes(int threads, int cap4) { return (size_t)(threads / 32) * cap4 * sizeof(float4); }

cudaError_t launch_tele(const Geo &g, const TeleSet &t, const DevPair *pairs, int cap4, int *err, int grid,
                        int threads, cudaStream_t s) {
    const size_t smem = tele_smem_bytes(threads, cap4);
    if (smem + sizeof(s_zero) > 48 * 1024) {   // static + dynamic above the default limit
        cudaError_t e = cudaFuncSetAttribute(k_tele, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_tele<<<grid, threads, smem, s>>>(g, t, pairs, cap4, err);
    return cudaGetLastError();
}

size_t im_smem_bytes(const Geo &g, int threads) { return (size_t)(threads / 32) * g.seg_floats * 4; }

template <int MODE>
static cudaError_t prepare_one(int threads, size_t smem, int *bps) {
    cudaError_t e = cudaFuncSetAttribute(k_im<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_imk<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_im<MODE>, threads, smem);
}

cudaError_t im_prepare(int mode, int threads, size_t smem, int *bps) {
    switch (mode) {
        case MODE_FWD: return prepare_one<MODE_FWD>(threads, smem, bps);
        case MODE_TAN: return prepare_one<MODE_TAN>(threads, smem, bps);
        default: return prepare_one<MODE_VJP>(threads, smem, bps);
    }
}

// Adjoint: grad_p[pair][k] = sum over the pair's actuators of the per-column
// partials of k_im<MODE_VJP>, one block per pair, each thread a fixed
// stride of actuators, then a fixed tree: the same order on every call.
__global__ void __launch_bounds__(256)
k_vjp_reduce(const __grid_constant__ Geo g, const double *__restrict__ part, double *__restrict__ gp) {
    const int p = blockIdx.x;
    const int d = p / g.n_wfs, w = p - d * g.n_wfs;
    int pos = 0;
    while (pos < g.n_dm && g.order_dm[pos] != d) ++pos;
    __shared__ double red[4][256];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (pos < g.n_dm) {
        const long first = g.order_start[pos], n = g.order_start[pos + 1] - first;
        for (long a = threadIdx.x; a < n; a += blockDim.x) {
            const double *q = part + 4 * ((first + a) * g.n_wfs + w);
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += q[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
#pragma unroll
            for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 4) gp[4 * p + threadIdx.x] = red[threadIdx.x][0];
}

cudaError_t launch_vjp_reduce(const Geo &g, const double *part, double *gp, cudaStream_t s) {
    k_vjp_reduce<<<g.n_dm * g.n_wfs, 256, 0, s>>>(g, part, gp);
    return cudaGetLastError();
}

cudaError_t launch_im(int mode, const Geo &g, const DevPair *pairs, int *err, double *gp, int grid, int threads,
                      size_t smem, cudaStream_t s, int kgrid) {
    switch (mode) {
        case MODE_FWD:
            if (kgrid > 0) k_imk<MODE_FWD><<<kgrid, threads, smem, s>>>(g, pairs, err, gp);
            else if (grid > 0) k_im<MODE_FWD><<<grid, threads, smem, s>>>(g, pairs, err, gp);
            break;
        case MODE_TAN:
            if (kgrid > 0) k_imk<MODE_TAN><<<kgrid, threads, smem, s>>>(g, pairs, err, gp);
            else if (grid > 0) k_im<MODE_TAN><<<grid, threads, smem, s>>>(g, pairs, err, gp);
            break;
        default:
            if (kgrid > 0) k_imk<MODE_VJP><<<kgrid, threads, smem, s>>>(g, pairs, err, gp);
            else if (grid > 0) k_im<MODE_VJP><<<grid, threads, smem, s>>>(g, pairs, err, gp);
            break;
    }
    return cudaGetLastError();
}

}  // namespace synim
