// synim_cnn.cu -- the learned misregistration estimator: a small BF16 CNN
// trained on the GPU on probe responses that the library itself generates.
//
// Network (input = slope maps of the attached probes, NHWC [H0][H0][C0]):
//   L1 conv 3x3 stride 1 pad 1, C0 -> 64, ReLU      [H1 = H0]
//   L2 conv 3x3 stride 2 pad 1, 64 -> 64, ReLU      [H2 = (H1 - 1) / 2 + 1]
//   L3 conv 3x3 stride 2 pad 1, 64 -> 64, ReLU      [H3 = (H2 - 1) / 2 + 1]
//   dense layer from the flattened H3 x H3 x 64 feature map to 4 outputs
// Output: the misregistration normalised to the training range,
// t = ((sx - c0) / r0, (sy - c1) / r1, (rot - c2) / r2, (mag - c3) / r3).
// Loss: mean over the batch and the 4 outputs of the squared error; Adam.
//
// Kernels (BF16 operands, FP32 accumulation):
//   k_conv_halo       stride-1 forward (first layer) on shifted windows of one
//                     halo per tile; + bias, ReLU, BF16; tcgen05.mma with
//                     TMEM accumulators;
//   k_conv_parity     stride-2 forwards (layers 2-3) on the four parity planes
//                     of the input, each input pixel staged once per tile;
//   k_conv_tc<DGRAD>  implicit GEMM of the transposed convolution: gradient
//                     of the layer input, masked by its ReLU, BF16;
//   k_wgrad_halo      weight and bias gradient of the first layer (32
//                     channels) on the shifted windows, tcgen05;
//   k_wgrad_tc        dW[co][k] = sum_m dz[m][co] im2col(in)[m][k] of the
//                     64-channel layers, tcgen05; both write one partial per
//                     CTA, summed in a fixed order;
//   small kernels for the head (dense layer, loss), bias sums, Adam.
// Parameters live as FP32 masters (flat vector, order W1 b1 W2 b2 W3 b3 Wfc
// bfc; W[co][ky][kx][ci], Wfc[j][y][x][c]) with BF16 copies for the GEMMs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "synim_internal.h"
#include "synim_cpasync.cuh"
#include "synim_tc.cuh"

namespace synim {

constexpr int CH = 64;               // hidden channels
constexpr int BM = 128;                // GEMM rows per tile
constexpr int kBatchCap = 256;       // samples per training / inference pass

typedef __nv_bfloat16 bf16;

struct CnnState {
    int H0 = 0, C0 = 0, H1 = 0, H2 = 0, H3 = 0;
    long long n_params = 0;
    long long off_w1 = 0, off_b1 = 0, off_w2 = 0, off_b2 = 0, off_w3 = 0, off_b3 = 0, off_fc = 0, off_bfc = 0;
    double center[4] = {0, 0, 0, 1}, range[4] = {1, 1, 1, 1};
    bool ready = false;
    int step = 0;
    float *master = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
    bf16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *w2t = nullptr, *w3t = nullptr;
    // activations / gradients for kBatchCap samples
    bf16 *x = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;
    bf16 *dz1 = nullptr, *dz2 = nullptr, *dz3 = nullptr;
    float *out = nullptr, *loss = nullptr, *dout = nullptr;
    float *hpart = nullptr;   // head partial sums [b][part][4], b * part <= kBatchCap * 32
    float *wpart = nullptr;   // weight-gradient partials [splits][64 K + 64]
    long long wpart_floats = 0;
    float *tgt = nullptr;   // [kBatchCap][4] targets of the current batch
    int *perm = nullptr;    // [n_data]
    bf16 *data = nullptr;   // training inputs [n_data][per_sample]
    float *targets = nullptr;  // [n_data][4]
    long long n_data = 0, data_cap = 0;
    float *h_loss = nullptr;   // pinned [kBatchCap]
    int *d_err = nullptr;      // bit 0: a bounded wait of the tensor-core convolution gave up
    CUtensorMap map_a1, map_a2;   // a1 / a2 as [kBatchCap][H][H][64] BF16, parity-plane boxes (k_conv_parity)
    CUtensorMap map_x, map_data;  // x [kBatchCap] and data [data_cap] inputs, halo boxes (k_conv_halo)
};

void cnn_destroy(CnnState *s) {
    if (!s) return;
    void *p[] = {s->master, s->adam_m, s->adam_v, s->grad, s->w1, s->w2, s->w3, s->w2t, s->w3t, s->x,
                 s->a1, s->a2, s->a3, s->dz1, s->dz2, s->dz3, s->out, s->loss, s->dout, s->hpart,
                 s->wpart, s->tgt, s->perm, s->data, s->targets, s->d_err};
    for (void *q : p) cudaFree(q);
    cudaFreeHost(s->h_loss);
    delete s;
}

__host__ __device__ __forceinline__ int conv_out(int h, int stride) { return (h - 1) / stride + 1; }

// ---------------------------------------------------------------------------
// Implicit-GEMM convolution (forward) and its transpose (input gradient)
// ---------------------------------------------------------------------------
struct ConvArgs {
    const bf16 *in;      // FWD: layer input [.][Hi][Hi][CIN]; DGRAD: dz of the layer output [B][Ho][Ho][64]
    const bf16 *w;       // FWD: W [64][9 CIN]; DGRAD: Wt [64 (ci)][9 x 64 (tap, co)]
    const float *bias;   // FWD
    const bf16 *act;     // DGRAD: layer input activation (ReLU mask) [B][Hi][Hi][64]
    bf16 *out;           // FWD: [B][Ho][Ho][64]; DGRAD: dz of the layer input [B][Hi][Hi][64]
    const int *perm;     // FWD of L1: input sample of batch row b is perm[b0 + b] (nullptr: b0 + b)
    long long b0;
    int B, Hi, Ho, stride;
};

// ---------------------------------------------------------------------------
// The convolution and its transpose on the 5th-generation tensor cores
// (tcgen05).
//
// One CTA walks 128-row tiles of the GEMM (rows = output pixels for the
// forward pass, input pixels for the input gradient) with three warp roles:
//   warps 0-3  gather, per 3x3 tap, each tile row's CIN channels (one pixel,
//              zero outside the image) into a shared-memory stage laid out as
//              K-major 8x16-byte core matrices; a stage holds one tap;
//   warp 8     one lane issues tcgen05.mma 128 x 64 x 16 per 16 channels of
//              the tap into a TMEM accumulator (two accumulators, so that the
//              epilogue of one tile overlaps the MMAs of the next);
//   warps 4-7  read the accumulator back (warp 4 + e owns TMEM lanes
//              32 e .. 32 e + 31), add the bias and apply the ReLU (forward)
//              or the ReLU mask of the layer input (input gradient), and
//              store BF16 rows.
// The weights (64 x 9 CIN, K-major) stay in shared memory for the whole
// kernel.  Stages are handed over through mbarriers: full (128 producer
// arrivals after their copies landed and were fenced for the async proxy),
// empty (tcgen05.commit of the MMAs that read the stage); accumulators
// through tfull (commit after a tile's last MMA) and tempty (128 epilogue
// arrivals).  Every wait is bounded; a wait that gives up sets bit 1 of *err
// and its role stops, so the kernel always ends.
// ---------------------------------------------------------------------------
constexpr int kTcThreads = 288;   // 4 producer warps, 4 epilogue warps, 1 MMA warp
// MMAs that accumulate into one TMEM accumulator serialise (a dependent
// chain costs ~173 cycles per tcgen05.mma on B300 whatever N is, against
// ~79 cycles per MMA for 4 interleaved chains), so a tile's MMAs go round
// robin into kTcParts partial accumulators that the epilogue adds.  Each
// tile needs at least kTcParts MMAs (it has 4 to 36).
constexpr int kTcParts = 4;
constexpr int kTcCols = 2 * kTcParts * CH;   // double-buffered: all 512 TMEM columns (one CTA per SM)

// Bias, ReLU, BF16 and the store of 32 channels (half h) of one output row.
__device__ __forceinline__ void store_relu32(const float (&v)[32], const float *__restrict__ bias, int h,
                                             bf16 *__restrict__ row) {
    uint4 o[4];
    uint32_t *ow = reinterpret_cast<uint32_t *>(o);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int n = 32 * h + 2 * u;
        __nv_bfloat162 r = __floats2bfloat162_rn(fmaxf(v[2 * u] + bias[n], 0.f), fmaxf(v[2 * u + 1] + bias[n + 1], 0.f));
        ow[u] = *reinterpret_cast<uint32_t *>(&r);
    }
    uint4 *out = reinterpret_cast<uint4 *>(row + 32 * h);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = o[q];
}

// v = sum over the kTcParts partial accumulators (64 columns apart, added in
// order) of 32 columns starting at taddr.
__device__ __forceinline__ void tc_ld_sum(uint32_t taddr, float (&v)[32]) {
    static_assert(kTcParts == 4, "one load per partial accumulator");
    uint32_t r[128];
    tc_ld32x4(taddr, CH, r);
#pragma unroll
    for (int q = 0; q < 32; ++q)
        v[q] = ((__uint_as_float(r[q]) + __uint_as_float(r[32 + q])) + __uint_as_float(r[64 + q])) +
               __uint_as_float(r[96 + q]);
}

template <int CIN>
struct TcCfg {
    static constexpr int K = 9 * CIN;
    static constexpr int KG = CIN / 8;             // core-matrix columns per tap
    static constexpr int A_BYTES = BM * CIN * 2;   // one tap of one 128-row tile
    static constexpr int B_BYTES = CH * K * 2;     // all weights
    static constexpr int STAGES = (CIN == 32) ? 6 : 8;
    static constexpr int LAG = STAGES - 2;         // taps in flight per producer thread
    static constexpr int N_BARS = 2 * STAGES + 4;
    static constexpr size_t SMEM = 128 + B_BYTES + (size_t)STAGES * A_BYTES + 8 * N_BARS + 16;
};

// Tiles of the GEMM.  Forward: one class, rows m = (b, y, x) of the output
// grid, all 9 taps.  Input gradient of a stride-2 convolution: the input
// pixels fall by parity (cy, cx) into four classes, rows (b, py, px) with
// (iy, ix) = (2 py + cy, 2 px + cx); only ky = 1 (cy = 0) or ky in {0, 2}
// (cy = 1), and likewise kx, reach a pixel of the class, from the output
// pixel oy = (iy + 1 - ky) / 2, ox = (ix + 1 - kx) / 2.  The classes hold
// 1, 2, 2 and 4 taps, instead of 9 with mostly zero rows.
struct TcTile {
    long long m0, M;   // first row of the tile within its class, rows of the class
    int cy, cx, ny, nx, ntap;
};

template <bool DGRAD>
__host__ __device__ __forceinline__ int tc_tile(const ConvArgs &a, int tile, TcTile *t) {
    if (!DGRAD) {
        const long long M = (long long)a.B * a.Ho * a.Ho;
        const int T = (int)((M + BM - 1) / BM);
        if (t && tile < T) *t = TcTile{(long long)tile * BM, M, 0, 0, a.Ho, a.Ho, 9};
        return T;
    }
    int first = 0;
    for (int c = 0; c < 4; ++c) {
        const int cy = c >> 1, cx = c & 1;
        const int ny = (a.Hi - cy + 1) >> 1, nx = (a.Hi - cx + 1) >> 1;
        const long long M = (long long)a.B * ny * nx;
        const int T = (int)((M + BM - 1) / BM);
        if (t && tile >= first && tile < first + T)
            *t = TcTile{(long long)(tile - first) * BM, M, cy, cx, ny, nx, (cy + 1) * (cx + 1)};
        first += T;
    }
    return first;   // the number of tiles
}

// Row m of a tile's class -> pixel (b, y, x) of the GEMM-row grid (output
// grid forward, input grid for the input gradient).
template <bool DGRAD>
__device__ __forceinline__ void tc_row(const TcTile &t, long long m, int &b, int &y, int &x) {
    const long long per = (long long)t.ny * t.nx;
    b = (int)(m / per);
    const int r = (int)(m - (long long)b * per);
    const int py = r / t.nx, px = r - py * t.nx;
    y = DGRAD ? 2 * py + t.cy : py;
    x = DGRAD ? 2 * px + t.cx : px;
}

// Tap q of a tile -> (ky, kx).
template <bool DGRAD>
__device__ __forceinline__ void tc_tap(const TcTile &t, int q, int &ky, int &kx) {
    if (DGRAD) {
        const int nkx = t.cx + 1;
        ky = t.cy ? 2 * (q / nkx) : 1;
        kx = t.cx ? 2 * (q % nkx) : 1;
    } else {
        ky = q / 3;
        kx = q - ky * 3;
    }
}

template <bool DGRAD, int CIN>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const ConvArgs a, int *__restrict__ err) {
    using C = TcCfg<CIN>;
    constexpr int S = C::STAGES;
    extern __shared__ __align__(128) unsigned char tc_raw[];
    unsigned char *base = tc_raw + ((128u - (tc_smem(tc_raw) & 127u)) & 127u);
    unsigned char *Bs = base;
    unsigned char *As = base + C::B_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(As + (size_t)S * C::A_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + C::N_BARS);
    const uint32_t bar0 = tc_smem(bars);
    // full[st] = bar0 + 8 st, empty[st] = bar0 + 8 (S + st),
    // tfull[j] = bar0 + 8 (2 S + j), tempty[j] = bar0 + 8 (2 S + 2 + j)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = tc_tile<DGRAD>(a, 0, nullptr);
    __shared__ float s_bias[CH];
    if (!DGRAD && tid < CH) s_bias[tid] = a.bias[tid];

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc_mbar_init(bar0 + 8 * i, 128);
            tc_mbar_init(bar0 + 8 * (S + i), 1);
        }
        for (int j = 0; j < 2; ++j) {
            tc_mbar_init(bar0 + 8 * (2 * S + j), 1);
            tc_mbar_init(bar0 + 8 * (2 * S + 2 + j), 128);
        }
        tc_fence_mbar_init();
    }
    if (warp == 8) tc_alloc(tc_smem(tslot), kTcCols);
    // weights: row n, 16-byte column kg -> core matrix (n / 8, kg), row n % 8
    for (int q = tid; q < CH * C::K / 8; q += kTcThreads) {
        const int n = q / (C::K / 8), kg = q - n * (C::K / 8);
        cp_async16_ca(Bs + ((size_t)(n >> 3) * (C::K / 8) + kg) * 128 + (n & 7) * 16, a.w + (size_t)n * C::K + kg * 8,
                      true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    tc_fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp < 4) {
        // ---- producers: thread tid gathers row tid of every tile
        int g = 0;
        bool run = true;
        for (int tile = blockIdx.x; tile < n_tiles && run; tile += gridDim.x) {
            TcTile t;
            tc_tile<DGRAD>(a, tile, &t);
            const long long m = t.m0 + tid;
            const bool row_ok = m < t.M;
            int rb = 0, ry = 0, rx = 0;
            if (row_ok) tc_row<DGRAD>(t, m, rb, ry, rx);
            const bf16 *img;
            if (DGRAD) {
                img = a.in + (size_t)rb * a.Ho * a.Ho * CH;
            } else {
                const long long sb = a.perm ? (long long)a.perm[a.b0 + rb] : a.b0 + rb;
                img = a.in + (size_t)sb * a.Hi * a.Hi * CIN;
            }
            unsigned char *dst0 = As + (size_t)(tid >> 3) * (C::KG * 128) + (tid & 7) * 16;
            for (int q = 0; q < t.ntap; ++q) {
                const int st = g % S;
                if (!tc_mbar_wait(bar0 + 8 * (S + st), ((g / S) & 1) ^ 1)) {
                    atomicOr(err, 1);
                    run = false;
                    break;
                }
                int ky, kx;
                tc_tap<DGRAD>(t, q, ky, kx);
                bool ok = row_ok;
                const bf16 *src = a.in;
                if (DGRAD) {
                    const int oy = (ry + 1 - ky) >> 1, ox = (rx + 1 - kx) >> 1;
                    ok = ok && oy < a.Ho && ox < a.Ho;
                    if (ok) src = img + ((size_t)oy * a.Ho + ox) * CH;
                } else {
                    const int iy = ry * a.stride + ky - 1, ix = rx * a.stride + kx - 1;
                    ok = ok && iy >= 0 && ix >= 0 && iy < a.Hi && ix < a.Hi;
                    if (ok) src = img + ((size_t)iy * a.Hi + ix) * CIN;
                }
                unsigned char *dst = dst0 + (size_t)st * C::A_BYTES;
#pragma unroll
                for (int c = 0; c < C::KG; ++c) cp_async16_ca(dst + c * 128, ok ? src + c * 8 : a.in, ok);
                cp_async_commit();
                if (g >= C::LAG) {
                    cp_async_wait<C::LAG>();
                    tc_fence_proxy_async();
                    tc_mbar_arrive(bar0 + 8 * ((g - C::LAG) % S));
                }
                ++g;
            }
        }
        cp_async_wait<0>();
        tc_fence_proxy_async();
        for (int q = (g > C::LAG ? g - C::LAG : 0); q < g; ++q) tc_mbar_arrive(bar0 + 8 * (q % S));
    } else if (warp == 8) {
        // ---- MMA issue: one lane
        if (lane == 0) {
            const uint32_t idesc = tc_idesc_bf16(BM, CH);
            const uint32_t a_base = tc_smem(As), b_base = tc_smem(Bs);
            int g = 0, i = 0;
            bool run = true;
            for (int tile = blockIdx.x; tile < n_tiles && run; tile += gridDim.x, ++i) {
                TcTile t;
                tc_tile<DGRAD>(a, tile, &t);
                const int ab = i & 1;
                if (!tc_mbar_wait(bar0 + 8 * (2 * S + 2 + ab), ((i >> 1) & 1) ^ 1)) {
                    atomicOr(err, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * kTcParts * CH);
                int n_mma = 0;
                for (int q = 0; q < t.ntap; ++q, ++g) {
                    const int st = g % S;
                    if (!tc_mbar_wait(bar0 + 8 * st, (g / S) & 1)) {
                        atomicOr(err, 1);
                        run = false;
                        break;
                    }
                    tc_fence_after();
                    int ky, kx;
                    tc_tap<DGRAD>(t, q, ky, kx);
                    const uint32_t as = a_base + (uint32_t)(st * C::A_BYTES);
                    const uint32_t bs = b_base + (uint32_t)((ky * 3 + kx) * C::KG * 128);
#pragma unroll
                    for (int j = 0; j < CIN / 16; ++j, ++n_mma)
                        tc_mma(d + (uint32_t)((n_mma % kTcParts) * CH), tc_desc(as + j * 256, 128, C::KG * 128),
                               tc_desc(bs + j * 256, 128, C::K * 16), idesc, n_mma >= kTcParts);
                    tc_commit(bar0 + 8 * (S + st));
                }
                if (run) tc_commit(bar0 + 8 * (2 * S + ab));
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp 4 + e reads TMEM lanes 32 e .. 32 e + 31 = tile rows
        const int e = warp - 4;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * e) << 16);
        int i = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
            TcTile t;
            tc_tile<DGRAD>(a, tile, &t);
            const int ab = i & 1;
            if (!tc_mbar_wait(bar0 + 8 * (2 * S + ab), (i >> 1) & 1)) {
                atomicOr(err, 1);
                break;
            }
            tc_fence_after();
            const long long m = t.m0 + 32 * e + lane;
            long long orow = 0;   // output row (pixel) of GEMM row m
            if (m < t.M) {
                int b, y, x;
                tc_row<DGRAD>(t, m, b, y, x);
                orow = DGRAD ? ((long long)b * a.Hi + y) * a.Hi + x : m;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[32];
                tc_ld_sum(lane_base + (uint32_t)(ab * kTcParts * CH + 32 * h), v);
                if (m < t.M) {
                    if (DGRAD) {
                        uint4 o[4];
                        uint32_t *ow = reinterpret_cast<uint32_t *>(o);
                        const uint4 *act = reinterpret_cast<const uint4 *>(a.act + orow * CH + 32 * h);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint4 av = act[q];
                            const uint32_t aw[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                __nv_bfloat162 am = *reinterpret_cast<const __nv_bfloat162 *>(&aw[u]);
                                const float v0 = (__bfloat162float(am.x) > 0.f) ? v[8 * q + 2 * u] : 0.f;
                                const float v1 = (__bfloat162float(am.y) > 0.f) ? v[8 * q + 2 * u + 1] : 0.f;
                                __nv_bfloat162 r = __floats2bfloat162_rn(v0, v1);
                                ow[4 * q + u] = *reinterpret_cast<uint32_t *>(&r);
                            }
                        }
                        uint4 *out = reinterpret_cast<uint4 *>(a.out + orow * CH + 32 * h);
#pragma unroll
                        for (int q = 0; q < 4; ++q) out[q] = o[q];
                    } else {
                        store_relu32(v, s_bias, h, a.out + orow * CH);
                    }
                }
            }
            tc_fence_before();
            tc_mbar_arrive(bar0 + 8 * (2 * S + 2 + ab));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        tc_dealloc(tmem, kTcCols);
    }
}

// ---------------------------------------------------------------------------
// Shifted-window kernels for the stride-1 layer (first convolution).
//
// GEMM rows are the pixels of a padded-pitch grid, r = y Wp + x with
// Wp = H + 2 (x >= H: padding rows, computed and dropped), in tiles of 128
// rows within one image.  Input pixel (y + ky - 1, x + kx - 1) of row r sits
// at padded position r + ky Wp + kx, so one halo of NS = 128 + 2 Wp + 2
// padded positions per tile serves all nine taps: tap (ky, kx) is the halo
// read from offset ky Wp + kx.  The halo is stored as CIN / 8 planes of
// 16-byte pixels (8 channels each), so that 8 consecutive rows of one plane
// are one 8 x 16-byte core matrix: K-major for the forward GEMM (rows =
// pixels, K = channels; the next 8 channels are the next plane) and
// MN-major for the weight gradient (K = pixels, N = channels).
// ---------------------------------------------------------------------------
struct HaloGeo {
    int H, Wp, NS, plane, per_img;   // side, pitch, halo positions, plane bytes, tiles per image
};

__host__ __device__ __forceinline__ HaloGeo halo_geo(int H) {
    HaloGeo g;
    g.H = H;
    g.Wp = H + 2;
    g.NS = (BM + 2 * g.Wp + 2 + 7) / 8 * 8;
    g.plane = g.NS * 16;
    g.per_img = (H * g.Wp + BM - 1) / BM;
    return g;
}

// Halo of one tile (image img, first row r0) into the CIN / 8 planes at dst,
// by the 128 producer threads; zero outside the image.
template <int CIN>
__device__ __forceinline__ void load_halo(unsigned char *dst, const bf16 *img, const HaloGeo &g, int r0, int tid,
                                          const bf16 *any) {
    constexpr int KG = CIN / 8;
    // a thread per halo position; 8 consecutive threads fill 128 contiguous
    // bytes of one plane (no bank conflicts)
    for (int sp = tid; sp < g.NS; sp += 128) {
        const int P = r0 + sp, py = P / g.Wp, px = P - py * g.Wp;
        const int iy = py - 1, ix = px - 1;
        const bool ok = iy >= 0 && iy < g.H && ix >= 0 && ix < g.H;
        const bf16 *src = ok ? img + ((size_t)iy * g.H + ix) * CIN : any;
#pragma unroll
        for (int kg = 0; kg < KG; ++kg) cp_async16_ca(dst + kg * g.plane + sp * 16, ok ? src + kg * 8 : any, ok);
    }
}

template <int CIN>
struct HaloCfg {
    static constexpr int K = 9 * CIN;
    static constexpr int KG = CIN / 8;
    static constexpr int B_BYTES = CH * K * 2;
    static constexpr int STAGES = (CIN == 32) ? 8 : 4;   // also keeps one CTA per SM
    static constexpr int N_BARS = 2 * STAGES + 4;
    __host__ __device__ static size_t smem(const HaloGeo &g) {
        return 128 + B_BYTES + (size_t)STAGES * KG * g.plane + 8 * N_BARS + 16;
    }
};

// One 4-D tensor-map tile load (TMA) into shared memory, completing on mbar.
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                          uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// The forward halo as tensor-map boxes: whole padded rows from row r0 / Wp,
// NR of them (rows r0 .. r0 + 127 read positions up to r0 + 127 + 2 Wp + 2),
// one box of 8 channels x Wp columns x NR rows per 8-channel group; a group's
// region is rounded up to 128 bytes.
struct HaloTma {
    int NR, plane;
};

__host__ __device__ __forceinline__ HaloTma halo_tma(const HaloGeo &g) {
    HaloTma t;
    t.NR = (BM + 2 * g.Wp + 2) / g.Wp + 2;
    t.plane = (t.NR * g.Wp * 16 + 127) / 128 * 128;
    return t;
}

template <int CIN>
struct HaloTmaCfg {
    static constexpr int K = 9 * CIN;
    static constexpr int KG = CIN / 8;
    static constexpr int B_BYTES = CH * K * 2;
    static constexpr int STAGES = (CIN == 32) ? 8 : 3;
    static constexpr int N_BARS = 2 * STAGES + 4;
    __host__ __device__ static size_t smem(const HaloTma &t) {
        return 128 + B_BYTES + (size_t)STAGES * KG * t.plane + 8 * N_BARS + 16;
    }
};

// Forward convolution, stride 1, pad 1: out = ReLU(conv(in) + bias), same
// warp roles, barriers and bounded waits as k_conv_tc; a stage holds one
// tile's halo and feeds 9 taps x CIN / 16 MMAs.
// The halo comes from the layer input's tensor map (4-D [samples][H][H][CIN]
// BF16, boxes as halo_tma): one producer thread issues the CIN / 8 box loads
// of a tile, starting at column -1 and row r0 / Wp - 1 of the image (zero
// fill outside it gives the padding).
template <int CIN>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_halo(const ConvArgs a, const __grid_constant__ CUtensorMap in_map,
                                                             int *__restrict__ err) {
    using C = HaloTmaCfg<CIN>;
    constexpr int S = C::STAGES;
    const HaloGeo hg = halo_geo(a.Ho);
    const HaloTma ht = halo_tma(hg);
    const int stage_bytes = C::KG * ht.plane;
    extern __shared__ __align__(128) unsigned char tc_raw[];
    unsigned char *base = tc_raw + ((128u - (tc_smem(tc_raw) & 127u)) & 127u);
    unsigned char *Bs = base;
    unsigned char *As = base + C::B_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(As + (size_t)S * stage_bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + C::N_BARS);
    const uint32_t bar0 = tc_smem(bars);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = a.B * hg.per_img;
    __shared__ float s_bias[CH];

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc_mbar_init(bar0 + 8 * i, 1);
            tc_mbar_init(bar0 + 8 * (S + i), 1);
        }
        for (int j = 0; j < 2; ++j) {
            tc_mbar_init(bar0 + 8 * (2 * S + j), 1);
            tc_mbar_init(bar0 + 8 * (2 * S + 2 + j), 128);
        }
        tc_fence_mbar_init();
    }
    if (tid < CH) s_bias[tid] = a.bias[tid];
    if (warp == 8) tc_alloc(tc_smem(tslot), kTcCols);
    for (int q = tid; q < CH * C::K / 8; q += kTcThreads) {
        const int n = q / (C::K / 8), kg = q - n * (C::K / 8);
        cp_async16_ca(Bs + ((size_t)(n >> 3) * (C::K / 8) + kg) * 128 + (n & 7) * 16, a.w + (size_t)n * C::K + kg * 8,
                      true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    tc_fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t box_bytes = (uint32_t)(ht.NR * hg.Wp * 16);
            int g = 0;
            for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++g) {
                const int b = tile / hg.per_img, r0 = (tile - b * hg.per_img) * BM;
                const int sb = a.perm ? a.perm[a.b0 + b] : (int)(a.b0 + b);
                const int st = g % S;
                if (!tc_mbar_wait(bar0 + 8 * (S + st), ((g / S) & 1) ^ 1)) {
                    atomicOr(err, 1);
                    break;
                }
                const uint32_t full = bar0 + 8 * st;
                mbar_expect_tx(full, C::KG * box_bytes);
                const uint32_t dst = tc_smem(As + (size_t)st * stage_bytes);
#pragma unroll
                for (int gg = 0; gg < C::KG; ++gg)
                    tma_load4(dst + (uint32_t)(gg * ht.plane), &in_map, gg * 8, -1, r0 / hg.Wp - 1, sb, full);
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // the other producer warps have nothing to stage
    } else if (warp == 8) {
        if (lane == 0) {
            const uint32_t idesc = tc_idesc_bf16(BM, CH);
            const uint32_t a_base = tc_smem(As), b_base = tc_smem(Bs);
            int g = 0;
            for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++g) {
                const int ab = g & 1;
                if (!tc_mbar_wait(bar0 + 8 * (2 * S + 2 + ab), ((g >> 1) & 1) ^ 1)) {
                    atomicOr(err, 1);
                    break;
                }
                const int st = g % S;
                if (!tc_mbar_wait(bar0 + 8 * st, (g / S) & 1)) {
                    atomicOr(err, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * kTcParts * CH);
                const uint32_t as = a_base + (uint32_t)(st * stage_bytes);
                const int r0 = (tile - (tile / hg.per_img) * hg.per_img) * BM;
                const int rel = r0 - (r0 / hg.Wp) * hg.Wp;   // the tile's first row within the loaded rows
                int n_mma = 0;
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - ky * 3;
                    const uint32_t at = as + (uint32_t)((rel + ky * hg.Wp + kx) * 16);
                    const uint32_t bt = b_base + (uint32_t)(tap * C::KG * 128);
#pragma unroll
                    for (int j = 0; j < CIN / 16; ++j, ++n_mma)
                        tc_mma(d + (uint32_t)((n_mma % kTcParts) * CH), tc_desc(at + 2 * j * ht.plane, ht.plane, 128),
                               tc_desc(bt + j * 256, 128, C::K * 16), idesc, n_mma >= kTcParts);
                }
                tc_commit(bar0 + 8 * (S + st));
                tc_commit(bar0 + 8 * (2 * S + ab));
            }
        }
        __syncwarp();
    } else {
        const int e = warp - 4;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * e) << 16);
        int g = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++g) {
            const int ab = g & 1;
            if (!tc_mbar_wait(bar0 + 8 * (2 * S + ab), (g >> 1) & 1)) {
                atomicOr(err, 1);
                break;
            }
            tc_fence_after();
            const int b = tile / hg.per_img;
            const int r = (tile - b * hg.per_img) * BM + 32 * e + lane;
            const int y = r / hg.Wp, x = r - y * hg.Wp;
            const bool keep = y < hg.H && x < hg.H;
            bf16 *row = a.out + (((size_t)b * hg.H + y) * hg.H + x) * CH;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[32];
                tc_ld_sum(lane_base + (uint32_t)(ab * kTcParts * CH + 32 * h), v);
                if (keep) store_relu32(v, s_bias, h, row);
            }
            tc_fence_before();
            tc_mbar_arrive(bar0 + 8 * (2 * S + 2 + ab));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        tc_dealloc(tmem, kTcCols);
    }
}

// ---------------------------------------------------------------------------
// Parity-plane kernel for the stride-2 forward convolutions (64 channels).
//
// Input pixel (2 oy - 1 + ky, 2 ox - 1 + kx) of output (oy, ox) lies in the
// parity plane (py, px) = (ky != 1, kx != 1) of the input, P_pq(Y, X) =
// in(2 Y + p, 2 X + q), at (Y, X) = (oy - (ky == 0), ox - (kx == 0)).  With
// GEMM rows r = oy Wq + ox on a padded pitch Wq = Ho + 1 (x = Ho: padding
// rows, computed and dropped) and each plane stored at padded positions
// R = (Y + 1) Wq + (X + 1) (zero outside the input), tap (ky, kx) of row r is
// plane (py, px) at R = r + (ky != 0) Wq + (kx != 0): one halo of
// NS2 = 128 + Wq + 2 positions per plane and tile serves all nine taps, and
// every input pixel is staged once per tile instead of once per tap.  A
// stage holds the four planes of one tile for half of the 64 input channels
// (4 planes x 4 eight-channel groups of 16-byte pixels), so that three
// stages and the resident weights fit one SM; a tile is two stages, 18 MMAs
// each.
// ---------------------------------------------------------------------------
struct ParGeo {
    int Hi, Ho, Wq, NR, plane, per_img;   // NR: plane rows per tile; plane: bytes of one 8-channel group
};

__host__ __device__ __forceinline__ ParGeo par_geo(int Hi, int Ho) {
    ParGeo g;
    g.Hi = Hi;
    g.Ho = Ho;
    g.Wq = Ho + 1;
    // a tile's rows r0 .. r0 + 127 read positions up to r0 + 128 + Wq, from plane row r0 / Wq on
    g.NR = (BM + g.Wq) / g.Wq + 2;
    g.plane = (g.NR * g.Wq * 16 + 127) / 128 * 128;
    g.per_img = (Ho * g.Wq + BM - 1) / BM;
    return g;
}

struct ParCfg {
    static constexpr int K = 9 * CH;
    static constexpr int B_BYTES = CH * K * 2;
    static constexpr int STAGES = 3;              // (tile, channel half) units in flight
    static constexpr int N_BARS = 2 * STAGES + 4;
    __host__ __device__ static size_t stage_bytes(const ParGeo &g) { return (size_t)16 * g.plane; }
    __host__ __device__ static size_t smem(const ParGeo &g) {
        return 128 + B_BYTES + (size_t)STAGES * stage_bytes(g) + 8 * N_BARS + 16;
    }
};


// Forward convolution, stride 2, pad 1, 64 -> 64 channels: out = ReLU(conv +
// bias); warp roles, barriers and bounded waits as k_conv_halo, with the
// stages counted in (tile, channel half) units.  One producer thread fills a
// stage with 16 tensor-map loads (4 planes x 4 eight-channel groups): the
// map's element strides of 2 along x and y pick one parity plane, its box
// covers NR plane rows x Wq columns from plane position (r0 / Wq) Wq, and
// coordinates outside the input (the zero padding) are filled with zeros.
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_parity(const ConvArgs a,
                                                               const __grid_constant__ CUtensorMap in_map,
                                                               int *__restrict__ err) {
    using C = ParCfg;
    constexpr int S = C::STAGES;
    const ParGeo pg = par_geo(a.Hi, a.Ho);
    const int stage_bytes = (int)C::stage_bytes(pg);
    extern __shared__ __align__(128) unsigned char tc_raw[];
    unsigned char *base = tc_raw + ((128u - (tc_smem(tc_raw) & 127u)) & 127u);
    unsigned char *Bs = base;
    unsigned char *As = base + C::B_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(As + (size_t)S * stage_bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + C::N_BARS);
    const uint32_t bar0 = tc_smem(bars);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = a.B * pg.per_img;
    __shared__ float s_bias[CH];

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc_mbar_init(bar0 + 8 * i, 1);
            tc_mbar_init(bar0 + 8 * (S + i), 1);
        }
        for (int j = 0; j < 2; ++j) {
            tc_mbar_init(bar0 + 8 * (2 * S + j), 1);
            tc_mbar_init(bar0 + 8 * (2 * S + 2 + j), 128);
        }
        tc_fence_mbar_init();
    }
    if (tid < CH) s_bias[tid] = a.bias[tid];
    if (warp == 8) tc_alloc(tc_smem(tslot), kTcCols);
    for (int q = tid; q < CH * C::K / 8; q += kTcThreads) {
        const int n = q / (C::K / 8), kg = q - n * (C::K / 8);
        cp_async16_ca(Bs + ((size_t)(n >> 3) * (C::K / 8) + kg) * 128 + (n & 7) * 16, a.w + (size_t)n * C::K + kg * 8,
                      true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    tc_fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t box_bytes = (uint32_t)(pg.NR * pg.Wq * 16);
            int u = 0;   // units issued: u = 2 g + h
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                const int b = tile / pg.per_img, r0 = (tile - b * pg.per_img) * BM;
                const int py0 = r0 / pg.Wq;
                for (int h = 0; h < 2; ++h, ++u) {
                    const int st = u % S;
                    if (!tc_mbar_wait(bar0 + 8 * (S + st), ((u / S) & 1) ^ 1)) {
                        atomicOr(err, 1);
                        ok = false;
                        break;
                    }
                    const uint32_t full = bar0 + 8 * st;
                    mbar_expect_tx(full, 16 * box_bytes);
                    const uint32_t dst = tc_smem(As + (size_t)st * stage_bytes);
#pragma unroll 1
                    for (int pq = 0; pq < 4; ++pq)
#pragma unroll
                        for (int gg = 0; gg < 4; ++gg)
                            tma_load4(dst + (uint32_t)((4 * pq + gg) * pg.plane), &in_map, h * 32 + gg * 8,
                                      (pq & 1) - 2, 2 * (py0 - 1) + (pq >> 1), (int)(a.b0 + b), full);
                }
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // the other producer warps have nothing to stage
    } else if (warp == 8) {
        if (lane == 0) {
            const uint32_t idesc = tc_idesc_bf16(BM, CH);
            const uint32_t a_base = tc_smem(As), b_base = tc_smem(Bs);
            int g = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++g) {
                const int ab = g & 1;
                if (!tc_mbar_wait(bar0 + 8 * (2 * S + 2 + ab), ((g >> 1) & 1) ^ 1)) {
                    atomicOr(err, 1);
                    break;
                }
                const uint32_t d = tmem + (uint32_t)(ab * kTcParts * CH);
                const int r0 = (tile - (tile / pg.per_img) * pg.per_img) * BM;
                const int rel = r0 - (r0 / pg.Wq) * pg.Wq;   // the tile's first row within the loaded box
                int n_mma = 0;
                for (int h = 0; h < 2; ++h) {
                    const int u = 2 * g + h, st = u % S;
                    if (!tc_mbar_wait(bar0 + 8 * st, (u / S) & 1)) {
                        atomicOr(err, 1);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t as = a_base + (uint32_t)(st * stage_bytes);
#pragma unroll 1
                    for (int tap = 0; tap < 9; ++tap) {
                        const int ky = tap / 3, kx = tap - ky * 3;
                        const int pq = 2 * (ky != 1) + (kx != 1);
                        const uint32_t at = as + (uint32_t)(4 * pq * pg.plane) +
                                            (uint32_t)((rel + (ky != 0) * pg.Wq + (kx != 0)) * 16);
                        const uint32_t bt = b_base + (uint32_t)((tap * 8 + 4 * h) * 128);
#pragma unroll
                        for (int j = 0; j < 2; ++j, ++n_mma)
                            tc_mma(d + (uint32_t)((n_mma % kTcParts) * CH),
                                   tc_desc(at + 2 * j * pg.plane, pg.plane, 128), tc_desc(bt + j * 256, 128, C::K * 16),
                                   idesc, n_mma >= kTcParts);
                    }
                    tc_commit(bar0 + 8 * (S + st));
                }
                if (!ok) break;
                tc_commit(bar0 + 8 * (2 * S + ab));
            }
        }
        __syncwarp();
    } else {
        const int e = warp - 4;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * e) << 16);
        int g = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++g) {
            const int ab = g & 1;
            if (!tc_mbar_wait(bar0 + 8 * (2 * S + ab), (g >> 1) & 1)) {
                atomicOr(err, 1);
                break;
            }
            tc_fence_after();
            const int b = tile / pg.per_img;
            const int r = (tile - b * pg.per_img) * BM + 32 * e + lane;
            const int y = r / pg.Wq, x = r - y * pg.Wq;
            const bool keep = y < pg.Ho && x < pg.Ho;
            bf16 *row = a.out + (((size_t)b * pg.Ho + y) * pg.Ho + x) * CH;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[32];
                tc_ld_sum(lane_base + (uint32_t)(ab * kTcParts * CH + 32 * h), v);
                if (keep) store_relu32(v, s_bias, h, row);
            }
            tc_fence_before();
            tc_mbar_arrive(bar0 + 8 * (2 * S + 2 + ab));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        tc_dealloc(tmem, kTcCols);
    }
}

// ---------------------------------------------------------------------------
// Weight gradients: arguments shared by the 64-channel kernel below.
// ---------------------------------------------------------------------------
struct WgArgs {
    const bf16 *dz;      // [B][Ho][Ho][64]
    const bf16 *in;      // layer input
    const int *perm;
    long long b0;
    int B, Hi, Ho, stride;
    float *part;         // [CTAs][64 x 9 CIN + 64]: weight, then bias partials
};

// ---------------------------------------------------------------------------
// Weight and bias gradient of the stride-1 layer with CIN = 32 channels, on
// the shifted windows: for each tile, the halo of the layer input and the
// tile's 128 rows of dz (zero on padding rows) are staged once; tap (ky, kx)
// contributes dz^T (64 x 128, MN-major) times the halo read from offset
// ky Wp + kx (128 x 32, MN-major) through tcgen05.mma M=64 N=32 K=16 into
// its own 32 TMEM columns, accumulated over all tiles of the CTA; a 10th
// product with an all-ones operand (N = 8) gives the bias gradient.  The
// epilogue writes part[cta][co][tap ci] and part[cta][64 K + co].  With
// M = 64, accumulator row i sits in TMEM lane 32 (i / 16) + i % 16.
// ---------------------------------------------------------------------------
struct HaloWgArgs {
    const bf16 *dz;      // [B][H][H][64]
    const bf16 *in;      // layer input [.][H][H][32]
    const int *perm;
    long long b0;
    int B, H;
    float *part;         // [gridDim.x][64 x 288 + 64]
};

constexpr int kHwStages = 6;
constexpr int kHwCols = 512;   // 9 x 32 + 8 columns, rounded up to a power of two

__host__ __device__ __forceinline__ size_t wgrad_halo_smem(const HaloGeo &g) {
    return 128 + 2048 + (size_t)kHwStages * (4 * g.plane + BM * CH * 2) + 8 * (2 * kHwStages + 1) + 16;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_wgrad_halo(const HaloWgArgs a, int *__restrict__ err) {
    constexpr int CIN = 32, K = 9 * CIN, KG = CIN / 8, S = kHwStages, LAG = S - 2;
    const HaloGeo hg = halo_geo(a.H);
    const int halo_bytes = KG * hg.plane, stage_bytes = halo_bytes + BM * CH * 2;
    extern __shared__ __align__(128) unsigned char tc_raw[];
    unsigned char *base = tc_raw + ((128u - (tc_smem(tc_raw) & 127u)) & 127u);
    unsigned char *ones = base;            // 128 rows x 8 BF16 ones
    unsigned char *St = base + 2048;       // stages: halo planes, then dz core matrices
    uint64_t *bars = reinterpret_cast<uint64_t *>(St + (size_t)S * stage_bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * S + 1);
    const uint32_t bar0 = tc_smem(bars);
    // full[st] = bar0 + 8 st, empty[st] = bar0 + 8 (S + st), done = bar0 + 16 S
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = a.B * hg.per_img;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc_mbar_init(bar0 + 8 * i, 128);
            tc_mbar_init(bar0 + 8 * (S + i), 1);
        }
        tc_mbar_init(bar0 + 16 * S, 1);
        tc_fence_mbar_init();
    }
    if (warp == 8) tc_alloc(tc_smem(tslot), kHwCols);
    for (int q = tid; q < 2048 / 16; q += kTcThreads)
        reinterpret_cast<uint4 *>(ones)[q] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    tc_fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp < 4) {
        int g = 0;
        long long sb_next = 0;
        if (blockIdx.x < n_tiles) {
            const int b = blockIdx.x / hg.per_img;
            sb_next = a.perm ? (long long)a.perm[a.b0 + b] : a.b0 + b;
        }
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++g) {
            const long long sb = sb_next;
            if (tile + (int)gridDim.x < n_tiles) {
                const int bn = (tile + (int)gridDim.x) / hg.per_img;
                sb_next = a.perm ? (long long)a.perm[a.b0 + bn] : a.b0 + bn;
            }
            const int st = g % S;
            if (!tc_mbar_wait(bar0 + 8 * (S + st), ((g / S) & 1) ^ 1)) {
                atomicOr(err, 1);
                break;
            }
            const int b = tile / hg.per_img, r0 = (tile - b * hg.per_img) * BM;
            unsigned char *stage = St + (size_t)st * stage_bytes;
            load_halo<CIN>(stage, a.in + (size_t)sb * a.H * a.H * CIN, hg, r0, tid, a.in);
            unsigned char *dzs = stage + halo_bytes;
            const bf16 *dzi = a.dz + (size_t)b * a.H * a.H * CH;
            {
                // a thread per row; 8 consecutive threads fill one core matrix
                const int i = tid;
                const int r = r0 + i, y = r / hg.Wp, x = r - y * hg.Wp;
                const bool ok = y < a.H && x < a.H;
                const bf16 *src = ok ? dzi + ((size_t)y * a.H + x) * CH : a.dz;
#pragma unroll
                for (int cg = 0; cg < 8; ++cg)
                    cp_async16_ca(dzs + ((i >> 3) * 8 + cg) * 128 + (i & 7) * 16, ok ? src + cg * 8 : a.dz, ok);
            }
            cp_async_commit();
            if (g >= LAG) {
                cp_async_wait<LAG>();
                tc_fence_proxy_async();
                tc_mbar_arrive(bar0 + 8 * ((g - LAG) % S));
            }
        }
        cp_async_wait<0>();
        tc_fence_proxy_async();
        for (int q = (g > LAG ? g - LAG : 0); q < g; ++q) tc_mbar_arrive(bar0 + 8 * (q % S));
    } else if (warp == 8) {
        if (lane == 0) {
            const uint32_t id_w = tc_idesc_bf16(64, CIN) | (1u << 15) | (1u << 16);   // both operands MN-major
            const uint32_t id_b = tc_idesc_bf16(64, 8) | (1u << 15) | (1u << 16);
            const uint32_t st_base = tc_smem(St), ones_a = tc_smem(ones);
            int g = 0;
            bool run = true;
            for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++g) {
                const int st = g % S;
                if (!tc_mbar_wait(bar0 + 8 * st, (g / S) & 1)) {
                    atomicOr(err, 1);
                    run = false;
                    break;
                }
                tc_fence_after();
                const uint32_t hs = st_base + (uint32_t)(st * stage_bytes), ds = hs + (uint32_t)halo_bytes;
                // the ten accumulators are independent: issue them interleaved
#pragma unroll 1
                for (int j = 0; j < BM / 16; ++j) {
                    const uint64_t adz = tc_desc(ds + j * 2048, 1024, 128);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int ky = tap / 3, kx = tap - ky * 3;
                        const uint32_t ht = hs + (uint32_t)((ky * hg.Wp + kx + 16 * j) * 16);
                        tc_mma(tmem + (uint32_t)(tap * CIN), adz, tc_desc(ht, 128, hg.plane), id_w, (g | j) != 0);
                    }
                    tc_mma(tmem + (uint32_t)K, adz, tc_desc(ones_a + j * 256, 128, 128), id_b, (g | j) != 0);
                }
                tc_commit(bar0 + 8 * (S + st));
            }
            if (run) tc_commit(bar0 + 16 * S);
            else atomicOr(err, 1);
        }
        __syncwarp();
    } else {
        // epilogue: warp 4 + e holds rows co = 16 e + lane (lanes 0-15)
        const int e = warp - 4;
        if (tc_mbar_wait(bar0 + 16 * S, 0)) {
            tc_fence_after();
            const int co = 16 * e + lane;
            float *dst = a.part + (size_t)blockIdx.x * (CH * K + CH);
#pragma unroll 1
            for (int c0 = 0; c0 < (K + 8 + 31) / 32; ++c0) {
                float v[32];
                tc_ld32(tmem + ((uint32_t)(32 * e) << 16) + (uint32_t)(32 * c0), v);
                if (lane < 16) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int k = 32 * c0 + q;
                        if (k < K) dst[(size_t)co * K + k] = v[q];
                        else if (k == K) dst[(size_t)CH * K + co] = v[q];
                    }
                }
            }
        } else {
            atomicOr(err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        tc_dealloc(tmem, kHwCols);
    }
}

// ---------------------------------------------------------------------------
// Weight and bias gradient of a 64-channel convolution (the stride-2 layers)
// on tcgen05: D^T[k][co] = sum_m im2col(in)[m][k] dz[m][co], k = tap 64 + ci.
// Each CTA takes chunks of 64 output pixels (m) and accumulates over all of
// them in TMEM; its partial goes to part[cta] and k_sum_parts adds the CTAs
// in order.
//   stage (per chunk): 80 planes of 64 pixels x 16 bytes, one per 8-channel
//     group k of the im2col: MN-major A operand, M = k, K = pixels.  Planes
//     0-71 are gathered; plane 72 holds ones and planes 73-79 zeros, written
//     once, so that M-tile 4 (planes 64-79) adds the bias gradient
//     sum_m dz[m][co] as accumulator row 576.  dz is stored as 8-pixel x
//     8-channel core matrices: MN-major B operand, N = co.
//   MMA: per 16 pixels, 5 M-tiles of 128 x 64 x 16 into 5 TMEM accumulators
//     (independent, interleaved).
//   epilogue: warp 4 + e reads accumulator rows 32 e .. 32 e + 31 of each
//     tile.
// ---------------------------------------------------------------------------
constexpr int kWt2Pix = 64;                      // pixels per chunk
constexpr int kWt2Planes = 80;                   // 72 im2col groups + ones + 7 zero planes
constexpr int kWt2PlaneBytes = kWt2Pix * 16;     // 1 KB
constexpr int kWt2StageBytes = kWt2Planes * kWt2PlaneBytes + kWt2Pix * CH * 2;   // 80 KB + 8 KB
constexpr int kWt2Stages = 2;
constexpr int kWt2Cols = 512;                    // 5 x 64 accumulator columns, rounded up to a power of two
constexpr size_t kWt2Smem = 128 + (size_t)kWt2Stages * kWt2StageBytes + 8 * (2 * kWt2Stages + 1) + 16;

__global__ void __launch_bounds__(kTcThreads, 1) k_wgrad_tc(const WgArgs a, int *__restrict__ err) {
    constexpr int K = 9 * CH, S = kWt2Stages;
    extern __shared__ __align__(128) unsigned char tc_raw[];
    unsigned char *base = tc_raw + ((128u - (tc_smem(tc_raw) & 127u)) & 127u);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)S * kWt2StageBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * S + 1);
    const uint32_t bar0 = tc_smem(bars);
    // full[st] = bar0 + 8 st, empty[st] = bar0 + 8 (S + st), done = bar0 + 16 S
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long M = (long long)a.B * a.Ho * a.Ho;
    const int n_chunks = (int)((M + kWt2Pix - 1) / kWt2Pix);

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc_mbar_init(bar0 + 8 * i, 128);
            tc_mbar_init(bar0 + 8 * (S + i), 1);
        }
        tc_mbar_init(bar0 + 16 * S, 1);
        tc_fence_mbar_init();
    }
    if (warp == 8) tc_alloc(tc_smem(tslot), kWt2Cols);
    // constant planes 72-79 of both stages: ones, then zeros
    for (int q = tid; q < S * 8 * kWt2PlaneBytes / 16; q += kTcThreads) {
        const int st = q / (8 * kWt2PlaneBytes / 16), r = q - st * (8 * kWt2PlaneBytes / 16);
        const uint32_t v = (r < kWt2PlaneBytes / 16) ? 0x3F803F80u : 0u;
        reinterpret_cast<uint4 *>(base + (size_t)st * kWt2StageBytes + 72 * kWt2PlaneBytes)[r] = make_uint4(v, v, v, v);
    }
    tc_fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp < 4) {
        // thread tid owns pixel p = tid % 64 of every chunk and the 8-channel
        // groups kg = tid / 64 + 2 i (im2col) and cg = tid / 64 + 2 i (dz)
        const int p = tid & 63, g0 = tid >> 6;
        constexpr int LAG = S - 1;
        int g = 0;
        for (int chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x, ++g) {
            const int st = g % S;
            if (!tc_mbar_wait(bar0 + 8 * (S + st), ((g / S) & 1) ^ 1)) {
                atomicOr(err, 1);
                break;
            }
            unsigned char *stage = base + (size_t)st * kWt2StageBytes;
            const long long m = (long long)chunk * kWt2Pix + p;
            const bool ok_m = m < M;
            int b = 0, oy = 0, ox = 0;
            if (ok_m) {
                b = (int)(m / ((long long)a.Ho * a.Ho));
                const int r = (int)(m - (long long)b * a.Ho * a.Ho);
                oy = r / a.Ho;
                ox = r - oy * a.Ho;
            }
            const long long sb = a.perm ? (long long)a.perm[a.b0 + b] : a.b0 + b;
            const bf16 *img = a.in + (size_t)sb * a.Hi * a.Hi * CH;
#pragma unroll 4
            for (int i = 0; i < 36; ++i) {
                const int kg = g0 + 2 * i, tap = kg >> 3, cgp = kg & 7;
                const int ky = tap / 3, kx = tap - ky * 3;
                const int iy = oy * a.stride + ky - 1, ix = ox * a.stride + kx - 1;
                const bool ok = ok_m && iy >= 0 && ix >= 0 && iy < a.Hi && ix < a.Hi;
                cp_async16_ca(stage + kg * kWt2PlaneBytes + p * 16,
                              ok ? img + ((size_t)iy * a.Hi + ix) * CH + cgp * 8 : a.in, ok);
            }
            unsigned char *dzs = stage + kWt2Planes * kWt2PlaneBytes;
            const bf16 *dzr = a.dz + (size_t)(ok_m ? m : 0) * CH;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int cg = g0 + 2 * i;
                cp_async16_ca(dzs + ((p >> 3) * 8 + cg) * 128 + (p & 7) * 16, ok_m ? dzr + cg * 8 : a.dz, ok_m);
            }
            cp_async_commit();
            if (g >= LAG) {
                cp_async_wait<LAG>();
                tc_fence_proxy_async();
                tc_mbar_arrive(bar0 + 8 * ((g - LAG) % S));
            }
        }
        cp_async_wait<0>();
        tc_fence_proxy_async();
        for (int q = (g > LAG ? g - LAG : 0); q < g; ++q) tc_mbar_arrive(bar0 + 8 * (q % S));
    } else if (warp == 8) {
        if (lane == 0) {
            // both operands MN-major
            const uint32_t idesc = tc_idesc_bf16(BM, CH) | (1u << 15) | (1u << 16);
            const uint32_t base_a = tc_smem(base);
            int g = 0;
            bool run = true;
            for (int chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x, ++g) {
                const int st = g % S;
                if (!tc_mbar_wait(bar0 + 8 * st, (g / S) & 1)) {
                    atomicOr(err, 1);
                    run = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = base_a + (uint32_t)(st * kWt2StageBytes);
                const uint32_t sd = sa + (uint32_t)(kWt2Planes * kWt2PlaneBytes);
#pragma unroll
                for (int s4 = 0; s4 < kWt2Pix / 16; ++s4) {
                    const uint64_t bdesc = tc_desc(sd + s4 * 2048, 1024, 128);
#pragma unroll
                    for (int t = 0; t < 5; ++t)
                        tc_mma(tmem + (uint32_t)(t * CH), tc_desc(sa + t * 16 * kWt2PlaneBytes + s4 * 256, 128,
                                                                  kWt2PlaneBytes),
                               bdesc, idesc, (g | s4) != 0);
                }
                tc_commit(bar0 + 8 * (S + st));
            }
            if (run) tc_commit(bar0 + 16 * S);
            else atomicOr(err, 1);
        }
        __syncwarp();
    } else {
        const int e = warp - 4;
        float *dst = a.part + (size_t)blockIdx.x * (CH * K + CH);
        const bool any = blockIdx.x < n_chunks;
        if (!any || tc_mbar_wait(bar0 + 16 * S, 0)) {
            tc_fence_after();
#pragma unroll 1
            for (int t = 0; t < 5; ++t) {
                const int k = 128 * t + 32 * e + lane;   // accumulator row of this lane
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    float v[32];
                    tc_ld32(tmem + ((uint32_t)(32 * e) << 16) + (uint32_t)(t * CH + 32 * h), v);
                    if (!any) {
#pragma unroll
                        for (int q = 0; q < 32; ++q) v[q] = 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int co = 32 * h + q;
                        if (k < K) dst[(size_t)co * K + k] = v[q];
                        else if (k == K) dst[(size_t)CH * K + co] = v[q];
                    }
                }
            }
        } else {
            atomicOr(err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        tc_dealloc(tmem, kWt2Cols);
    }
}

// grad[q] = sum over splits (in order) of part[split * stride + q], q < count.
// A CTA owns 32 consecutive q (one per lane); warp w adds splits w, w + 8, ...
// and the 8 warp sums are added in warp order.
__global__ void __launch_bounds__(256) k_sum_parts(const float *__restrict__ part, int splits, int count,
                                                   long long stride, float *__restrict__ grad) {
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    float sum = 0.f;
    if (q < count) {
#pragma unroll 4
        for (int p = w; p < splits; p += 8) sum += part[(size_t)p * stride + q];
    }
    red[w][lane] = sum;
    __syncthreads();
    if (w == 0 && q < count) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += red[k][lane];
        grad[q] = t;
    }
}

// The same sums four consecutive q per lane (16-byte loads and stores; count,
// stride and both base addresses multiples of 4 floats): a CTA owns 128 q.
// Each q is added in the same order as by k_sum_parts.
__global__ void __launch_bounds__(256) k_sum_parts4(const float4 *__restrict__ part, int splits, int count4,
                                                    long long stride4, float4 *__restrict__ grad) {
    __shared__ float4 red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < count4) {
#pragma unroll 4
        for (int p = w; p < splits; p += 8) {
            const float4 v = part[(size_t)p * stride4 + q];
            sum.x += v.x;
            sum.y += v.y;
            sum.z += v.z;
            sum.w += v.w;
        }
    }
    red[w][lane] = sum;
    __syncthreads();
    if (w == 0 && q < count4) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            t.x += red[k][lane].x;
            t.y += red[k][lane].y;
            t.z += red[k][lane].z;
            t.w += red[k][lane].w;
        }
        grad[q] = t;
    }
}


// ---------------------------------------------------------------------------
// Head: dense layer from the flattened last feature map (F = H3 H3 64 values
// per sample, NHWC order) to the 4 outputs; loss; and their backward.
// ---------------------------------------------------------------------------
constexpr int kHeadThreads = 256;

// part_out[b][part][j] = sum over features e of part `part` of Wfc[j][e]
// a3[b][e].  Block (part, g) takes samples 8 g .. 8 g + 7 (so that each
// weight loaded serves eight samples) and features [part seg, (part + 1)
// seg); k_head_combine adds the parts in order.
constexpr int kHeadSamples = 8;
__global__ void __launch_bounds__(kHeadThreads)
k_head_fwd(const bf16 *__restrict__ a3, int F, int B, const float *__restrict__ wfc, int parts,
           float *__restrict__ part_out) {
    const int part = blockIdx.x, b0 = blockIdx.y * kHeadSamples, seg = (F + parts - 1) / parts;
    const int e0 = part * seg, e1 = min(F, e0 + seg);
    const int nb = min(kHeadSamples, B - b0);
    float acc[kHeadSamples][4];
#pragma unroll
    for (int s = 0; s < kHeadSamples; ++s)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[s][j] = 0.f;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = wfc[(size_t)j * F + e];
#pragma unroll
        for (int s = 0; s < kHeadSamples; ++s) {
            if (s < nb) {
                const float v = __bfloat162float(a3[(size_t)(b0 + s) * F + e]);
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[s][j] = fmaf(w[j], v, acc[s][j]);
            }
        }
    }
    __shared__ float sh[kHeadThreads / 32][kHeadSamples * 4];
#pragma unroll
    for (int s = 0; s < kHeadSamples; ++s)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v = acc[s][j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][s * 4 + j] = v;
        }
    __syncthreads();
    if (threadIdx.x < kHeadSamples * 4) {
        const int s = threadIdx.x >> 2, j = threadIdx.x & 3;
        if (s < nb) {
            float o = 0.f;
            for (int w = 0; w < kHeadThreads / 32; ++w) o += sh[w][threadIdx.x];
            part_out[((size_t)(b0 + s) * parts + part) * 4 + j] = o;
        }
    }
}

// out[b][j] = bfc[j] + the parts' sums in part order; with targets, loss[b]
// = sum_j (out - tgt)^2 and dout = d(mean loss)/d out.
__global__ void k_head_combine(const float *__restrict__ part_out, int parts, int B, const float *__restrict__ bfc,
                               const float *__restrict__ tgt, float *__restrict__ out, float *__restrict__ loss,
                               float *__restrict__ dout) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float l = 0.f;
    for (int j = 0; j < 4; ++j) {
        float o = bfc[j];
        for (int p = 0; p < parts; ++p) o += part_out[((size_t)b * parts + p) * 4 + j];
        out[b * 4 + j] = o;
        if (tgt) {
            const float d = o - tgt[b * 4 + j];
            l = fmaf(d, d, l);
            dout[b * 4 + j] = 2.f / (4.f * (float)B) * d;
        }
    }
    if (tgt) loss[b] = l;
}

// Head backward in one pass over a3: dz3[b][e] = (a3 > 0) sum_j dout[b][j]
// Wfc[j][e], and the weight / bias gradient partials of sample group
// blockIdx.y: part[g][j * F + e] = sum_{b in g} dout[b][j] a3[b][e],
// part[g][4 F + j] = sum_{b in g} dout[b][j] (k_sum_parts adds the groups in
// order).  A CTA owns 64 features (two per lane) and its 8 warps split the
// group's samples (b = warp, warp + 8, ...), their sums added in warp order.
// F is a multiple of 64.
constexpr int kHeadGroups = 8;
__global__ void __launch_bounds__(256) k_head_bwd(const bf16 *__restrict__ a3, const float *__restrict__ dout,
                                                  const float *__restrict__ wfc, int B, int F, int per_group,
                                                  bf16 *__restrict__ dz3, float *__restrict__ part) {
    __shared__ float red[8][4][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 64 + 2 * lane;
    const int g = blockIdx.y, bs = g * per_group, be = min(B, bs + per_group);
    float wf[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        wf[j][0] = wfc[(size_t)j * F + e];
        wf[j][1] = wfc[(size_t)j * F + e + 1];
    }
    float acc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
    for (int b = bs + w; b < be; b += 8) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(a3 + (size_t)b * F + e);
        const float v0 = __low2float(v), v1 = __high2float(v);
        const float4 d = *reinterpret_cast<const float4 *>(dout + 4 * b);
        const float dj[4] = {d.x, d.y, d.z, d.w};
        float g0 = 0.f, g1 = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[j][0] = fmaf(dj[j], v0, acc[j][0]);
            acc[j][1] = fmaf(dj[j], v1, acc[j][1]);
            g0 = fmaf(dj[j], wf[j][0], g0);
            g1 = fmaf(dj[j], wf[j][1], g1);
        }
        *reinterpret_cast<__nv_bfloat162 *>(dz3 + (size_t)b * F + e) =
            __floats2bfloat162_rn(v0 > 0.f ? g0 : 0.f, v1 > 0.f ? g1 : 0.f);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        red[w][j][2 * lane] = acc[j][0];
        red[w][j][2 * lane + 1] = acc[j][1];
    }
    __syncthreads();
    float *pg = part + (size_t)g * (4 * (size_t)F + 4);
    const int j = threadIdx.x >> 6, c = threadIdx.x & 63;
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += red[q][j][c];
    pg[(size_t)j * F + blockIdx.x * 64 + c] = sum;
    if (blockIdx.x == 0 && w == 0) {
        float sb[4] = {0.f, 0.f, 0.f, 0.f};
        for (int b = bs + lane; b < be; b += 32) {
            const float4 d = *reinterpret_cast<const float4 *>(dout + 4 * b);
            sb[0] += d.x;
            sb[1] += d.y;
            sb[2] += d.z;
            sb[3] += d.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sb[q] += __shfl_xor_sync(0xffffffffu, sb[q], o);
        if (lane < 4) pg[4 * (size_t)F + lane] = sb[lane];
    }
}

// ---------------------------------------------------------------------------
// Parameters: Adam, BF16 copies (and the transposed copies for the input
// gradient), normalisation of targets and outputs.
// ---------------------------------------------------------------------------
// Where the three convolutions' weights sit in the parameter vector, and
// their BF16 copies (wt: the transposed copy of a 64-channel layer).
struct PackDst {
    long long off[3];
    int cin[3];
    bf16 *wb[3], *wt[3];
};

// One Adam step (as k_adam) that also refreshes the BF16 copies of the
// updated convolution weights (as k_pack_w): one pass over the parameters.
__global__ void k_adam_pack(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2, const PackDst pd) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    w[q] = wq;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const long long r = q - pd.off[l], K = 9LL * pd.cin[l];
        if (r >= 0 && r < CH * K) {
            const bf16 b = __float2bfloat16_rn(wq);
            pd.wb[l][r] = b;
            if (pd.wt[l]) {
                const int co = (int)(r / K), k = (int)(r - co * K);
                const int tap = k / pd.cin[l], ci = k - tap * pd.cin[l];
                pd.wt[l][(size_t)ci * (9 * CH) + tap * CH + co] = b;
            }
        }
    }
}

// w_bf16[co][k] = w[co][k]; wt[ci][tap * 64 + co] = w[co][tap * cin + ci] (cin = 64 only).
__global__ void k_pack_w(const float *__restrict__ w, int cin, bf16 *__restrict__ wb, bf16 *__restrict__ wt) {
    const int K = 9 * cin;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= CH * K) return;
    const int co = q / K, k = q - co * K;
    const bf16 v = __float2bfloat16_rn(w[q]);
    wb[q] = v;
    if (wt) {
        const int tap = k / cin, ci = k - tap * cin;
        wt[(size_t)ci * (9 * CH) + tap * CH + co] = v;
    }
}

// Normalisation of the four misregistration parameters (centre, range).
struct Norm4 {
    double c[4], r[4];
};

__global__ void k_targets(const double *__restrict__ p, long long n, const Norm4 nm, float *__restrict__ t) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) t[4 * q + k] = (float)((p[4 * q + k] - nm.c[k]) / nm.r[k]);
}

__global__ void k_denorm(const float *__restrict__ o, long long n, const Norm4 nm, double *__restrict__ p) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) p[4 * q + k] = nm.c[k] + nm.r[k] * (double)o[4 * q + k];
}

__global__ void k_gather_targets(const float *__restrict__ t, const int *__restrict__ perm, long long b0, int B,
                                 float *__restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    const long long s = perm[b0 + q];
    for (int k = 0; k < 4; ++k) out[4 * q + k] = t[4 * s + k];
}

__global__ void k_to_bf16(const float *__restrict__ x, long long n, bf16 *__restrict__ y) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) y[q] = __float2bfloat16_rn(x[q]);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

template <typename T>
cudaError_t dmalloc(T **p, size_t count) {
    return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t sum_parts(const float *part, int splits, int count, long long stride, float *grad, cudaStream_t st) {
    const bool v4 = count % 4 == 0 && stride % 4 == 0 && (reinterpret_cast<uintptr_t>(part) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(grad) & 15) == 0;
    if (v4)
        k_sum_parts4<<<blocks_for(count / 4, 32), 256, 0, st>>>(reinterpret_cast<const float4 *>(part), splits,
                                                               count / 4, stride / 4, reinterpret_cast<float4 *>(grad));
    else
        k_sum_parts<<<blocks_for(count, 32), 256, 0, st>>>(part, splits, count, stride, grad);
    return cudaGetLastError();
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
    }
    return n;
}

// The tensor-core kernels allocate all 512 TMEM columns of an SM; asking for
// more than half of an SM's shared memory keeps a second CTA off the SM
// (it would only wait in tcgen05.alloc for the first to finish).
constexpr size_t kExclusiveSmem = 116 * 1024;

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (once per size).
template <typename F>
cudaError_t smem_limit(F *k, size_t bytes, size_t &set_to) {
    if (bytes <= set_to) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) set_to = bytes;
    return e;
}

// Persistent launch of the tcgen05 convolution: as many CTAs as fit on the
// device at once (shared memory limits them to one or two per SM, so that
// their TMEM columns always fit in the 512 of an SM), at most one per tile.
template <bool DGRAD, int CIN>
cudaError_t launch_tc(const ConvArgs &a, int *err, cudaStream_t st) {
    static size_t set_to = 0;
    static int per_sm = 0;
    const size_t smem = std::max(TcCfg<CIN>::SMEM, kExclusiveSmem);
    cudaError_t e = smem_limit(k_conv_tc<DGRAD, CIN>, smem, set_to);
    if (e != cudaSuccess) return e;
    if (per_sm == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_tc<DGRAD, CIN>, kTcThreads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        if (per_sm * kTcCols > 512) per_sm = 512 / kTcCols;
    }
    if (DGRAD && a.stride != 2) return cudaErrorInvalidValue;   // parity classes assume stride 2
    const long long tiles = tc_tile<DGRAD>(a, 0, nullptr);
    if (tiles == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)sm_count() * per_sm);
    k_conv_tc<DGRAD, CIN><<<grid, kTcThreads, smem, st>>>(a, err);
    return cudaGetLastError();
}

// Stride-1 forward convolution on shifted windows: persistent, as many CTAs
// as fit (shared memory limits them to one or two per SM, whose TMEM columns
// then fit in the 512 of an SM), at most one per tile.
template <int CIN>
cudaError_t launch_halo_fwd(const ConvArgs &a, const CUtensorMap &map, int *err, cudaStream_t st) {
    static size_t set_to = 0;
    static int per_sm = 0, per_sm_for = -1;
    const HaloGeo hg = halo_geo(a.Ho);
    const size_t smem = std::max(HaloTmaCfg<CIN>::smem(halo_tma(hg)), kExclusiveSmem);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = smem_limit(k_conv_halo<CIN>, smem, set_to);
    if (e != cudaSuccess) return e;
    if (per_sm_for != a.Ho) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_halo<CIN>, kTcThreads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        if (per_sm * kTcCols > 512) per_sm = 512 / kTcCols;
        per_sm_for = a.Ho;
    }
    const long long tiles = (long long)a.B * hg.per_img;
    if (tiles == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)sm_count() * per_sm);
    k_conv_halo<CIN><<<grid, kTcThreads, smem, st>>>(a, map, err);
    return cudaGetLastError();
}

// Tensor map of n samples of a [n][H][H][C] BF16 activation (16-byte
// aligned): boxes of 8 channels x bx columns x by rows, element stride es
// along x and y, zero fill outside.
cudaError_t make_act_map(CUtensorMap *map, const bf16 *act, long long n, int H, int C, int bx, int by, int es) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if ((reinterpret_cast<uintptr_t>(act) & 15) != 0 || n < 1) return cudaErrorInvalidValue;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)H, (cuuint64_t)H, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)H * C * 2, (cuuint64_t)H * H * C * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)(es * bx), (cuuint32_t)(es * by), 1};
    const cuuint32_t estr[4] = {1, (cuuint32_t)es, (cuuint32_t)es, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(act), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// k_conv_parity's map of a 64-channel activation ([kBatchCap][H][H][64]).
cudaError_t make_parity_map(CUtensorMap *map, const bf16 *act, int H) {
    const ParGeo pg = par_geo(H, conv_out(H, 2));
    return make_act_map(map, act, kBatchCap, H, CH, pg.Wq, pg.NR, 2);
}

// k_conv_halo's map of n network inputs ([n][H0][H0][C0]).
cudaError_t make_input_map(CUtensorMap *map, const bf16 *x, long long n, int H, int C) {
    const HaloGeo hg = halo_geo(H);
    return make_act_map(map, x, n, H, C, hg.Wp, halo_tma(hg).NR, 1);
}

// Stride-2 forward convolution on parity planes: persistent, one CTA per SM
// (shared memory), at most one per tile.
cudaError_t launch_parity_fwd(const ConvArgs &a, const CUtensorMap &map, int *err, cudaStream_t st) {
    static size_t set_to = 0;
    const ParGeo pg = par_geo(a.Hi, a.Ho);
    const size_t smem = std::max(ParCfg::smem(pg), kExclusiveSmem);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = smem_limit(k_conv_parity, smem, set_to);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)a.B * pg.per_img;
    if (tiles == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)sm_count());
    k_conv_parity<<<grid, kTcThreads, smem, st>>>(a, map, err);
    return cudaGetLastError();
}

cudaError_t launch_conv_fwd(const CnnState &S, int layer, const bf16 *in, const CUtensorMap &map, const int *perm,
                            long long b0, int B, cudaStream_t st) {
    ConvArgs a{};
    a.in = in;
    a.perm = perm;
    a.b0 = b0;
    a.B = B;
    if (layer == 1) {
        a.w = S.w1; a.bias = S.master + S.off_b1; a.out = S.a1; a.Hi = S.H0; a.Ho = S.H1; a.stride = 1;
    } else if (layer == 2) {
        a.w = S.w2; a.bias = S.master + S.off_b2; a.out = S.a2; a.Hi = S.H1; a.Ho = S.H2; a.stride = 2;
    } else {
        a.w = S.w3; a.bias = S.master + S.off_b3; a.out = S.a3; a.Hi = S.H2; a.Ho = S.H3; a.stride = 2;
    }
    if (layer == 1)
        return S.C0 == 32 ? launch_halo_fwd<32>(a, map, S.d_err, st) : launch_halo_fwd<64>(a, map, S.d_err, st);
    return launch_parity_fwd(a, map, S.d_err, st);
}

// Input gradient of layer 3 (into dz2) or layer 2 (into dz1).
cudaError_t launch_conv_dgrad(const CnnState &S, int layer, int B, cudaStream_t st) {
    ConvArgs a{};
    a.B = B;
    a.stride = 2;
    if (layer == 3) {
        a.in = S.dz3; a.w = S.w3t; a.act = S.a2; a.out = S.dz2; a.Hi = S.H2; a.Ho = S.H3;
    } else {
        a.in = S.dz2; a.w = S.w2t; a.act = S.a1; a.out = S.dz1; a.Hi = S.H1; a.Ho = S.H2;
    }
    return launch_tc<true, 64>(a, S.d_err, st);
}

cudaError_t launch_wgrad(const CnnState &S, int layer, const bf16 *in, const int *perm, long long b0, int B,
                         cudaStream_t st) {
    WgArgs a{};
    a.in = in;
    a.perm = perm;
    a.b0 = b0;
    a.B = B;
    a.part = S.wpart;
    int cin;
    long long off_w;
    if (layer == 1) {
        a.dz = S.dz1; a.Hi = S.H0; a.Ho = S.H1; a.stride = 1; cin = S.C0; off_w = S.off_w1;
    } else if (layer == 2) {
        a.dz = S.dz2; a.Hi = S.H1; a.Ho = S.H2; a.stride = 2; cin = CH; off_w = S.off_w2;
    } else {
        a.dz = S.dz3; a.Hi = S.H2; a.Ho = S.H3; a.stride = 2; cin = CH; off_w = S.off_w3;
    }
    if (layer == 1 && cin == 32) {
        // shifted windows on tcgen05, one CTA per SM
        static size_t set_to = 0;
        HaloWgArgs h{};
        h.dz = a.dz;
        h.in = in;
        h.perm = perm;
        h.b0 = b0;
        h.B = B;
        h.H = a.Ho;
        h.part = S.wpart;
        const HaloGeo hg = halo_geo(h.H);
        const size_t smem = std::max(wgrad_halo_smem(hg), kExclusiveSmem);
        if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
        cudaError_t e = smem_limit(k_wgrad_halo, smem, set_to);
        if (e != cudaSuccess) return e;
        const long long tiles = (long long)B * hg.per_img;
        const int grid = (int)std::min<long long>(std::min<long long>(tiles, sm_count()), 296);
        if (grid < 1) return cudaErrorInvalidConfiguration;
        k_wgrad_halo<<<grid, kTcThreads, smem, st>>>(h, S.d_err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int K = 9 * cin;
        return sum_parts(S.wpart, grid, CH * K + CH, (long long)CH * K + CH, S.grad + off_w, st);
    }
    if (cin == CH) {
        // 64-channel layers: tcgen05, one CTA per SM, one partial per CTA
        static size_t set_to = 0;
        const size_t smem = std::max(kWt2Smem, kExclusiveSmem);
        cudaError_t e = smem_limit(k_wgrad_tc, smem, set_to);
        if (e != cudaSuccess) return e;
        const long long chunks = ((long long)B * a.Ho * a.Ho + kWt2Pix - 1) / kWt2Pix;
        const int grid = (int)std::min<long long>(std::min<long long>(chunks, sm_count()), 296);
        if (grid < 1) return cudaErrorInvalidConfiguration;
        k_wgrad_tc<<<grid, kTcThreads, smem, st>>>(a, S.d_err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int K = 9 * cin;
        return sum_parts(S.wpart, grid, CH * K + CH, (long long)CH * K + CH, S.grad + off_w, st);
    }
    return cudaErrorInvalidValue;   // layer 1 has 32 or 64 channels, layers 2-3 64
}

PackDst pack_dst(const CnnState &S) {
    PackDst d;
    d.off[0] = S.off_w1; d.off[1] = S.off_w2; d.off[2] = S.off_w3;
    d.cin[0] = S.C0; d.cin[1] = CH; d.cin[2] = CH;
    d.wb[0] = S.w1; d.wb[1] = S.w2; d.wb[2] = S.w3;
    d.wt[0] = nullptr; d.wt[1] = S.w2t; d.wt[2] = S.w3t;
    return d;
}

cudaError_t pack_weights(CnnState &S, cudaStream_t st) {
    k_pack_w<<<blocks_for(CH * 9 * S.C0, 256), 256, 0, st>>>(S.master + S.off_w1, S.C0, S.w1, nullptr);
    k_pack_w<<<blocks_for(CH * 9 * CH, 256), 256, 0, st>>>(S.master + S.off_w2, CH, S.w2, S.w2t);
    k_pack_w<<<blocks_for(CH * 9 * CH, 256), 256, 0, st>>>(S.master + S.off_w3, CH, S.w3, S.w3t);
    return cudaGetLastError();
}

// Forward of B <= kBatchCap samples (inputs at in / perm / b0); with targets,
// the per-sample squared errors go to S.loss.
cudaError_t forward(CnnState &S, const bf16 *in, const CUtensorMap &in_map, const int *perm, long long b0, int B,
                    const float *tgt, cudaStream_t st) {
    cudaError_t e;
    if ((e = launch_conv_fwd(S, 1, in, in_map, perm, b0, B, st)) != cudaSuccess) return e;
    if ((e = launch_conv_fwd(S, 2, S.a1, S.map_a1, nullptr, 0, B, st)) != cudaSuccess) return e;
    if ((e = launch_conv_fwd(S, 3, S.a2, S.map_a2, nullptr, 0, B, st)) != cudaSuccess) return e;
    // the head: blocks of 8 samples x a share of the features, about 256
    // blocks in all (32 feature parts for one group of 8, 8 for 32 groups)
    const int groups = (B + kHeadSamples - 1) / kHeadSamples;
    const int parts = std::max(1, std::min(32, kBatchCap / groups));
    k_head_fwd<<<dim3(parts, groups), kHeadThreads, 0, st>>>(S.a3, S.H3 * S.H3 * CH, B, S.master + S.off_fc, parts,
                                                             S.hpart);
    k_head_combine<<<blocks_for(B, 64), 64, 0, st>>>(S.hpart, parts, B, S.master + S.off_bfc, tgt, S.out, S.loss,
                                                     S.dout);
    return cudaGetLastError();
}

cudaError_t backward(CnnState &S, const bf16 *in, const int *perm, long long b0, int B, const float *tgt,
                     cudaStream_t st) {
    cudaError_t e;
    const int F = S.H3 * S.H3 * CH;
    (void)tgt;   // dout was formed by the forward pass
    // head: dz3 and the dense layer's gradient partials of up to 8 sample
    // groups in one pass over a3, then the groups added in order
    const int per_group = (B + kHeadGroups - 1) / kHeadGroups;
    const int groups = (B + per_group - 1) / per_group;
    k_head_bwd<<<dim3(F / 64, groups), 256, 0, st>>>(S.a3, S.dout, S.master + S.off_fc, B, F, per_group, S.dz3,
                                                     S.wpart);
    if ((e = sum_parts(S.wpart, groups, 4 * F + 4, 4LL * F + 4, S.grad + S.off_fc, st)) != cudaSuccess) return e;
    if ((e = launch_wgrad(S, 3, S.a2, nullptr, 0, B, st)) != cudaSuccess) return e;
    if ((e = launch_conv_dgrad(S, 3, B, st)) != cudaSuccess) return e;
    if ((e = launch_wgrad(S, 2, S.a1, nullptr, 0, B, st)) != cudaSuccess) return e;
    if ((e = launch_conv_dgrad(S, 2, B, st)) != cudaSuccess) return e;
    return launch_wgrad(S, 1, in, perm, b0, B, st);
}

cudaError_t alloc_state(CnnState &S) {
    cudaError_t e = cudaSuccess;
    const long long P = S.n_params;
    const size_t a1 = (size_t)kBatchCap * S.H1 * S.H1 * CH, a2 = (size_t)kBatchCap * S.H2 * S.H2 * CH,
                 a3 = (size_t)kBatchCap * S.H3 * S.H3 * CH;
    const int splits = 296;
    S.wpart_floats = (long long)splits * (CH * 9 * CH + CH);
#define SYNIM_A(ptr, n) \
    if (e == cudaSuccess) e = dmalloc(&(ptr), (n))
    SYNIM_A(S.master, P);
    SYNIM_A(S.adam_m, P);
    SYNIM_A(S.adam_v, P);
    SYNIM_A(S.grad, P);
    SYNIM_A(S.w1, (size_t)CH * 9 * S.C0);
    SYNIM_A(S.w2, (size_t)CH * 9 * CH);
    SYNIM_A(S.w3, (size_t)CH * 9 * CH);
    SYNIM_A(S.w2t, (size_t)CH * 9 * CH);
    SYNIM_A(S.w3t, (size_t)CH * 9 * CH);
    SYNIM_A(S.x, (size_t)kBatchCap * S.H0 * S.H0 * S.C0);
    SYNIM_A(S.a1, a1);
    SYNIM_A(S.a2, a2);
    SYNIM_A(S.a3, a3);
    SYNIM_A(S.dz1, a1);
    SYNIM_A(S.dz2, a2);
    SYNIM_A(S.dz3, a3);
    SYNIM_A(S.out, (size_t)kBatchCap * 4);
    SYNIM_A(S.loss, (size_t)kBatchCap);
    SYNIM_A(S.dout, (size_t)kBatchCap * 4);
    SYNIM_A(S.hpart, (size_t)kBatchCap * 32 * 4);
    SYNIM_A(S.tgt, (size_t)kBatchCap * 4);
    SYNIM_A(S.wpart, (size_t)S.wpart_floats);
    SYNIM_A(S.d_err, 1);
#undef SYNIM_A
    if (e == cudaSuccess) e = cudaMemset(S.d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&S.h_loss, sizeof(float) * kBatchCap);
    if (e == cudaSuccess) e = make_parity_map(&S.map_a1, S.a1, S.H1);
    if (e == cudaSuccess) e = make_parity_map(&S.map_a2, S.a2, S.H2);
    if (e == cudaSuccess) e = make_input_map(&S.map_x, S.x, kBatchCap, S.H0, S.C0);
    return e;
}

synim_status cfail(synim_ctx *c, synim_status s, const std::string &m) {
    c->err = m;
    return s;
}

synim_status ccuda(synim_ctx *c, cudaError_t e, const char *what) {
    return cfail(c, e == cudaErrorMemoryAllocation ? SYNIM_ERR_OOM : SYNIM_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

Norm4 norm4(const CnnState &S) {
    Norm4 nm;
    for (int k = 0; k < 4; ++k) {
        nm.c[k] = S.center[k];
        nm.r[k] = S.range[k];
    }
    return nm;
}

// After a synchronisation: SYNIM_ERR_TIMEOUT if a tensor-core convolution
// flagged a bounded wait that gave up (the flag is cleared).
synim_status check_tc(synim_ctx *c, CnnState &S, const char *what) {
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, S.d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ccuda(c, e, what);
    if (flag == 0) return SYNIM_OK;
    cudaMemset(S.d_err, 0, sizeof(int));
    return cfail(c, SYNIM_ERR_TIMEOUT, std::string(what) + ": a tensor-core pipeline wait timed out");
}

}  // namespace

int cnn_n_params(int C0, int H0) {
    const int H3 = conv_out(conv_out(H0, 2), 2);
    return CH * 9 * C0 + CH + 2 * (CH * 9 * CH + CH) + 4 * H3 * H3 * CH + 4;
}

bool cnn_ready(const synim_ctx *c, std::string &why) {
    if (c->cnn && c->cnn->ready) return true;
    why = "the network has not been initialised (synim_cnn_init) or trained";
    return false;
}

cudaError_t cnn_predict_slopes(synim_ctx *c, const float *y, long long n, double *params_out, cudaStream_t st,
                               std::string &why) {
    CnnState *S = c->cnn;
    if (!S || !S->ready) {
        why = "the network has not been initialised (synim_cnn_init) or trained";
        return cudaErrorNotReady;
    }
    const long long per = (long long)S->H0 * S->H0 * S->C0;
    cudaError_t e = cudaSuccess;
    for (long long s0 = 0; s0 < n && e == cudaSuccess; s0 += kBatchCap) {
        const int B = (int)std::min<long long>(kBatchCap, n - s0);
        k_to_bf16<<<blocks_for(B * per, 256), 256, 0, st>>>(y + s0 * per, B * per, S->x);
        if ((e = forward(*S, S->x, S->map_x, nullptr, 0, B, nullptr, st)) != cudaSuccess) break;
        k_denorm<<<blocks_for(B, 128), 128, 0, st>>>(S->out, B, norm4(*S), params_out + 4 * s0);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace synim

using namespace synim;

extern "C" {

int32_t synim_cnn_n_params(int32_t n_sub, int32_t n_channels) { return cnn_n_params(n_channels, n_sub); }

synim_status synim_cnn_init(synim_ctx *ctx, const float *params, const double *norm) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->probe) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_init: attach probes first");
    if (!params || !norm) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_init: params and norm are required");
    int n_sub = 0, C = 0;
    synim_probe_query(ctx, &n_sub, &C, nullptr);
    if (C != 32 && C != 64) return cfail(ctx, SYNIM_ERR_SHAPE, "cnn_init: 2 n_modes must be 32 or 64");
    for (int k = 0; k < 4; ++k)
        if (!(norm[4 + k] > 0.0)) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_init: ranges must be > 0");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cnn_destroy(ctx->cnn);
    ctx->cnn = nullptr;
    ++ctx->est_gen;
    CnnState *S = new CnnState();
    S->H0 = n_sub;
    S->C0 = C;
    S->H1 = n_sub;
    S->H2 = conv_out(S->H1, 2);
    S->H3 = conv_out(S->H2, 2);
    S->n_params = cnn_n_params(C, n_sub);
    S->off_w1 = 0;
    S->off_b1 = S->off_w1 + (long long)CH * 9 * C;
    S->off_w2 = S->off_b1 + CH;
    S->off_b2 = S->off_w2 + (long long)CH * 9 * CH;
    S->off_w3 = S->off_b2 + CH;
    S->off_b3 = S->off_w3 + (long long)CH * 9 * CH;
    S->off_fc = S->off_b3 + CH;
    S->off_bfc = S->off_fc + 4LL * S->H3 * S->H3 * CH;
    for (int k = 0; k < 4; ++k) {
        S->center[k] = norm[k];
        S->range[k] = norm[4 + k];
    }
    cudaError_t e = alloc_state(*S);
    if (e == cudaSuccess) e = cudaMemcpy(S->master, params, sizeof(float) * S->n_params, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(S->adam_m, 0, sizeof(float) * S->n_params);
    if (e == cudaSuccess) e = cudaMemset(S->adam_v, 0, sizeof(float) * S->n_params);
    if (e == cudaSuccess) e = pack_weights(*S, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cnn_destroy(S);
        return ccuda(ctx, e, "cnn_init");
    }
    S->ready = true;
    ctx->cnn = S;
    return SYNIM_OK;
}

synim_status synim_cnn_get(const synim_ctx *ctx, float *params, double *norm) {
    if (!ctx || !ctx->cnn) return SYNIM_ERR_INVALID_ARG;
    const CnnState *S = ctx->cnn;
    if (params && cudaMemcpy(params, S->master, sizeof(float) * S->n_params, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SYNIM_ERR_CUDA;
    if (norm)
        for (int k = 0; k < 4; ++k) {
            norm[k] = S->center[k];
            norm[4 + k] = S->range[k];
        }
    return SYNIM_OK;
}

// Checkpoint: a 128-byte little-endian header, then the FP32 parameters,
// Adam first and second moments ([n_params] each).
struct CnnCkpt {
    char magic[8];         // "SYNIMCNN"
    uint32_t version;      // 1
    int32_t n_sub, channels, step;
    int64_t n_params;
    double norm[8];        // center[4], range[4]
    uint8_t reserved[128 - 8 - 4 - 12 - 8 - 64];
};
static_assert(sizeof(CnnCkpt) == 128, "checkpoint header is 128 bytes");
constexpr char kCkptMagic[8] = {'S', 'Y', 'N', 'I', 'M', 'C', 'N', 'N'};

synim_status synim_cnn_save(const synim_ctx *ctx, void *buf, int64_t cap, int64_t *bytes) {
    if (!ctx || !ctx->cnn || !bytes) return SYNIM_ERR_INVALID_ARG;
    const CnnState *S = ctx->cnn;
    const int64_t total = (int64_t)sizeof(CnnCkpt) + 3 * (int64_t)sizeof(float) * S->n_params;
    *bytes = total;
    if (!buf) return SYNIM_OK;
    if (cap < total) return SYNIM_ERR_INVALID_ARG;
    CnnCkpt h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.n_sub = S->H0;
    h.channels = S->C0;
    h.step = S->step;
    h.n_params = S->n_params;
    for (int k = 0; k < 4; ++k) {
        h.norm[k] = S->center[k];
        h.norm[4 + k] = S->range[k];
    }
    unsigned char *out = static_cast<unsigned char *>(buf);
    std::memcpy(out, &h, sizeof(h));
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    const size_t P = sizeof(float) * (size_t)S->n_params;
    cudaError_t e = cudaMemcpy(out + sizeof(h), S->master, P, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out + sizeof(h) + P, S->adam_m, P, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out + sizeof(h) + 2 * P, S->adam_v, P, cudaMemcpyDeviceToHost);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return e == cudaSuccess ? SYNIM_OK : SYNIM_ERR_CUDA;
}

synim_status synim_cnn_load(synim_ctx *ctx, const void *buf, int64_t bytes) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!buf || bytes < (int64_t)sizeof(CnnCkpt))
        return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_load: no buffer or shorter than the header");
    CnnCkpt h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1)
        return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_load: not a version-1 network checkpoint");
    if (!ctx->probe) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_load: attach probes first");
    int n_sub = 0, C = 0;
    synim_probe_query(ctx, &n_sub, &C, nullptr);
    if (h.n_sub != n_sub || h.channels != C || h.n_params != cnn_n_params(C, n_sub))
        return cfail(ctx, SYNIM_ERR_SHAPE, "cnn_load: the checkpoint's map shape differs from the attached probes'");
    if (h.step < 0 || bytes < (int64_t)sizeof(CnnCkpt) + 3 * (int64_t)sizeof(float) * h.n_params)
        return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_load: truncated checkpoint");
    const unsigned char *in = static_cast<const unsigned char *>(buf) + sizeof(CnnCkpt);
    const size_t P = sizeof(float) * (size_t)h.n_params;
    std::vector<float> w((size_t)h.n_params);
    std::memcpy(w.data(), in, P);
    synim_status st = synim_cnn_init(ctx, w.data(), h.norm);
    if (st != SYNIM_OK) return st;
    CnnState *S = ctx->cnn;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpy(S->adam_m, in + P, P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(S->adam_v, in + 2 * P, P, cudaMemcpyHostToDevice);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return ccuda(ctx, e, "cnn_load");
    S->step = h.step;
    return SYNIM_OK;
}

synim_status synim_cnn_forward(synim_ctx *ctx, const uint16_t *x, int64_t n, float *out, void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->cnn) return cfail(ctx, SYNIM_ERR_NOT_TRAINED, "cnn_forward: no network");
    if (n < 0 || (n > 0 && (!x || !out))) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_forward: bad arguments");
    CnnState &S = *ctx->cnn;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    const bf16 *xb = reinterpret_cast<const bf16 *>(x);
    CUtensorMap xmap;
    if (n > 0 && (e = make_input_map(&xmap, xb, n, S.H0, S.C0)) != cudaSuccess)
        return e == cudaErrorInvalidValue ? cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_forward: x must be 16-byte aligned")
                                          : ccuda(ctx, e, "cnn_forward");
    for (long long s0 = 0; s0 < n && e == cudaSuccess; s0 += kBatchCap) {
        const int B = (int)std::min<long long>(kBatchCap, n - s0);
        if ((e = forward(S, xb, xmap, nullptr, s0, B, nullptr, st)) != cudaSuccess) break;
        e = cudaMemcpyAsync(out + 4 * s0, S.out, sizeof(float) * 4 * B, cudaMemcpyDeviceToDevice, st);
    }
    return e == cudaSuccess ? SYNIM_OK : ccuda(ctx, e, "cnn_forward");
}

synim_status synim_cnn_grad(synim_ctx *ctx, const uint16_t *x, const float *target, int64_t n, double *loss_out,
                            float *grad_out, void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->cnn) return cfail(ctx, SYNIM_ERR_NOT_TRAINED, "cnn_grad: no network");
    if (n < 1 || n > kBatchCap || !x || !target)
        return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_grad: 1 <= n <= 256 samples, x and target required");
    CnnState &S = *ctx->cnn;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const bf16 *xb = reinterpret_cast<const bf16 *>(x);
    CUtensorMap xmap;
    cudaError_t e = make_input_map(&xmap, xb, n, S.H0, S.C0);
    if (e == cudaErrorInvalidValue) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_grad: x must be 16-byte aligned");
    if (e == cudaSuccess) e = forward(S, xb, xmap, nullptr, 0, (int)n, target, st);
    if (e == cudaSuccess) e = backward(S, xb, nullptr, 0, (int)n, target, st);
    std::vector<float> l((size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(l.data(), S.loss, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, S.grad, sizeof(float) * S.n_params, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ccuda(ctx, e, "cnn_grad");
    if (synim_status t = check_tc(ctx, S, "cnn_grad")) return t;
    if (loss_out) {
        double s = 0.0;
        for (float v : l) s += v;
        *loss_out = s / (4.0 * (double)n);
    }
    return SYNIM_OK;
}

synim_status synim_cnn_train(synim_ctx *ctx, const double *params, int64_t n, const synim_train_opts *opts,
                             double *loss_out, void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->cnn) return cfail(ctx, SYNIM_ERR_NOT_TRAINED, "cnn_train: call synim_cnn_init first");
    if (!opts || n < 1 || !params || opts->epochs < 1 || opts->batch < 1 || opts->batch > kBatchCap ||
        !(opts->lr > 0.f) || !(opts->noise_rel >= 0.f))
        return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_train: bad n, params or options (batch <= 256)");
    CnnState &S = *ctx->cnn;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long per = (long long)S.H0 * S.H0 * S.C0;
    cudaError_t e = cudaSuccess;
    if (n > S.data_cap) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return ccuda(ctx, e, "cnn_train");
        cudaFree(S.data);
        cudaFree(S.targets);
        cudaFree(S.perm);
        S.data = nullptr;
        S.targets = nullptr;
        S.perm = nullptr;
        S.data_cap = 0;
        e = dmalloc(&S.data, (size_t)n * per);
        if (e == cudaSuccess) e = dmalloc(&S.targets, (size_t)n * 4);
        if (e == cudaSuccess) e = dmalloc(&S.perm, (size_t)n);
        if (e != cudaSuccess) return ccuda(ctx, e, "cnn_train data");
        S.data_cap = n;
        if ((e = make_input_map(&S.map_data, S.data, n, S.H0, S.C0)) != cudaSuccess) return ccuda(ctx, e, "cnn_train data map");
    }
    // training inputs: one noisy bfloat16 response per sample, generated here
    synim_status ss = synim_probe_generate(ctx, params, n, opts->seed, opts->sample0, opts->noise_rel,
                                           reinterpret_cast<uint16_t *>(S.data), cuda_stream);
    if (ss != SYNIM_OK) return ss;
    k_targets<<<blocks_for(n, 128), 128, 0, st>>>(params, n, norm4(S), S.targets);
    S.n_data = n;
    std::vector<int> perm((size_t)n);
    std::mt19937_64 rng(opts->seed ^ 0x5851F42D4C957F2DULL);
    const float b1 = opts->beta1 > 0 ? opts->beta1 : 0.9f, b2 = opts->beta2 > 0 ? opts->beta2 : 0.999f;
    const float eps = opts->eps > 0 ? opts->eps : 1e-8f;
    const long long nb = n / opts->batch;  // full batches only
    if (nb < 1) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_train: fewer samples than one batch");
    std::vector<float> hl((size_t)opts->batch);
    for (int ep = 0; ep < opts->epochs && e == cudaSuccess; ++ep) {
        std::iota(perm.begin(), perm.end(), 0);
        std::shuffle(perm.begin(), perm.end(), rng);
        if ((e = cudaMemcpyAsync(S.perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            break;
        // the host copy of the permutation must outlive the copy
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        double ep_loss = 0.0;
        const float lr = opts->lr * (opts->lr_final > 0.f && opts->epochs > 1
                                         ? std::pow(opts->lr_final / opts->lr, (float)ep / (opts->epochs - 1))
                                         : 1.f);
        for (long long bi = 0; bi < nb && e == cudaSuccess; ++bi) {
            const int B = opts->batch;
            const long long b0 = bi * B;
            // this batch's targets in permuted order
            k_gather_targets<<<blocks_for(B, 128), 128, 0, st>>>(S.targets, S.perm, b0, B, S.tgt);
            if ((e = forward(S, S.data, S.map_data, S.perm, b0, B, S.tgt, st)) != cudaSuccess) break;
            if ((e = backward(S, S.data, S.perm, b0, B, S.tgt, st)) != cudaSuccess) break;
            ++S.step;
            const float c1 = 1.f - std::pow(b1, (float)S.step), c2 = 1.f - std::pow(b2, (float)S.step);
            k_adam_pack<<<blocks_for(S.n_params, 256), 256, 0, st>>>(S.master, S.adam_m, S.adam_v, S.grad,
                                                                    S.n_params, lr, b1, b2, eps, c1, c2, pack_dst(S));
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if (loss_out && (bi % 64 == 0 || bi == nb - 1)) {
                if ((e = cudaMemcpyAsync(S.h_loss, S.loss, sizeof(float) * B, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                    break;
                if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
                double s = 0.0;
                for (int q = 0; q < B; ++q) s += S.h_loss[q];
                ep_loss = s / (4.0 * B);
            }
        }
        if (loss_out) loss_out[ep] = ep_loss;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ccuda(ctx, e, "cnn_train");
    return check_tc(ctx, S, "cnn_train");
}

}  // extern "C"

