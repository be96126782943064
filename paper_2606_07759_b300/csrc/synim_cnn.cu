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
// Kernels (BF16 operands, FP32 accumulation, mma.sync m16n8k16):
//   k_conv<FWD>    implicit GEMM out[m][co] = sum_k im2col(in)[m][k] W[co][k],
//                  m = (sample, oy, ox), k = (ky, kx, ci); + bias, ReLU, BF16;
//   k_conv<DGRAD>  implicit GEMM of the transposed convolution: gradient of
//                  the layer input, masked by its ReLU, BF16;
//   k_wgrad        dW[co][k] = sum_m dz[m][co] im2col(in)[m][k], split over
//                  m into per-CTA partials summed in a fixed order;
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

#include <cuda_bf16.h>

#include "synim_internal.h"
#include "synim_mma.cuh"

namespace synim {

constexpr int CH = 64;               // hidden channels
constexpr int BM = 128, BN = 64, BK = 32, LDA = BK + 8;
constexpr int kConvThreads = 128;
constexpr int kWgThreads = 128;
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
    float *wpart = nullptr, *bpart = nullptr;
    long long wpart_floats = 0;
    float *tgt = nullptr;   // [kBatchCap][4] targets of the current batch
    int *perm = nullptr;    // [n_data]
    bf16 *data = nullptr;   // training inputs [n_data][per_sample]
    float *targets = nullptr;  // [n_data][4]
    long long n_data = 0, data_cap = 0;
    float *h_loss = nullptr;   // pinned [kBatchCap]
};

void cnn_destroy(CnnState *s) {
    if (!s) return;
    void *p[] = {s->master, s->adam_m, s->adam_v, s->grad, s->w1, s->w2, s->w3, s->w2t, s->w3t, s->x,
                 s->a1, s->a2, s->a3, s->dz1, s->dz2, s->dz3, s->out, s->loss, s->dout,
                 s->wpart, s->bpart, s->tgt, s->perm, s->data, s->targets};
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

template <bool DGRAD, int CIN>
__global__ void __launch_bounds__(kConvThreads) k_conv(const ConvArgs a) {
    __shared__ __align__(16) bf16 As[2][BM][LDA];
    __shared__ __align__(16) bf16 Bs[2][BN][LDA];
    constexpr int K = 9 * CIN;
    constexpr int KT = K / BK;
    const int Hr = DGRAD ? a.Hi : a.Ho;  // rows of the GEMM are pixels of this grid
    const long long M = (long long)a.B * Hr * Hr;
    const long long m0 = (long long)blockIdx.x * BM;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // this thread loads GEMM row m0 + tid of A
    const long long mrow = m0 + tid;
    const bool row_ok = mrow < M;
    int rb = 0, ry = 0, rx = 0;
    if (row_ok) {
        rb = (int)(mrow / ((long long)Hr * Hr));
        const int r = (int)(mrow - (long long)rb * Hr * Hr);
        ry = r / Hr;
        rx = r - ry * Hr;
    }
    const bf16 *src_img;
    if (DGRAD) {
        src_img = a.in + (size_t)rb * a.Ho * a.Ho * CH;
    } else {
        const long long sb = a.perm ? (long long)a.perm[a.b0 + rb] : a.b0 + rb;
        src_img = a.in + (size_t)sb * a.Hi * a.Hi * CIN;
    }

    auto load_tile = [&](int kt, int buf) {
        const int k0 = kt * BK;
        const int tap = k0 / CIN, c0 = k0 - tap * CIN;
        const int ky = tap / 3, kx = tap - ky * 3;
        bool ok = row_ok;
        const bf16 *src = a.in;
        if (DGRAD) {
            const int ny = ry + 1 - ky, nx = rx + 1 - kx;
            ok = ok && ny >= 0 && nx >= 0 && (ny % a.stride) == 0 && (nx % a.stride) == 0;
            const int oy = ny / a.stride, ox = nx / a.stride;
            ok = ok && oy < a.Ho && ox < a.Ho;
            if (ok) src = src_img + ((size_t)oy * a.Ho + ox) * CH + c0;
        } else {
            const int iy = ry * a.stride + ky - 1, ix = rx * a.stride + kx - 1;
            ok = ok && iy >= 0 && ix >= 0 && iy < a.Hi && ix < a.Hi;
            if (ok) src = src_img + ((size_t)iy * a.Hi + ix) * CIN + c0;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) cp_async16(&As[buf][tid][c * 8], ok ? src + c * 8 : a.in, ok);
        // B: 64 rows x 4 chunks, two per thread
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = tid * 2 + q, n = idx >> 2, c = idx & 3;
            cp_async16(&Bs[buf][n][c * 8], a.w + (size_t)n * K + k0 + c * 8, true);
        }
        cp_async_commit();
    };

    float acc[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[i][j][t] = 0.f;

    load_tile(0, 0);
    for (int kt = 0; kt < KT; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < KT) {
            load_tile(kt + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = warp * 32 + mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int c = ks + (lane >> 4) * 8;
                ldsm_x4(af[mt], &As[buf][r][c]);
            }
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                uint32_t bfr[4];
                const int n = np * 16 + (lane & 7) + (lane >> 4) * 8;
                const int c = ks + ((lane >> 3) & 1) * 8;
                ldsm_x4(bfr, &Bs[buf][n][c]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(acc[mt][2 * np], af[mt], bfr[0], bfr[1]);
                    mma_bf16(acc[mt][2 * np + 1], af[mt], bfr[2], bfr[3]);
                }
            }
        }
        __syncthreads();
    }

    // epilogue
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long m = m0 + warp * 32 + mt * 16 + g + h * 8;
            if (m >= M) continue;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int n = nt * 8 + 2 * tg;
                float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
                if (DGRAD) {
                    const __nv_bfloat162 am = *reinterpret_cast<const __nv_bfloat162 *>(a.act + m * CH + n);
                    if (!(__bfloat162float(am.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(am.y) > 0.f)) v1 = 0.f;
                } else {
                    v0 = fmaxf(v0 + a.bias[n], 0.f);
                    v1 = fmaxf(v1 + a.bias[n + 1], 0.f);
                }
                *reinterpret_cast<__nv_bfloat162 *>(a.out + m * CH + n) = __floats2bfloat162_rn(v0, v1);
            }
        }
}

// ---------------------------------------------------------------------------
// Weight gradient: part[split][co][k] = sum over this split's rows m of
// dz[m][co] im2col(in)[m][k], k in one tile of BKW columns.
// ---------------------------------------------------------------------------
struct WgArgs {
    const bf16 *dz;      // [B][Ho][Ho][64]
    const bf16 *in;      // layer input
    const int *perm;
    long long b0;
    int B, Hi, Ho, stride;
    long long rows_per_split;
    float *part;         // [splits][64][9 CIN]
};

template <int CIN, int BKW>
__global__ void __launch_bounds__(kWgThreads) k_wgrad(const WgArgs a) {
    constexpr int K = 9 * CIN;
    constexpr int LDZ = CH + 8, LDC = BKW + 8;
    constexpr int NT = BKW / 8;
    __shared__ __align__(16) bf16 Zs[2][32][LDZ];
    __shared__ __align__(16) bf16 Cs[2][32][LDC];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kbase = blockIdx.x * BKW;
    const long long M = (long long)a.B * a.Ho * a.Ho;
    const long long r0 = (long long)blockIdx.y * a.rows_per_split;
    const long long r1 = (r0 + a.rows_per_split < M) ? r0 + a.rows_per_split : M;

    auto load = [&](long long mb, int buf) {
        // dz rows: 32 x 8 chunks
        for (int q = tid; q < 32 * 8; q += kWgThreads) {
            const int r = q >> 3, c = q & 7;
            const long long m = mb + r;
            const bool ok = m < r1;
            cp_async16(&Zs[buf][r][c * 8], ok ? a.dz + m * CH + c * 8 : a.dz, ok);
        }
        // im2col rows: 32 x (BKW / 8) chunks
        for (int q = tid; q < 32 * (BKW / 8); q += kWgThreads) {
            const int r = q / (BKW / 8), c = q - r * (BKW / 8);
            const long long m = mb + r;
            bool ok = m < r1;
            const bf16 *src = a.in;
            if (ok) {
                const int b = (int)(m / ((long long)a.Ho * a.Ho));
                const int rr = (int)(m - (long long)b * a.Ho * a.Ho);
                const int oy = rr / a.Ho, ox = rr - oy * a.Ho;
                const int k = kbase + c * 8;
                const int tap = k / CIN, ci = k - tap * CIN;
                const int ky = tap / 3, kx = tap - ky * 3;
                const int iy = oy * a.stride + ky - 1, ix = ox * a.stride + kx - 1;
                ok = iy >= 0 && ix >= 0 && iy < a.Hi && ix < a.Hi;
                if (ok) {
                    const long long sb = a.perm ? (long long)a.perm[a.b0 + b] : a.b0 + b;
                    src = a.in + (((size_t)sb * a.Hi + iy) * a.Hi + ix) * CIN + ci;
                }
            }
            cp_async16(&Cs[buf][r][c * 8], src, ok);
        }
        cp_async_commit();
    };

    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[j][t] = 0.f;

    if (r0 < r1) {
        load(r0, 0);
        int buf = 0;
        for (long long mb = r0; mb < r1; mb += 32, buf ^= 1) {
            if (mb + 32 < r1) {
                load(mb + 32, buf ^ 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
#pragma unroll
            for (int ks = 0; ks < 32; ks += 16) {
                uint32_t af[4];
                {
                    const int j = lane >> 3;
                    const int r = ks + (lane & 7) + (j >> 1) * 8;
                    const int c = warp * 16 + (j & 1) * 8;
                    ldsm_x4_t(af, &Zs[buf][r][c]);
                }
#pragma unroll
                for (int np = 0; np < NT / 2; ++np) {
                    uint32_t bfr[4];
                    const int r = ks + (lane & 7) + ((lane >> 3) & 1) * 8;
                    const int c = (2 * np + (lane >> 4)) * 8;
                    ldsm_x4_t(bfr, &Cs[buf][r][c]);
                    mma_bf16(acc[2 * np], af, bfr[0], bfr[1]);
                    mma_bf16(acc[2 * np + 1], af, bfr[2], bfr[3]);
                }
            }
            __syncthreads();
        }
    }
    const int g = lane >> 2, tg = lane & 3;
    float *dst = a.part + (size_t)blockIdx.y * CH * K;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n = warp * 16 + g + h * 8;
            const int k = kbase + nt * 8 + 2 * tg;
            dst[(size_t)n * K + k] = acc[nt][2 * h];
            dst[(size_t)n * K + k + 1] = acc[nt][2 * h + 1];
        }
}

// Bias gradient partials: part[split][co] = sum over the split's rows of dz[m][co].
__global__ void k_bias_part(const bf16 *__restrict__ dz, long long M, long long rows_per_split,
                            float *__restrict__ part) {
    __shared__ float sh[4][CH];
    const int co = threadIdx.x & (CH - 1), lane4 = threadIdx.x >> 6;
    const long long r0 = (long long)blockIdx.x * rows_per_split;
    const long long r1 = (r0 + rows_per_split < M) ? r0 + rows_per_split : M;
    float s = 0.f;
    for (long long m = r0 + lane4; m < r1; m += 4) s += __bfloat162float(dz[m * CH + co]);
    sh[lane4][co] = s;
    __syncthreads();
    if (threadIdx.x < CH) part[(size_t)blockIdx.x * CH + co] = sh[0][co] + sh[1][co] + sh[2][co] + sh[3][co];
}

// grad[off + q] = sum over splits (in order) of part[split][q], q < count.
__global__ void k_sum_parts(const float *__restrict__ part, int splits, int count, float *__restrict__ grad) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    float s = 0.f;
    for (int p = 0; p < splits; ++p) s += part[(size_t)p * count + q];
    grad[q] = s;
}

// ---------------------------------------------------------------------------
// Head: dense layer from the flattened last feature map (F = H3 H3 64 values
// per sample, NHWC order) to the 4 outputs; loss; and their backward.
// ---------------------------------------------------------------------------
constexpr int kHeadThreads = 256;

// out[b][j] = bfc[j] + sum_e Wfc[j][e] a3[b][e]; loss[b] = sum_j (out - tgt)^2.
__global__ void __launch_bounds__(kHeadThreads)
k_head_fwd(const bf16 *__restrict__ a3, int F, const float *__restrict__ wfc, const float *__restrict__ bfc,
           const float *__restrict__ tgt, float *__restrict__ out, float *__restrict__ loss) {
    const int b = blockIdx.x;
    const bf16 *x = a3 + (size_t)b * F;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int e = threadIdx.x; e < F; e += blockDim.x) {
        const float v = __bfloat162float(x[e]);
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = fmaf(wfc[(size_t)j * F + e], v, acc[j]);
    }
    __shared__ float sh[kHeadThreads / 32][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float v = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[j] = v;
    }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[threadIdx.x >> 5][j] = acc[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int j = 0; j < 4; ++j) {
            float o = bfc[j];
            for (int w = 0; w < kHeadThreads / 32; ++w) o += sh[w][j];
            out[b * 4 + j] = o;
            if (tgt) {
                const float d = o - tgt[b * 4 + j];
                l = fmaf(d, d, l);
            }
        }
        if (tgt) loss[b] = l;
    }
}

// dout = d(mean loss)/d out.
__global__ void k_head_dout(const float *__restrict__ out, const float *__restrict__ tgt, int B,
                            float *__restrict__ dout) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < 4 * B) dout[q] = 2.f / (4.f * (float)B) * (out[q] - tgt[q]);
}

// gfc[j][e] = sum_b dout[b][j] a3[b][e] (fixed order); thread e = 4 outputs.
__global__ void k_head_wgrad(const bf16 *__restrict__ a3, const float *__restrict__ dout, int B, int F,
                             float *__restrict__ gfc, float *__restrict__ gbfc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < F) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int b = 0; b < B; ++b) {
            const float v = __bfloat162float(a3[(size_t)b * F + e]);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = fmaf(dout[b * 4 + j], v, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) gfc[(size_t)j * F + e] = acc[j];
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        float sb = 0.f;
        for (int b = 0; b < B; ++b) sb += dout[b * 4 + threadIdx.x];
        gbfc[threadIdx.x] = sb;
    }
}

// dz3[b][e] = (a3 > 0) sum_j dout[b][j] Wfc[j][e].
__global__ void k_head_dgrad(const bf16 *__restrict__ a3, const float *__restrict__ dout,
                             const float *__restrict__ wfc, int B, int F, bf16 *__restrict__ dz3) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)B * F) return;
    const int b = (int)(q / F), e = (int)(q - (long long)b * F);
    const float *d = dout + b * 4;
    const float g = d[0] * wfc[e] + d[1] * wfc[(size_t)F + e] + d[2] * wfc[2 * (size_t)F + e] +
                    d[3] * wfc[3 * (size_t)F + e];
    dz3[q] = __float2bfloat16_rn(__bfloat162float(a3[q]) > 0.f ? g : 0.f);
}

// ---------------------------------------------------------------------------
// Parameters: Adam, BF16 copies (and the transposed copies for the input
// gradient), normalisation of targets and outputs.
// ---------------------------------------------------------------------------
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
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

__global__ void k_targets(const double *__restrict__ p, long long n, const double4 center, const double4 range,
                          float *__restrict__ t) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    t[4 * q + 0] = (float)((p[4 * q + 0] - center.x) / range.x);
    t[4 * q + 1] = (float)((p[4 * q + 1] - center.y) / range.y);
    t[4 * q + 2] = (float)((p[4 * q + 2] - center.z) / range.z);
    t[4 * q + 3] = (float)((p[4 * q + 3] - center.w) / range.w);
}

__global__ void k_denorm(const float *__restrict__ o, long long n, const double4 center, const double4 range,
                         double *__restrict__ p) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    p[4 * q + 0] = center.x + range.x * (double)o[4 * q + 0];
    p[4 * q + 1] = center.y + range.y * (double)o[4 * q + 1];
    p[4 * q + 2] = center.z + range.z * (double)o[4 * q + 2];
    p[4 * q + 3] = center.w + range.w * (double)o[4 * q + 3];
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

cudaError_t launch_conv_fwd(const CnnState &S, int layer, const bf16 *in, const int *perm, long long b0, int B,
                            cudaStream_t st) {
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
    const long long M = (long long)B * a.Ho * a.Ho;
    const unsigned nb = blocks_for(M, BM);
    if (layer == 1 && S.C0 == 32) k_conv<false, 32><<<nb, kConvThreads, 0, st>>>(a);
    else if (layer == 1) k_conv<false, 64><<<nb, kConvThreads, 0, st>>>(a);
    else k_conv<false, 64><<<nb, kConvThreads, 0, st>>>(a);
    return cudaGetLastError();
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
    const long long M = (long long)B * a.Hi * a.Hi;
    k_conv<true, 64><<<blocks_for(M, BM), kConvThreads, 0, st>>>(a);
    return cudaGetLastError();
}

int n_splits(long long M) {
    // enough CTAs for a few waves, at least 64 rows each
    return (int)std::max<long long>(1, std::min<long long>(296, M / 64));
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
    long long off_w, off_b;
    if (layer == 1) {
        a.dz = S.dz1; a.Hi = S.H0; a.Ho = S.H1; a.stride = 1; cin = S.C0; off_w = S.off_w1; off_b = S.off_b1;
    } else if (layer == 2) {
        a.dz = S.dz2; a.Hi = S.H1; a.Ho = S.H2; a.stride = 2; cin = CH; off_w = S.off_w2; off_b = S.off_b2;
    } else {
        a.dz = S.dz3; a.Hi = S.H2; a.Ho = S.H3; a.stride = 2; cin = CH; off_w = S.off_w3; off_b = S.off_b3;
    }
    const long long M = (long long)B * a.Ho * a.Ho;
    const int splits = n_splits(M);
    a.rows_per_split = (M + splits - 1) / splits;
    a.rows_per_split = (a.rows_per_split + 31) / 32 * 32;
    const int K = 9 * cin;
    if (cin == 32) {
        dim3 grid(K / 96, splits);
        k_wgrad<32, 96><<<grid, kWgThreads, 0, st>>>(a);
    } else {
        dim3 grid(K / 64, splits);
        k_wgrad<64, 64><<<grid, kWgThreads, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_parts<<<blocks_for(CH * K, 256), 256, 0, st>>>(S.wpart, splits, CH * K, S.grad + off_w);
    k_bias_part<<<splits, 256, 0, st>>>(a.dz, M, a.rows_per_split, S.bpart);
    k_sum_parts<<<1, CH, 0, st>>>(S.bpart, splits, CH, S.grad + off_b);
    return cudaGetLastError();
}

cudaError_t pack_weights(CnnState &S, cudaStream_t st) {
    k_pack_w<<<blocks_for(CH * 9 * S.C0, 256), 256, 0, st>>>(S.master + S.off_w1, S.C0, S.w1, nullptr);
    k_pack_w<<<blocks_for(CH * 9 * CH, 256), 256, 0, st>>>(S.master + S.off_w2, CH, S.w2, S.w2t);
    k_pack_w<<<blocks_for(CH * 9 * CH, 256), 256, 0, st>>>(S.master + S.off_w3, CH, S.w3, S.w3t);
    return cudaGetLastError();
}

// Forward of B <= kBatchCap samples (inputs at in / perm / b0); with targets,
// the per-sample squared errors go to S.loss.
cudaError_t forward(CnnState &S, const bf16 *in, const int *perm, long long b0, int B, const float *tgt,
                    cudaStream_t st) {
    cudaError_t e;
    if ((e = launch_conv_fwd(S, 1, in, perm, b0, B, st)) != cudaSuccess) return e;
    if ((e = launch_conv_fwd(S, 2, S.a1, nullptr, 0, B, st)) != cudaSuccess) return e;
    if ((e = launch_conv_fwd(S, 3, S.a2, nullptr, 0, B, st)) != cudaSuccess) return e;
    k_head_fwd<<<B, kHeadThreads, 0, st>>>(S.a3, S.H3 * S.H3 * CH, S.master + S.off_fc, S.master + S.off_bfc,
                                           tgt, S.out, S.loss);
    return cudaGetLastError();
}

cudaError_t backward(CnnState &S, const bf16 *in, const int *perm, long long b0, int B, const float *tgt,
                     cudaStream_t st) {
    cudaError_t e;
    const int F = S.H3 * S.H3 * CH;
    k_head_dout<<<blocks_for(4 * B, 256), 256, 0, st>>>(S.out, tgt, B, S.dout);
    k_head_wgrad<<<blocks_for(F, 128), 128, 0, st>>>(S.a3, S.dout, B, F, S.grad + S.off_fc, S.grad + S.off_bfc);
    k_head_dgrad<<<blocks_for((long long)B * F, 256), 256, 0, st>>>(S.a3, S.dout, S.master + S.off_fc, B, F, S.dz3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
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
    S.wpart_floats = (long long)splits * CH * 9 * CH;
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
    SYNIM_A(S.tgt, (size_t)kBatchCap * 4);
    SYNIM_A(S.wpart, (size_t)S.wpart_floats);
    SYNIM_A(S.bpart, (size_t)splits * CH);
#undef SYNIM_A
    if (e == cudaSuccess) e = cudaMallocHost(&S.h_loss, sizeof(float) * kBatchCap);
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

double4 d4(const double *v) { return make_double4(v[0], v[1], v[2], v[3]); }

}  // namespace

int cnn_n_params(int C0, int H0) {
    const int H3 = conv_out(conv_out(H0, 2), 2);
    return CH * 9 * C0 + CH + 2 * (CH * 9 * CH + CH) + 4 * H3 * H3 * CH + 4;
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
        if ((e = forward(*S, S->x, nullptr, 0, B, nullptr, st)) != cudaSuccess) break;
        k_denorm<<<blocks_for(B, 128), 128, 0, st>>>(S->out, B, d4(S->center), d4(S->range), params_out + 4 * s0);
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
    if (C % 32 != 0) return cfail(ctx, SYNIM_ERR_SHAPE, "cnn_init: 2 n_modes must be a multiple of 32");
    for (int k = 0; k < 4; ++k)
        if (!(norm[4 + k] > 0.0)) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_init: ranges must be > 0");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cnn_destroy(ctx->cnn);
    ctx->cnn = nullptr;
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

synim_status synim_cnn_forward(synim_ctx *ctx, const uint16_t *x, int64_t n, float *out, void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->cnn) return cfail(ctx, SYNIM_ERR_NOT_TRAINED, "cnn_forward: no network");
    if (n < 0 || (n > 0 && (!x || !out))) return cfail(ctx, SYNIM_ERR_INVALID_ARG, "cnn_forward: bad arguments");
    CnnState &S = *ctx->cnn;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    const bf16 *xb = reinterpret_cast<const bf16 *>(x);
    for (long long s0 = 0; s0 < n && e == cudaSuccess; s0 += kBatchCap) {
        const int B = (int)std::min<long long>(kBatchCap, n - s0);
        if ((e = forward(S, xb, nullptr, s0, B, nullptr, st)) != cudaSuccess) break;
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
    cudaError_t e = forward(S, xb, nullptr, 0, (int)n, target, st);
    if (e == cudaSuccess) e = backward(S, xb, nullptr, 0, (int)n, target, st);
    std::vector<float> l((size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(l.data(), S.loss, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, S.grad, sizeof(float) * S.n_params, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ccuda(ctx, e, "cnn_grad");
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
    }
    // training inputs: one noisy bfloat16 response per sample, generated here
    synim_status ss = synim_probe_generate(ctx, params, n, opts->seed, opts->sample0, opts->noise_rel,
                                           reinterpret_cast<uint16_t *>(S.data), cuda_stream);
    if (ss != SYNIM_OK) return ss;
    k_targets<<<blocks_for(n, 128), 128, 0, st>>>(params, n, d4(S.center), d4(S.range), S.targets);
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
            if ((e = forward(S, S.data, S.perm, b0, B, S.tgt, st)) != cudaSuccess) break;
            if ((e = backward(S, S.data, S.perm, b0, B, S.tgt, st)) != cudaSuccess) break;
            ++S.step;
            const float c1 = 1.f - std::pow(b1, (float)S.step), c2 = 1.f - std::pow(b2, (float)S.step);
            k_adam<<<blocks_for(S.n_params, 256), 256, 0, st>>>(S.master, S.adam_m, S.adam_v, S.grad, S.n_params,
                                                               lr, b1, b2, eps, c1, c2);
            if ((e = pack_weights(S, st)) != cudaSuccess) break;
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
    return e == cudaSuccess ? SYNIM_OK : ccuda(ctx, e, "cnn_train");
}

}  // extern "C"

