// synim_dense.cu -- FP32-accurate dense linear algebra on the 5th-generation
// tensor cores, for the tomographic operators (Sec. 2.4 MMSE reconstructor,
// Sec. 2.5 P_opt = (P_DM^T P_DM + lambda I)^-1 P_DM^T P_Layer).
//
// k_gemm3     C = beta C + alpha op(A) op(B) on tcgen05.mma .kind::tf32 with
//             split operands: x = hi + lo, hi = x with its low 13 mantissa
//             bits cleared (a TF32 value), lo = x - hi (exact in FP32).  C
//             accumulates hi.hi + hi.lo + lo.hi in FP32 TMEM (the lo.lo term
//             is below FP32 rounding), so a product carries ~2^-21 relative
//             error, against 2^-11 for one TF32 pass.  Operand tiles arrive
//             by 4-byte cp.async two chunks ahead of their use (four raw
//             stages) and are split in shared memory.
// k_potrf_diag  unblocked Cholesky of one diagonal block and the inverse of
//             its factor (one CTA, shared memory);
// blocked     right-looking Cholesky S = L L^T whose panel and trailing
//             updates are k_gemm3 calls, and the solve Y <- Y S^-1 as two
//             block triangular sweeps whose updates are k_gemm3 calls.
//
// All matrices are row-major FP32 with a leading dimension.  GEMM operands:
// A(m, k) = A[m lda + k]; B(k, n) = B[n ldb + k] ("N x K", K contiguous) or
// B[k ldb + n] ("K x N", N contiguous); both are staged into shared memory
// as K-major core-matrix tiles, so the tensor core always reads one layout.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "synim_cpasync.cuh"
#include "synim_internal.h"
#include "synim_tc.cuh"

namespace synim {

namespace {

constexpr int kGBM = 128;   // tile rows (TMEM lanes)
constexpr int kGBN = 128;   // tile columns (TMEM columns)
constexpr int kGBK = 32;    // K chunk (floats): 8 core matrices of 16 bytes
constexpr int kGThreads = 128;
constexpr int kTileBytes = kGBM * kGBK * 4;            // one operand tile, one part (16 KB)
constexpr int kRawStages = 4;                          // raw (= hi) operand stages in flight
constexpr int kRawBytes = 2 * kTileBytes;              // A raw, B raw
constexpr int kLoBytes = 2 * kTileBytes;               // A lo, B lo
constexpr int kGemmSmem = kRawStages * kRawBytes + 2 * kLoBytes + 2048;   // + barriers, 1024-byte alignment slack

// Instruction descriptor of tcgen05.mma .kind::tf32: D F32, A and B TF32,
// both K-major, shape M x N.
__host__ __device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                     // D format F32
           | (2u << 7)                   // A format TF32
           | (2u << 10)                  // B format TF32
           | ((uint32_t)(N >> 3) << 17)  // N / 8
           | ((uint32_t)(M >> 4) << 24); // M / 16
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Byte offset of element (r, k) of a 128 x 32 K-major tile: 8-row groups
// 1024 bytes apart (SBO), core matrices along K 128 bytes apart (LBO), rows
// of a core matrix 16 bytes apart.
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

struct GemmArgs {
    const float *A, *B;
    float *C;
    long lda, ldb, ldc;
    int M, N, K;
    float alpha, beta;
    int b_kn;    // 0: B(k, n) = B[n ldb + k]; 1: B(k, n) = B[k ldb + n]
    int lower;   // 1: only tiles that touch the lower triangle (n <= m) of C
    int ksplit;  // K per blockIdx.z (K when gridDim.z = 1)
    long zstride;   // C offset of blockIdx.z's partial (0 when gridDim.z = 1)
};

// Issue the asynchronous 4-byte copies of K chunk k0 of one operand tile
// (128 rows from r0) into its raw tile (zero where out of range), any
// alignment.  kcont (K contiguous in memory): a warp instruction copies 8
// rows x 4 consecutive k, so the shared-memory writes are 32 consecutive
// words of one core-matrix row group; otherwise a warp copies 32 consecutive
// rows at one k (coalesced reads of the contiguous row index).
__device__ __forceinline__ void issue_tile(const float *X, long ld, bool kcont, int rows, int r0, int K, int k0,
                                           uint8_t *raw) {
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (kcont) {
#pragma unroll 8
        for (int it = 0; it < 32; ++it) {
            const int pr = it * 4 + warp;                  // (row group, k group) pair, 0..127
            const int r = (pr >> 3) * 8 + (lane & 7), k = (pr & 7) * 4 + (lane >> 3);
            const bool ok = r0 + r < rows && k0 + k < K;
            const float *src = ok ? X + (long)(r0 + r) * ld + (k0 + k) : X;
            cp_async4(raw + tile_off(r, k), src, ok);
        }
    } else {
#pragma unroll 8
        for (int k = 0; k < kGBK; ++k) {
            const int r = t;
            const bool ok = r0 + r < rows && k0 + k < K;
            const float *src = ok ? X + (long)(k0 + k) * ld + (r0 + r) : X;
            cp_async4(raw + tile_off(r, k), src, ok);
        }
    }
}

// Split both raw tiles of a stage in place: hi = x with its low 13 mantissa
// bits cleared (written back, so that hi + lo = x exactly whatever the tensor
// core does with the bits below TF32), lo = x - hi; 16 bytes per step (raw
// and lo tiles share the layout).
__device__ __forceinline__ void make_lo(uint8_t *raw, uint8_t *lo) {
    float4 *src = reinterpret_cast<float4 *>(raw);
    float4 *dst = reinterpret_cast<float4 *>(lo);
#pragma unroll 4
    for (int q = threadIdx.x; q < kRawBytes / 16; q += kGThreads) {
        const float4 v = src[q];
        float4 h, l;
        h.x = __uint_as_float(__float_as_uint(v.x) & 0xffffe000u);
        h.y = __uint_as_float(__float_as_uint(v.y) & 0xffffe000u);
        h.z = __uint_as_float(__float_as_uint(v.z) & 0xffffe000u);
        h.w = __uint_as_float(__float_as_uint(v.w) & 0xffffe000u);
        l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
        src[q] = h;
        dst[q] = l;
    }
}

// One 128 x 128 tile of C per CTA.  All threads stage K chunks (double
// buffered); thread 0 issues the three split products of each chunk into one
// TMEM accumulator and commits to the chunk's mbarrier; the four warps then
// read their 32 TMEM lanes (rows) back and update C.  Waits are bounded: a
// wait that gives up sets *err and the CTA stops issuing work.
__global__ void __launch_bounds__(kGThreads, 1) k_gemm3(const GemmArgs g, int *err) {
    extern __shared__ __align__(1024) uint8_t gsm[];
    const int bm = blockIdx.y, bn = blockIdx.x;
    const int m0 = bm * kGBM, n0 = bn * kGBN;
    if (g.lower && n0 > m0 + kGBM - 1) return;   // tile wholly above the diagonal
    // split K: this CTA's share [kbeg, kbeg + Kz) of the sum, into its own partial
    const int kbeg = blockIdx.z * g.ksplit, Kz = max(0, min(g.K, kbeg + g.ksplit) - kbeg);
    const float *Ag = g.A + kbeg;
    const float *Bg = g.b_kn ? g.B + (long)kbeg * g.ldb : g.B + kbeg;
    float *Cg = g.C + (long)blockIdx.z * g.zstride;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~uintptr_t(1023));
    uint8_t *lo_base = base + kRawStages * kRawBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(lo_base + 2 * kLoBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc_mbar_init(tc_smem(&bars[0]), 1);
        tc_mbar_init(tc_smem(&bars[1]), 1);
        tc_fence_mbar_init();
    }
    if (warp == 0) tc_alloc(tc_smem(tslot), kGBN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int nch = (Kz + kGBK - 1) / kGBK;
    const uint32_t idesc = idesc_tf32(kGBM, kGBN);
    // chunk c: raw (= hi) tiles in stage c % 4, written by cp.async two chunks
    // ahead; lo tiles in slot c % 2, written once the MMAs of chunk c - 2
    // (which read that slot and raw stage (c + 2) % 4) have completed
    auto issue = [&](int c) {
        uint8_t *raw = base + (c % kRawStages) * kRawBytes;
        issue_tile(Ag, g.lda, true, g.M, m0, Kz, c * kGBK, raw);
        issue_tile(Bg, g.ldb, g.b_kn == 0, g.N, n0, Kz, c * kGBK, raw + kTileBytes);
        cp_async_commit();
    };
    if (nch > 0) issue(0);
    if (nch > 1) issue(1);
    bool ok = true;
    int committed = -1;   // last chunk whose MMAs were committed
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        uint8_t *raw = base + (c % kRawStages) * kRawBytes, *lo = lo_base + b * kLoBytes;
        if (c + 1 < nch) cp_async_wait<1>();   // chunk c landed (chunk c + 1 may be in flight)
        else cp_async_wait<0>();
        if (c >= 2 && !tc_mbar_wait(tc_smem(&bars[b]), ((c - 2) >> 1) & 1)) ok = false;
        if (!__syncthreads_and(ok)) break;
        if (c + 2 < nch) issue(c + 2);
        make_lo(raw, lo);
        tc_fence_proxy_async();   // this thread's cp.async and lo writes -> the tensor core's reads
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t sah = tc_smem(raw), sbh = tc_smem(raw + kTileBytes);
            const uint32_t sal = tc_smem(lo), sbl = tc_smem(lo + kTileBytes);
#pragma unroll
            for (int j = 0; j < kGBK / 8; ++j) {
                const uint32_t o = (uint32_t)j * 256;
                const uint64_t dah = tc_desc(sah + o, 128, 1024), dal = tc_desc(sal + o, 128, 1024);
                const uint64_t dbh = tc_desc(sbh + o, 128, 1024), dbl = tc_desc(sbl + o, 128, 1024);
                tc_mma_tf32(tmem, dah, dbh, idesc, (c | j) != 0);
                tc_mma_tf32(tmem, dah, dbl, idesc, 1);
                tc_mma_tf32(tmem, dal, dbh, idesc, 1);
            }
            tc_commit(tc_smem(&bars[b]));
        }
        committed = c;
    }
    cp_async_wait<0>();   // no copy may still target shared memory when the CTA leaves
    // every issued MMA has completed before TMEM is read or freed (bounded)
    if (committed >= 0 && !tc_mbar_wait(tc_smem(&bars[committed & 1]), (committed >> 1) & 1)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (!ok) {
        if (tid == 0) atomicOr(err, ERR_TIMEOUT);
    } else {
        // epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31.  Each
        // 32-column slice goes through shared memory (the operand stages are
        // free now) so that C is read and written a row at a time by a warp
        // (coalesced), not a column at a time.
        float *stile = reinterpret_cast<float *>(base);   // [128][33]
#pragma unroll 1
        for (int q = 0; q < kGBN / 32; ++q) {
            float v[32];
            tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * 32), v);
            if (nch == 0)
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) stile[(warp * 32 + lane) * 33 + j] = v[j];
            __syncwarp();
            const int n = n0 + q * 32 + lane;
            for (int rr = 0; rr < 32; ++rr) {
                const int r = m0 + warp * 32 + rr;
                if (r < g.M && n < g.N && (!g.lower || n <= r)) {
                    float *cp = Cg + (long)r * g.ldc + n;
                    const float acc = stile[(warp * 32 + rr) * 33 + lane];
                    *cp = g.beta != 0.f ? fmaf(g.alpha, acc, g.beta * *cp) : g.alpha * acc;
                }
            }
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, kGBN);
}

// Unblocked Cholesky of the nb x nb diagonal block at S (row-major, lds):
// L (lower) written back over S, the inverse of L into Linv (nb x nb of a
// kNB x kNB row-major block, zero above the diagonal).  A non-positive pivot
// sets *info = 1 (not positive definite).  One CTA of 512 threads as 16 x 32:
// thread (ty, tx) holds elements (ty + 16 a, tx + 32 b), a < 8, b < 4, of the
// block in registers, so that a step's update is 32 register FMAs per
// thread fed by 12 shared-memory loads of the published column / row.  Both
// loops are right-looking:
//   factor:  for k: L_kk = sqrt(a_kk); L_ik = a_ik / L_kk (i > k);
//            a_ij -= L_ik L_jk (k < j <= i);
//   inverse: X = I; for k: X_k. /= L_kk; X_i. -= L_ik X_k. (i > k), where
//            only X_kc, c <= k, are non-zero.
// The owners of column k (row k of X) publish it unscaled and keep their
// registers unscaled; every thread applies 1 / L_kk as it reads, and the
// final values are scaled on the way out (L_ij = a_ij / L_jj, X_ic =
// x_ic / L_ii), so no register is selected by a run-time index inside the
// step.
constexpr int kNB = 128;
constexpr int kPotrfThreads = 512;

__global__ void __launch_bounds__(kPotrfThreads) k_potrf_diag(float *S, long lds, int nb, float *Linv, int *info) {
    constexpr int ldl = kNB;
    extern __shared__ float a[];   // [kNB][kNB + 1]: L once factored
    constexpr int ld = kNB + 1;
    __shared__ float colk[kNB], pivv[kNB], rpv[kNB];
    __shared__ int bad;
    const int t = threadIdx.x, ty = t >> 5, tx = t & 31;
    float r[8][4];
#pragma unroll
    for (int ai = 0; ai < 8; ++ai)
#pragma unroll
        for (int bi = 0; bi < 4; ++bi) {
            const int i = ty + 16 * ai, j = tx + 32 * bi;
            r[ai][bi] = (i < nb && j <= i) ? S[(long)i * lds + j] : 0.f;
        }
    if (t == 0) bad = 0;
    for (int k = 0; k < nb; ++k) {
        const int bk = k >> 5;
        // the owners of column k publish it (rows k .. nb - 1, unscaled)
        if (tx == (k & 31)) {
#pragma unroll
            for (int bi = 0; bi < 4; ++bi)
                if (bi == bk)
#pragma unroll
                    for (int ai = 0; ai < 8; ++ai) {
                        const int i = ty + 16 * ai;
                        if (i >= k && i < nb) colk[i] = r[ai][bi];
                    }
        }
        __syncthreads();
        const float d = colk[k];
        const float piv = d > 0.f ? sqrtf(d) : 1.f, rp = 1.f / piv;
        if (t == 0) {
            pivv[k] = piv;
            rpv[k] = rp;
            if (!(d > 0.f)) bad = 1;
        }
        float ci[8], cj[4];
#pragma unroll
        for (int ai = 0; ai < 8; ++ai) {
            const int i = ty + 16 * ai;
            ci[ai] = (i > k && i < nb) ? colk[i] * rp : 0.f;
        }
#pragma unroll
        for (int bi = 0; bi < 4; ++bi) {
            const int j = tx + 32 * bi;
            cj[bi] = (j > k && j < nb) ? colk[j] * rp : 0.f;
        }
#pragma unroll
        for (int ai = 0; ai < 8; ++ai)
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) r[ai][bi] = fmaf(-ci[ai], cj[bi], r[ai][bi]);
        __syncthreads();   // column k read by all before column k + 1 is published
    }
    // L to shared memory (and back to S); the upper triangle reads as zero
#pragma unroll
    for (int ai = 0; ai < 8; ++ai)
#pragma unroll
        for (int bi = 0; bi < 4; ++bi) {
            const int i = ty + 16 * ai, j = tx + 32 * bi;
            if (i < nb && j < nb) {
                const float l = i == j ? pivv[j] : (j < i ? r[ai][bi] * rpv[j] : 0.f);
                a[i * ld + j] = l;
                if (j <= i) S[(long)i * lds + j] = l;
            }
        }
    // inverse: X (unscaled rows) in the same registers, row k published through colk
#pragma unroll
    for (int ai = 0; ai < 8; ++ai)
#pragma unroll
        for (int bi = 0; bi < 4; ++bi) r[ai][bi] = (ty + 16 * ai == tx + 32 * bi) ? 1.f : 0.f;
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        const int ak = k >> 4;
        if (ty == (k & 15)) {
#pragma unroll
            for (int ai = 0; ai < 8; ++ai)
                if (ai == ak)
#pragma unroll
                    for (int bi = 0; bi < 4; ++bi) {
                        const int c = tx + 32 * bi;
                        if (c <= k) colk[c] = r[ai][bi];
                    }
        }
        __syncthreads();
        const float rp = rpv[k];
        float li[8], xk[4];
#pragma unroll
        for (int ai = 0; ai < 8; ++ai) {
            const int i = ty + 16 * ai;
            li[ai] = (i > k && i < nb) ? a[i * ld + k] : 0.f;
        }
#pragma unroll
        for (int bi = 0; bi < 4; ++bi) {
            const int c = tx + 32 * bi;
            xk[bi] = c <= k ? colk[c] * rp : 0.f;
        }
#pragma unroll
        for (int ai = 0; ai < 8; ++ai)
#pragma unroll
            for (int bi = 0; bi < 4; ++bi) r[ai][bi] = fmaf(-li[ai], xk[bi], r[ai][bi]);
        __syncthreads();   // row k read by all before row k + 1 is published
    }
#pragma unroll
    for (int ai = 0; ai < 8; ++ai)
#pragma unroll
        for (int bi = 0; bi < 4; ++bi) {
            const int i = ty + 16 * ai, j = tx + 32 * bi;
            if (i < nb && j < nb) Linv[(long)i * ldl + j] = j <= i ? r[ai][bi] * rpv[i] : 0.f;
        }
    if (t == 0 && bad) atomicOr(info, 1);
}

// C[r][n] = alpha sum_z part[z][r][n] + beta C[r][n] (z in order; beta = 0
// reads nothing): the split-K partials of k_gemm3 added.
__global__ void k_splitk_reduce(const float *__restrict__ part, int splits, int M, int N, float alpha, float beta,
                                float *__restrict__ C, long ldc) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)M * N) return;
    const int r = (int)(q / N), n = (int)(q - (long)r * N);
    float acc = 0.f;
    for (int z = 0; z < splits; ++z) acc += part[(long)z * M * N + q];
    float *cp = C + (long)r * ldc + n;
    *cp = beta != 0.f ? fmaf(alpha, acc, beta * *cp) : alpha * acc;
}

// Split-K workspace, one per device, grown on demand.  The dense routines
// are synchronous host calls; cudaFree of a smaller buffer waits for the
// device, so no launch still reads it.
float *splitk_ws(size_t floats) {
    static std::mutex mu;
    static std::map<int, std::pair<float *, size_t>> ws;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    auto &w = ws[dev];
    if (w.second >= floats) return w.first;
    if (w.first) cudaFree(w.first);
    w.first = nullptr;
    w.second = 0;
    if (cudaMalloc(&w.first, floats * sizeof(float)) != cudaSuccess) {
        w.first = nullptr;
        return nullptr;
    }
    w.second = floats;
    return w.first;
}

int device_sms() {
    int dev = 0, n = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

// Copy an r x c block (row-major, leading dimensions) from src to dst.
__global__ void k_copy_block(const float *src, long lds, float *dst, long ldd, int r, int c) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)r * c) return;
    const int i = (int)(q / c), j = (int)(q - (long)i * c);
    dst[(long)i * ldd + j] = src[(long)i * lds + j];
}

}  // namespace

cudaError_t dense_gemm(const float *A, long lda, const float *B, long ldb, bool b_kn, float *C, long ldc, int M,
                       int N, int K, float alpha, float beta, bool lower, int *err, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    // per call: the attribute belongs to the current device
    cudaError_t ea = cudaFuncSetAttribute(k_gemm3, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    if (ea != cudaSuccess) return ea;
    GemmArgs g;
    g.A = A; g.B = B; g.C = C; g.lda = lda; g.ldb = ldb; g.ldc = ldc; g.M = M; g.N = N; g.K = K;
    g.alpha = alpha; g.beta = beta; g.b_kn = b_kn ? 1 : 0; g.lower = lower ? 1 : 0;
    g.ksplit = K;
    g.zstride = 0;
    dim3 grid((unsigned)((N + kGBN - 1) / kGBN), (unsigned)((M + kGBM - 1) / kGBM));
    // Few tiles and a long K (the panel updates of the blocked solves, m x 128
    // with K up to n) would leave most SMs idle: split K over blockIdx.z into
    // partials and add them in order.
    const long tiles = (long)grid.x * grid.y;
    const int n_sm = device_sms();
    int splits = 1;
    if (!lower && K >= 256 && 2 * tiles <= n_sm)
        splits = (int)std::min<long>(std::min<long>((n_sm + tiles - 1) / tiles, K / 128), 16);
    float *ws = nullptr;
    if (splits > 1) {
        const int ks = ((K + splits - 1) / splits + kGBK - 1) / kGBK * kGBK;
        splits = (K + ks - 1) / ks;
        ws = splitk_ws((size_t)splits * M * N);
        if (ws) {
            g.ksplit = ks;
            g.C = ws;
            g.ldc = N;
            g.zstride = (long)M * N;
            g.alpha = 1.f;
            g.beta = 0.f;
            grid.z = (unsigned)splits;
        }
    }
    k_gemm3<<<grid, kGThreads, kGemmSmem, s>>>(g, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || grid.z == 1) return e;
    const long cnt = (long)M * N;
    k_splitk_reduce<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(ws, (int)grid.z, M, N, alpha, beta, C, ldc);
    return cudaGetLastError();
}

// S = L L^T in place (lower triangle), blocked right-looking: for each block
// column j, factor the diagonal block and invert its factor into
// linvs[j] (kNB x kNB), solve the panel below it (L_ij = S_ij L_jj^-T, a GEMM
// into work and a copy back), and update the trailing lower triangle
// (S -= L_panel L_panel^T).  linvs: dense_blocks(n) * kNB * kNB floats; work:
// n * kNB floats.  *info = 1 if S is not positive definite.
cudaError_t dense_potrf(float *S, long lds, int n, float *linvs, float *work, int *info, int *err, cudaStream_t s) {
    const size_t dsm = (size_t)kNB * (kNB + 1) * sizeof(float);
    cudaError_t ea = cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    if (ea != cudaSuccess) return ea;
    float *panel = work;
    for (int j0 = 0; j0 < n; j0 += kNB) {
        const int nb = std::min(kNB, n - j0), rest = n - j0 - nb;
        float *Linv = linvs + (size_t)(j0 / kNB) * kNB * kNB;
        float *Sjj = S + (long)j0 * lds + j0;
        k_potrf_diag<<<1, kPotrfThreads, dsm, s>>>(Sjj, lds, nb, Linv, info);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || rest == 0) {
            if (e != cudaSuccess) return e;
            continue;
        }
        float *Sij = S + (long)(j0 + nb) * lds + j0;
        // panel: rows below, B(k, n) = L_jj^-T(k, n) = Linv[n][k] ("N x K")
        if ((e = dense_gemm(Sij, lds, Linv, kNB, false, panel, nb, rest, nb, nb, 1.f, 0.f, false, err, s)) !=
            cudaSuccess)
            return e;
        const long cnt = (long)rest * nb;
        k_copy_block<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(panel, nb, Sij, lds, rest, nb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // trailing lower triangle: S_rr -= L_r L_r^T
        float *Srr = S + (long)(j0 + nb) * lds + (j0 + nb);
        if ((e = dense_gemm(Sij, lds, Sij, lds, false, Srr, lds, rest, rest, nb, -1.f, 1.f, true, err, s)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

int dense_blocks(int n) { return (n + kNB - 1) / kNB; }

// Y <- Y S^-1 for S = L L^T factored by dense_potrf (Y: m x n, row-major),
// left-looking, so that each block's update is one long-K GEMM: first
// Z = Y L^-T (block columns ascending: Y_j -= Z_{<j} L_{j,<j}^T, then
// Z_j = Y_j Linv_jj^T), then W = Z L^-1 (descending: Z_j -= W_{>j} L_{>j,j},
// then W_j = Z_j Linv_jj).  Every step is a k_gemm3 call; work: m * kNB
// floats.
cudaError_t dense_posolve_right(const float *S, long lds, int n, const float *linvs, float *Y, long ldy, int m,
                                float *work, int *err, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    const int nblk = dense_blocks(n);
    auto copy_back = [&](float *dst, int nb) {
        const long cnt = (long)m * nb;
        k_copy_block<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(work, kNB, dst, ldy, m, nb);
        return cudaGetLastError();
    };
    for (int jb = 0; jb < nblk && e == cudaSuccess; ++jb) {
        const int j0 = jb * kNB, nb = std::min(kNB, n - j0);
        const float *Linv = linvs + (size_t)jb * kNB * kNB;
        float *Yj = Y + j0;
        if (j0 > 0)   // B(k, n) = L[j0 + n][k], k < j0
            e = dense_gemm(Y, ldy, S + (long)j0 * lds, lds, false, Yj, ldy, m, nb, j0, -1.f, 1.f, false, err, s);
        if (e == cudaSuccess) e = dense_gemm(Yj, ldy, Linv, kNB, false, work, kNB, m, nb, nb, 1.f, 0.f, false, err, s);
        if (e == cudaSuccess) e = copy_back(Yj, nb);
    }
    for (int jb = nblk - 1; jb >= 0 && e == cudaSuccess; --jb) {
        const int j0 = jb * kNB, nb = std::min(kNB, n - j0), rest = n - j0 - nb;
        const float *Linv = linvs + (size_t)jb * kNB * kNB;
        float *Yj = Y + j0;
        if (rest > 0)   // B(k, n) = L[j0 + nb + k][j0 + n], k < rest
            e = dense_gemm(Y + j0 + nb, ldy, S + (long)(j0 + nb) * lds + j0, lds, true, Yj, ldy, m, nb, rest, -1.f,
                           1.f, false, err, s);
        if (e == cudaSuccess) e = dense_gemm(Yj, ldy, Linv, kNB, true, work, kNB, m, nb, nb, 1.f, 0.f, false, err, s);
        if (e == cudaSuccess) e = copy_back(Yj, nb);
    }
    return e;
}

}  // namespace synim

// ---------------------------------------------------------------------------
// C ABI (context-free)
// ---------------------------------------------------------------------------
namespace {

synim_status la_fail(synim_status st, const std::string &m) {
    synim::set_global_error(m);
    return st;
}

// Device scratch freed on scope exit (after the caller's synchronisation).
struct LaScratch {
    std::vector<void *> p;
    ~LaScratch() {
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

extern "C" synim_status synim_linalg_gemm(int32_t M, int32_t N, int32_t K, float alpha, const float *A, int64_t lda,
                                          const float *B, int64_t ldb, int32_t b_kn, float beta, float *C,
                                          int64_t ldc, void *cuda_stream) {
    synim::clear_create_error();
    // operand leading dimensions matter only when there is something to read
    if (M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!C || (K > 0 && (!A || !B)))) ||
        (K > 0 && (lda < K || ldb < (b_kn ? N : K))) || ldc < N || (b_kn != 0 && b_kn != 1))
        return la_fail(SYNIM_ERR_INVALID_ARG, "linalg_gemm: invalid sizes or pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    LaScratch sc;
    int *err = nullptr;
    cudaError_t e = sc.alloc(&err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = synim::dense_gemm(A, lda, B, ldb, b_kn != 0, C, ldc, M, N, K, alpha, beta, false, err, st);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return la_fail(SYNIM_ERR_CUDA, std::string("linalg_gemm: ") + cudaGetErrorString(e));
    if (h) return la_fail(SYNIM_ERR_TIMEOUT, "linalg_gemm: a tensor-core wait gave up");
    return SYNIM_OK;
}

extern "C" synim_status synim_linalg_spd_solve(float *S, int32_t n, int64_t lds, float *Y, int32_t m, int64_t ldy,
                                               void *cuda_stream) {
    synim::clear_create_error();
    if (n < 1 || m < 0 || !S || (m > 0 && !Y) || lds < n || ldy < n)
        return la_fail(SYNIM_ERR_INVALID_ARG, "linalg_spd_solve: invalid sizes or pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    LaScratch sc;
    int *flags = nullptr;
    float *linvs = nullptr, *work = nullptr;
    cudaError_t e = sc.alloc(&flags, 2);
    if (e == cudaSuccess) e = sc.alloc(&linvs, (size_t)synim::dense_blocks(n) * 128 * 128);
    if (e == cudaSuccess) e = sc.alloc(&work, (size_t)std::max(n, m) * 128);
    if (e != cudaSuccess) return la_fail(SYNIM_ERR_OOM, "linalg_spd_solve: scratch");
    e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = synim::dense_potrf(S, lds, n, linvs, work, flags, flags + 1, st);
    if (e == cudaSuccess && m > 0) e = synim::dense_posolve_right(S, lds, n, linvs, Y, ldy, m, work, flags + 1, st);
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return la_fail(SYNIM_ERR_CUDA, std::string("linalg_spd_solve: ") + cudaGetErrorString(e));
    if (h[1]) return la_fail(SYNIM_ERR_TIMEOUT, "linalg_spd_solve: a tensor-core wait gave up");
    if (h[0]) return la_fail(SYNIM_ERR_NOT_CONVERGED, "linalg_spd_solve: S is not positive definite");
    return SYNIM_OK;
}
