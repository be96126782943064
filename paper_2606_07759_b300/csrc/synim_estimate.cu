// synim_estimate.cu -- misregistration estimators of one (DM, sensor) pair
// from measured probe responses: a batched Gauss-Newton / Levenberg-
// Marquardt fit whose Jacobian comes from the probe tangents, the learned
// network (synim_cnn.cu), and the network's estimate refined by the fit.
//
// One fit pass over a batch of samples:
//   probe_launch  responses s(p_t) and tangents ds/dp at every sample's trial
//                 point p_t (Sec. 2.1-2.3, forward mode);
//   k_gn_reduce   one CTA per sample: r = y - s, sums r.r, J^T J (10), J^T r,
//                 y.y in FP64 over all map entries (fixed order: per-thread
//                 strided sums, then a fixed tree);
//   k_gn_step     one thread per sample: accept / reject the trial point,
//                 update the damping, solve (J^T J + mu diag) dp = J^T r by
//                 Cholesky in FP64, next trial point.
// The host repeats passes until every sample has stopped.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "synim_internal.h"

namespace synim {

constexpr int kRedThreads = 256;
constexpr int kRed = 16;  // c, H (10), g (4), y.y
// A few samples leave most SMs idle, and the FP64 sums of one sample on one
// SM are slow: each sample's elements are split over `parts` blocks (about
// two blocks per SM in all, at most 128 per sample), whose partial sums a
// second kernel adds in a fixed order.  n * parts <= max(n, kPartRows).
constexpr int kMaxParts = 128;
constexpr int kPartRows = 320;
inline int reduce_parts(long long n, int n_sm) {
    return (int)std::max<long long>(1, std::min<long long>(kMaxParts, std::min<long long>(2LL * n_sm, kPartRows) / n));
}

enum : int { GN_DONE = 1, GN_CONV = 2, GN_FIRST = 4 };

struct GnState {
    double p[4], pt[4], c, yy, H[10], g[4], mu, dnorm;
    int it, flags;
};

struct EstState {
    int max_iter = 30;
    double tol = 1e-4;
    double scale[4] = {8.0, 8.0, 2.0, 0.02};
    long long cap = 0;          // samples the buffers hold
    float *maps = nullptr;      // [cap][per_sample]
    float *dmaps = nullptr;     // [4][cap][per_sample]
    double *red = nullptr;      // [cap][kRed]
    double *red_part = nullptr; // [n * parts][kRed] partial sums (parts blocks per sample)
    double *pt = nullptr;       // [cap][4]
    GnState *st = nullptr;      // [cap]
    int *n_active = nullptr;    // device counter
    int *h_active = nullptr;    // pinned
    double *p0 = nullptr;       // [cap][4] start points / network estimates
    double *h_p = nullptr;      // pinned [cap][4]
    double *h_r = nullptr;      // pinned [cap][2] residual sums
    std::vector<int> iters, conv;  // of the last estimate
    // small-batch path: one captured graph per (method, n, passes)
    struct Graph {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
    };
    std::map<std::tuple<int, long long, int>, Graph> graphs;
    float *ybuf = nullptr;      // [cap][per_sample] the call's probe slopes (the graph's input)
    GnState *h_st = nullptr;    // pinned [cap]
    unsigned long long gen = 0; // synim_ctx::est_gen the graphs were captured at
    cudaStream_t cap_st = nullptr;
};

void est_drop_graphs(EstState *e) {
    for (auto &kv : e->graphs) {
        if (kv.second.x) cudaGraphExecDestroy(kv.second.x);
        if (kv.second.g) cudaGraphDestroy(kv.second.g);
    }
    e->graphs.clear();
}

void est_destroy(EstState *e) {
    if (!e) return;
    est_drop_graphs(e);
    if (e->cap_st) cudaStreamDestroy(e->cap_st);
    cudaFree(e->ybuf);
    cudaFreeHost(e->h_st);
    cudaFree(e->maps);
    cudaFree(e->dmaps);
    cudaFree(e->red);
    cudaFree(e->red_part);
    cudaFree(e->pt);
    cudaFree(e->st);
    cudaFree(e->n_active);
    cudaFree(e->p0);
    cudaFreeHost(e->h_active);
    cudaFreeHost(e->h_p);
    cudaFreeHost(e->h_r);
    delete e;
}

// Index of (a, b), a <= b, in the packed upper triangle of a 4x4 matrix.
__host__ __device__ __forceinline__ int tri(int a, int b) {
    return a * 4 - a * (a - 1) / 2 + (b - a);
}

__global__ void __launch_bounds__(kRedThreads)
k_gn_reduce(const float *__restrict__ y, const float *__restrict__ s, const float *__restrict__ ds,
            long n, int per_sample, int parts, double *__restrict__ red_part) {
    const long q = blockIdx.y;
    const int part = blockIdx.x, seg = (per_sample + parts - 1) / parts;
    const int e0 = part * seg, e1 = min(per_sample, e0 + seg);
    const float *yq = y + q * per_sample, *sq = s + q * per_sample;
    const size_t plane = (size_t)n * per_sample;
    double acc[kRed];
#pragma unroll
    for (int t = 0; t < kRed; ++t) acc[t] = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double yv = yq[e];
        const double r = yv - (double)sq[e];
        double j[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) j[k] = ds[(size_t)k * plane + (size_t)q * per_sample + e];
        acc[0] += r * r;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int b = a; b < 4; ++b) acc[1 + tri(a, b)] += j[a] * j[b];
            acc[11 + a] += j[a] * r;
        }
        acc[15] += yv * yv;
    }
    __shared__ double sh[kRedThreads / 32][kRed];
#pragma unroll
    for (int t = 0; t < kRed; ++t) {
        double v = acc[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[t] = v;
    }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int t = 0; t < kRed; ++t) sh[threadIdx.x >> 5][t] = acc[t];
    __syncthreads();
    if (threadIdx.x < kRed) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
        red_part[(q * parts + part) * kRed + threadIdx.x] = v;
    }
}

// out[q][t] = sum over the parts of sample q of part[q][b][t] (t < nq), one
// warp per quantity, fixed order for a given number of parts.  Rows of out
// are ostride apart, and the last quantity goes to slot last (nq - 1 for a
// packed row; kRed - 1 puts a residual pair (r.r, y.y) where k_gn_step reads
// them).
__global__ void k_red_combine(const double *__restrict__ part, int parts, int nq, double *__restrict__ out,
                              int ostride, int last) {
    const long q = blockIdx.x;
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (t >= nq) return;
    double v = 0.0;
    for (int b = lane; b < parts; b += 32) v += part[(q * parts + b) * nq + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) out[q * ostride + (t == nq - 1 ? last : t)] = v;
}

// Residual sums only: red2[q] = (r.r, y.y) of sample q.
__global__ void __launch_bounds__(kRedThreads)
k_resid_reduce(const float *__restrict__ y, const float *__restrict__ s, int per_sample, int parts,
               double *__restrict__ red2_part) {
    const long q = blockIdx.y;
    const int part = blockIdx.x, seg = (per_sample + parts - 1) / parts;
    const int e0 = part * seg, e1 = min(per_sample, e0 + seg);
    const float *yq = y + q * per_sample, *sq = s + q * per_sample;
    double rr = 0.0, yy = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double yv = yq[e], r = yv - (double)sq[e];
        rr += r * r;
        yy += yv * yv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        yy += __shfl_xor_sync(0xffffffffu, yy, o);
    }
    __shared__ double sh[kRedThreads / 32][2];
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5][0] = rr;
        sh[threadIdx.x >> 5][1] = yy;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
        red2_part[(q * parts + part) * 2 + threadIdx.x] = v;
    }
}

// Cholesky solve of the 4x4 SPD system (packed upper triangle); false if a
// pivot is not positive.
// FP64 division and square root are long instruction sequences on the
// narrow FP64 pipe, so each pivot is inverted once and the rest multiplies.
__device__ bool chol_solve4(const double *Hp, const double *g, double mu, double *x) {
    double L[4][4] = {}, rl[4];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b <= a; ++b) {
            double v = Hp[tri(b, a)];
            if (a == b) v += mu * Hp[tri(a, a)];
            for (int k = 0; k < b; ++k) v -= L[a][k] * L[b][k];
            if (a == b) {
                if (!(v > 0.0)) return false;
                L[a][a] = sqrt(v);
                rl[a] = 1.0 / L[a][a];
            } else {
                L[a][b] = v * rl[b];
            }
        }
    double z[4];
    for (int a = 0; a < 4; ++a) {
        double v = g[a];
        for (int k = 0; k < a; ++k) v -= L[a][k] * z[k];
        z[a] = v * rl[a];
    }
    for (int a = 3; a >= 0; --a) {
        double v = z[a];
        for (int k = a + 1; k < 4; ++k) v -= L[k][a] * x[k];
        x[a] = v * rl[a];
    }
    return true;
}

struct GnCfg {
    int max_iter;
    double tol, rscale[4];   // 1 / scale
};

GnCfg gn_cfg(const EstState *E) {
    GnCfg cfg;
    cfg.max_iter = E->max_iter;
    cfg.tol = E->tol;
    for (int k = 0; k < 4; ++k) cfg.rscale[k] = 1.0 / E->scale[k];
    return cfg;
}

__global__ void k_gn_step(GnState *__restrict__ S, const double *__restrict__ red, long n, const GnCfg cfg,
                          double *__restrict__ pt, int *__restrict__ n_active) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    GnState s = S[q];
    if (!(s.flags & GN_DONE)) {
        const double *R = red + q * kRed;
        const double ct = R[0];
        bool accept = false;
        if (s.flags & GN_FIRST) {
            accept = true;
            s.flags &= ~GN_FIRST;
        } else if (ct <= s.c) {
            accept = true;
            if (s.dnorm < cfg.tol) s.flags |= GN_DONE | GN_CONV;
            s.mu = (s.mu * 0.1 < 1e-7) ? 0.0 : s.mu * 0.1;
        } else {
            s.mu = (s.mu == 0.0) ? 1e-3 : s.mu * 10.0;
            if (s.mu > 1e12) s.flags |= GN_DONE;
        }
        if (accept) {
            for (int k = 0; k < 4; ++k) s.p[k] = s.pt[k];
            s.c = ct;
            s.yy = R[15];
            for (int t = 0; t < 10; ++t) s.H[t] = R[1 + t];
            for (int k = 0; k < 4; ++k) s.g[k] = R[11 + k];
        }
        if (!(s.flags & GN_DONE) && s.it >= cfg.max_iter) s.flags |= GN_DONE;
        if (!(s.flags & GN_DONE)) {
            double dp[4];
            if (chol_solve4(s.H, s.g, s.mu, dp)) {
                double d2 = 0.0;
                for (int k = 0; k < 4; ++k) {
                    s.pt[k] = s.p[k] + dp[k];
                    const double u = dp[k] * cfg.rscale[k];
                    d2 += u * u;
                }
                s.dnorm = sqrt(d2);
            } else {
                // singular normal matrix: stay, damp harder
                for (int k = 0; k < 4; ++k) s.pt[k] = s.p[k];
                s.dnorm = 0.0;
                s.mu = (s.mu == 0.0) ? 1e-3 : s.mu * 10.0;
                s.flags |= GN_FIRST;  // re-evaluate at p, accepted as is
            }
            ++s.it;
            atomicAdd(n_active, 1);
        } else {
            for (int k = 0; k < 4; ++k) s.pt[k] = s.p[k];
        }
    }
    for (int k = 0; k < 4; ++k) pt[4 * q + k] = s.pt[k];
    S[q] = s;
}

__global__ void k_gn_init(GnState *__restrict__ S, const double *__restrict__ p0, long n,
                          double *__restrict__ pt) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    GnState s;
    memset(&s, 0, sizeof(s));
    for (int k = 0; k < 4; ++k) s.p[k] = s.pt[k] = pt[4 * q + k] = p0[4 * q + k];
    s.flags = GN_FIRST;
    S[q] = s;
}

namespace {

synim_status efail(synim_ctx *c, synim_status s, const std::string &m) {
    c->err = m;
    return s;
}

synim_status ecuda(synim_ctx *c, cudaError_t e, const char *what) {
    return efail(c, e == cudaErrorMemoryAllocation ? SYNIM_ERR_OOM : SYNIM_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

EstState *est_get(synim_ctx *c) {
    if (!c->est) c->est = new EstState();
    return c->est;
}

cudaError_t est_reserve(EstState *E, long long cap, int per_sample) {
    if (cap <= E->cap) return cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    est_drop_graphs(E);   // they hold the old buffers' addresses
    cudaFree(E->ybuf);
    cudaFreeHost(E->h_st);
    E->ybuf = nullptr;
    E->h_st = nullptr;
    cudaFree(E->maps);
    cudaFree(E->dmaps);
    cudaFree(E->red);
    cudaFree(E->red_part);
    cudaFree(E->pt);
    cudaFree(E->st);
    cudaFree(E->p0);
    cudaFreeHost(E->h_p);
    cudaFreeHost(E->h_r);
    E->maps = E->dmaps = nullptr;
    E->red = E->red_part = E->pt = E->p0 = E->h_p = E->h_r = nullptr;
    E->st = nullptr;
    E->cap = 0;
    if ((e = cudaMalloc(&E->maps, sizeof(float) * per_sample * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&E->dmaps, sizeof(float) * 4 * per_sample * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&E->red, sizeof(double) * kRed * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&E->red_part, sizeof(double) * kRed * std::max<long long>(cap, kPartRows))) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&E->pt, sizeof(double) * 4 * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&E->st, sizeof(GnState) * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&E->p0, sizeof(double) * 4 * cap)) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&E->h_p, sizeof(double) * 4 * cap)) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&E->h_r, sizeof(double) * 2 * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&E->ybuf, sizeof(float) * per_sample * cap)) != cudaSuccess) return e;
    if ((e = cudaMallocHost(&E->h_st, sizeof(GnState) * cap)) != cudaSuccess) return e;
    if (!E->n_active && (e = cudaMalloc(&E->n_active, sizeof(int))) != cudaSuccess) return e;
    if (!E->h_active && (e = cudaMallocHost(&E->h_active, sizeof(int))) != cudaSuccess) return e;
    E->cap = cap;
    return cudaSuccess;
}

}  // namespace

// One fit pass over n samples whose probe slopes are y: responses (and,
// unless this is the last pass, tangents) at the trial points, the sums,
// the step.  On pass max_iter every sample still running only evaluates its
// trial point and stops, so that pass regenerates values alone and sums
// r.r and y.y (the slots k_gn_step reads then).
cudaError_t fit_pass(synim_ctx *c, const float *y, long long n, int pass, const GnCfg &cfg, cudaStream_t st) {
    EstState *E = c->est;
    const int per_sample = probe_per_sample(c->probe);
    const int parts = reduce_parts(n, c->n_sm);
    const dim3 grid((unsigned)parts, (unsigned)n);
    cudaError_t e;
    if (pass >= cfg.max_iter) {
        if ((e = probe_launch(c, E->pt, n, E->maps, nullptr, nullptr, st)) != cudaSuccess) return e;
        k_resid_reduce<<<grid, kRedThreads, 0, st>>>(y, E->maps, per_sample, parts, E->red_part);
        k_red_combine<<<(unsigned)n, 64, 0, st>>>(E->red_part, parts, 2, E->red, kRed, kRed - 1);
    } else {
        if ((e = probe_launch(c, E->pt, n, E->maps, E->dmaps, nullptr, st)) != cudaSuccess) return e;
        k_gn_reduce<<<grid, kRedThreads, 0, st>>>(y, E->maps, E->dmaps, n, per_sample, parts, E->red_part);
        k_red_combine<<<(unsigned)n, 32 * kRed, 0, st>>>(E->red_part, parts, kRed, E->red, kRed, kRed - 1);
    }
    k_gn_step<<<(unsigned)((n + 63) / 64), 64, 0, st>>>(E->st, E->red, n, cfg, E->pt, E->n_active);
    return cudaGetLastError();
}

// Fit n samples (n <= E->cap) from initial points p0 (device [n][4]); writes
// the estimates to p_out (host [n][4]), the relative residual to res (host
// [n], may be null) and the per-sample statistics.
cudaError_t gn_fit(synim_ctx *c, const float *y, long long n, const double *p0, double *p_out, double *res,
                   int *iters, int *conv, cudaStream_t st) {
    EstState *E = c->est;
    const GnCfg cfg = gn_cfg(E);
    k_gn_init<<<(unsigned)((n + 63) / 64), 64, 0, st>>>(E->st, p0, n, E->pt);
    cudaError_t e = cudaGetLastError();
    for (int pass = 0; pass <= E->max_iter && e == cudaSuccess; ++pass) {
        if ((e = cudaMemsetAsync(E->n_active, 0, sizeof(int), st)) != cudaSuccess) break;
        if ((e = fit_pass(c, y, n, pass, cfg, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(E->h_active, E->n_active, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        if (*E->h_active == 0) break;
    }
    if (e != cudaSuccess) return e;
    std::vector<GnState> hs((size_t)n);
    if ((e = cudaMemcpyAsync(hs.data(), E->st, sizeof(GnState) * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    for (long long q = 0; q < n; ++q) {
        for (int k = 0; k < 4; ++k) p_out[4 * q + k] = hs[q].p[k];
        if (res) res[q] = hs[q].yy > 0 ? std::sqrt(hs[q].c / hs[q].yy) : 0.0;
        if (iters) iters[q] = hs[q].it;
        if (conv) conv[q] = (hs[q].flags & GN_CONV) ? 1 : 0;
    }
    return cudaSuccess;
}

// CNN estimate of n samples (synim_cnn.cu): params_out device [n][4].
cudaError_t cnn_predict_slopes(synim_ctx *c, const float *y, long long n, double *params_out, cudaStream_t st,
                               std::string &why);
bool cnn_ready(const synim_ctx *c, std::string &why);

// Small batches (the latency regime of a single estimate) spend most of
// their time in launch gaps and per-pass host synchronisation.  For the
// network alone (method 1) and the network plus a few fit passes (method 2,
// max_iter <= kGraphMaxIter), the whole device chain of one batch size is
// captured once as a CUDA graph reading the batch from E->ybuf and leaving
// its results in pinned host memory: a call is one device copy, one graph
// launch and one synchronisation.  The fit runs its max_iter + 1 passes
// unconditionally; k_gn_step leaves stopped samples untouched, so the result
// equals the host-driven loop's, which stops once no sample is active.
constexpr long long kGraphMaxN = 32;
constexpr int kGraphMaxIter = 4;

cudaError_t small_chain(synim_ctx *c, int method, bool resid, long long n, cudaStream_t st) {
    EstState *E = c->est;
    std::string why;
    cudaError_t e = cnn_predict_slopes(c, E->ybuf, n, E->p0, st, why);
    if (e != cudaSuccess) return e;
    const int per_sample = probe_per_sample(c->probe);
    const int parts = reduce_parts(n, c->n_sm);
    if (method == 1) {
        if (resid) {
            if ((e = probe_launch(c, E->p0, n, E->maps, nullptr, nullptr, st)) != cudaSuccess) return e;
            k_resid_reduce<<<dim3((unsigned)parts, (unsigned)n), kRedThreads, 0, st>>>(E->ybuf, E->maps, per_sample,
                                                                                       parts, E->red_part);
            k_red_combine<<<(unsigned)n, 64, 0, st>>>(E->red_part, parts, 2, E->red, 2, 1);
            if ((e = cudaMemcpyAsync(E->h_r, E->red, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
                return e;
        }
        if ((e = cudaMemcpyAsync(E->h_p, E->p0, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return e;
        return cudaGetLastError();
    }
    const GnCfg cfg = gn_cfg(E);
    const unsigned nb = (unsigned)((n + 63) / 64);
    k_gn_init<<<nb, 64, 0, st>>>(E->st, E->p0, n, E->pt);
    if ((e = cudaMemsetAsync(E->n_active, 0, sizeof(int), st)) != cudaSuccess) return e;
    for (int pass = 0; pass <= E->max_iter; ++pass)
        if ((e = fit_pass(c, E->ybuf, n, pass, cfg, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(E->h_st, E->st, sizeof(GnState) * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    return cudaGetLastError();
}

// Run one small batch (y: device [n][per_sample]) through its cached graph,
// capturing it on first use.  Results: hout [n][4], res [n] (may be null),
// iters / conv [n] (method 2).
cudaError_t small_estimate(synim_ctx *c, const float *y, long long n, int method, double *hout, double *res,
                           int *iters, int *conv, cudaStream_t st) {
    EstState *E = c->est;
    cudaError_t e;
    if ((e = probe_reserve(c, n)) != cudaSuccess) return e;
    if (E->gen != c->est_gen) {
        est_drop_graphs(E);
        E->gen = c->est_gen;
    }
    if (!E->cap_st && (e = cudaStreamCreateWithFlags(&E->cap_st, cudaStreamNonBlocking)) != cudaSuccess) return e;
    const bool resid = method == 1 && res != nullptr;
    const auto key = std::make_tuple(2 * method + (resid ? 1 : 0), n, method == 2 ? E->max_iter : 0);
    auto it = E->graphs.find(key);
    if (it == E->graphs.end()) {
        EstState::Graph g;
        if ((e = cudaStreamBeginCapture(E->cap_st, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return e;
        cudaError_t e1 = small_chain(c, method, resid, n, E->cap_st);
        e = cudaStreamEndCapture(E->cap_st, &g.g);
        if (e1 != cudaSuccess || e != cudaSuccess) {
            if (g.g) cudaGraphDestroy(g.g);
            cudaGetLastError();
            return e1 != cudaSuccess ? e1 : e;
        }
        if ((e = cudaGraphInstantiate(&g.x, g.g, 0)) != cudaSuccess) {
            cudaGraphDestroy(g.g);
            return e;
        }
        it = E->graphs.emplace(key, g).first;
    }
    const int per_sample = probe_per_sample(c->probe);
    if ((e = cudaMemcpyAsync(E->ybuf, y, sizeof(float) * per_sample * n, cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
        return e;
    if ((e = cudaGraphLaunch(it->second.x, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    for (long long q = 0; q < n; ++q) {
        if (method == 1) {
            for (int k = 0; k < 4; ++k) hout[4 * q + k] = E->h_p[4 * q + k];
            if (res) res[q] = E->h_r[2 * q + 1] > 0 ? std::sqrt(E->h_r[2 * q] / E->h_r[2 * q + 1]) : 0.0;
        } else {
            const GnState &g = E->h_st[q];
            for (int k = 0; k < 4; ++k) hout[4 * q + k] = g.p[k];
            if (res) res[q] = g.yy > 0 ? std::sqrt(g.c / g.yy) : 0.0;
            iters[q] = g.it;
            conv[q] = (g.flags & GN_CONV) ? 1 : 0;
        }
    }
    return cudaSuccess;
}

}  // namespace synim

using namespace synim;

extern "C" {

synim_status synim_gn_config(synim_ctx *ctx, int32_t max_iter, double tol, const double *scale) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (max_iter < 1 || max_iter > 1000 || !(tol > 0.0))
        return efail(ctx, SYNIM_ERR_INVALID_ARG, "gn_config: max_iter in 1..1000, tol > 0");
    EstState *E = est_get(ctx);
    ++ctx->est_gen;   // the captured fits hold the settings by value
    E->max_iter = max_iter;
    E->tol = tol;
    if (scale)
        for (int k = 0; k < 4; ++k) {
            if (!(scale[k] > 0.0)) return efail(ctx, SYNIM_ERR_INVALID_ARG, "gn_config: scale must be > 0");
            E->scale[k] = scale[k];
        }
    return SYNIM_OK;
}

synim_status synim_misreg_estimate(synim_ctx *ctx, const float *probe_slopes, int64_t n, int32_t method,
                                   synim_misreg *inout, double *residual_out, void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->probe) return efail(ctx, SYNIM_ERR_INVALID_ARG, "misreg_estimate: no probes attached");
    if (n < 0 || (n > 0 && (!probe_slopes || !inout)) || method < 0 || method > 2)
        return efail(ctx, SYNIM_ERR_INVALID_ARG, "misreg_estimate: bad n, probe_slopes, inout or method");
    EstState *E = est_get(ctx);
    E->iters.assign((size_t)n, 0);
    E->conv.assign((size_t)n, 0);
    if (n == 0) return SYNIM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int per_sample = probe_per_sample(ctx->probe);
    const long long chunk = std::min<long long>(n, 512);
    cudaError_t e = est_reserve(E, chunk, per_sample);
    if (e != cudaSuccess) return ecuda(ctx, e, "misreg_estimate scratch");
    double *p0 = E->p0;
    std::vector<double> hout((size_t)4 * chunk);
    if (ctx->use_graph && n <= kGraphMaxN && (method == 1 || (method == 2 && E->max_iter <= kGraphMaxIter))) {
        std::string why;
        if (!cnn_ready(ctx, why)) return efail(ctx, SYNIM_ERR_NOT_TRAINED, "misreg_estimate: " + why);
        e = small_estimate(ctx, probe_slopes, n, method, hout.data(), residual_out, E->iters.data(), E->conv.data(),
                           st);
        if (e != cudaSuccess) return ecuda(ctx, e, "misreg_estimate (graph)");
        for (long long q = 0; q < n; ++q) {
            synim_misreg &m = inout[q];
            m.shift_x_px = hout[4 * q + 0];
            m.shift_y_px = hout[4 * q + 1];
            m.rot_deg = hout[4 * q + 2];
            m.mag = hout[4 * q + 3];
        }
        return SYNIM_OK;
    }
    synim_status status = SYNIM_OK;
    for (long long s0 = 0; s0 < n && status == SYNIM_OK; s0 += chunk) {
        const long long b = std::min(chunk, n - s0);
        const float *y = probe_slopes + (size_t)s0 * per_sample;
        if (method == 0) {
            for (long long q = 0; q < b; ++q) {
                const synim_misreg &m = inout[s0 + q];
                E->h_p[4 * q + 0] = m.shift_x_px;
                E->h_p[4 * q + 1] = m.shift_y_px;
                E->h_p[4 * q + 2] = m.rot_deg;
                E->h_p[4 * q + 3] = m.mag;
            }
            e = cudaMemcpyAsync(p0, E->h_p, sizeof(double) * 4 * b, cudaMemcpyHostToDevice, st);
        } else {
            std::string why;
            e = cnn_predict_slopes(ctx, y, b, p0, st, why);
            if (e == cudaErrorNotReady) {
                status = efail(ctx, SYNIM_ERR_NOT_TRAINED, "misreg_estimate: " + why);
                break;
            }
        }
        if (e != cudaSuccess) {
            status = ecuda(ctx, e, "misreg_estimate");
            break;
        }
        if (method == 1) {
            // network only; the estimate is checked by the residual of the regenerated responses
            if (residual_out) {
                e = probe_launch(ctx, p0, b, E->maps, nullptr, nullptr, st);
                if (e == cudaSuccess) {
                    const int parts = reduce_parts(b, ctx->n_sm);
                    k_resid_reduce<<<dim3((unsigned)parts, (unsigned)b), kRedThreads, 0, st>>>(y, E->maps, per_sample,
                                                                                               parts, E->red_part);
                    k_red_combine<<<(unsigned)b, 64, 0, st>>>(E->red_part, parts, 2, E->red, 2, 1);
                    e = cudaMemcpyAsync(E->h_r, E->red, sizeof(double) * 2 * b, cudaMemcpyDeviceToHost, st);
                }
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(E->h_p, p0, sizeof(double) * 4 * b, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) {
                std::memcpy(hout.data(), E->h_p, sizeof(double) * 4 * b);
                if (residual_out)
                    for (long long q = 0; q < b; ++q)
                        residual_out[s0 + q] = E->h_r[2 * q + 1] > 0 ? std::sqrt(E->h_r[2 * q] / E->h_r[2 * q + 1]) : 0.0;
            }
        } else {
            e = gn_fit(ctx, y, b, p0, hout.data(), residual_out ? residual_out + s0 : nullptr,
                       E->iters.data() + s0, E->conv.data() + s0, st);
        }
        if (e != cudaSuccess) {
            status = ecuda(ctx, e, "misreg_estimate fit");
            break;
        }
        for (long long q = 0; q < b; ++q) {
            synim_misreg &m = inout[s0 + q];
            m.shift_x_px = hout[4 * q + 0];
            m.shift_y_px = hout[4 * q + 1];
            m.rot_deg = hout[4 * q + 2];
            m.mag = hout[4 * q + 3];
        }
    }
    return status;
}

synim_status synim_misreg_estimate_stats(const synim_ctx *ctx, int32_t *iters, int32_t *converged) {
    if (!ctx || !ctx->est) return SYNIM_ERR_INVALID_ARG;
    const EstState *E = ctx->est;
    for (size_t q = 0; q < E->iters.size(); ++q) {
        if (iters) iters[q] = E->iters[q];
        if (converged) converged[q] = E->conv[q];
    }
    return SYNIM_OK;
}

}  // extern "C"
