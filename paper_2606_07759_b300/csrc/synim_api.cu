// synim_api.cu -- host side of the C ABI declared in include/synim.h.
//
// create:  uploads the IF cubes, scans supports and packs windows (device),
//          builds the per-sensor subaperture tables and telescoped
//          derivative stencils (host), allocates the per-pair state maps.
// compute: builds the composite affine of every pair (Sec. 2.1, FP64 host),
//          copies the small per-pair block to the device and runs
//          pixel classes -> the IM kernel, replayed from a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "synim.h"
#include "synim_internal.h"
#include "synim_tc.cuh"

using namespace synim;

namespace {

thread_local std::string g_create_error;

}  // namespace


// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

synim_status fail(synim_ctx *c, synim_status s, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

synim_status cuda_fail(synim_ctx *c, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? SYNIM_ERR_OOM : SYNIM_ERR_CUDA, m);
}

// Device allocation charged against the context's memory cap (if any).
cudaError_t capped_malloc(synim_ctx *c, void **q, size_t bytes) {
    if (c->mem_cap > 0 && c->mem_used + bytes > (size_t)c->mem_cap) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(q, bytes);
    if (e == cudaSuccess) c->mem_used += bytes;
    return e;
}

template <typename T>
cudaError_t dev_alloc(synim_ctx *c, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = capped_malloc(c, &q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
        c->dev_allocs.push_back(q);
        *p = static_cast<T *>(q);
    }
    return e;
}

template <typename T>
cudaError_t dev_upload(synim_ctx *c, T **p, const std::vector<T> &v) {
    cudaError_t e = dev_alloc(c, p, v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

namespace synim {

void clear_create_error() { g_create_error.clear(); }
void set_global_error(const std::string &m) { g_create_error = m; }

int ctx_valid_rows(const synim_ctx *ctx, int w, const int **vsub, int *n_sub) {
    *vsub = ctx->geo.wfs[w].vsub;
    *n_sub = ctx->geo.wfs[w].n_sub;
    return ctx->geo.wfs[w].nv;
}

// Composite affine (Sec. 2.1) in closed form:
//   A = c dw / (dd m) R(-td) R(tw) diag(mw)
//   b = cN + R(-td) (c s_w + h theta - s_d) / (dd m) - A (cM, cM)
// with c = 1 - h/H the LGS cone factor, s_d the DM shift in metres, cN and
// cM the DM and sensor grid centres.
bool invert2(const double A[4], double Ai[4]) {
    const double det = A[0] * A[3] - A[1] * A[2];
    if (!(std::fabs(det) > 1e-300) || !std::isfinite(det)) return false;
    Ai[0] = A[3] / det; Ai[1] = -A[1] / det; Ai[2] = -A[2] / det; Ai[3] = A[0] / det;
    return true;
}

void split_pair(DevPair &P) {
    for (int q = 0; q < 4; ++q) {
        P.Ahi[q] = (float)P.A[q];
        P.Alo[q] = (float)(P.A[q] - (double)P.Ahi[q]);
        P.Aif[q] = (float)P.Ai[q];
    }
    for (int q = 0; q < 2; ++q) {
        P.bhi[q] = (float)P.b[q];
        P.blo[q] = (float)(P.b[q] - (double)P.bhi[q]);
    }
}

int largest_divisor_le(int k, int cap) {
    for (int c = std::min(k, cap); c >= 1; --c)
        if (k % c == 0) return c;
    return 1;
}

}  // namespace synim

namespace {

// Host tables of one sensor (Sec. 2.2): lit pixels, valid subapertures,
// scale factors, and the telescoped derivative stencil.
struct WfsTables {
    std::vector<uint8_t> xcode, ycode;
    std::vector<int> irr_pix, irr_sub, irr_sr, vsub, vrow, irrc_row, vidx;
    // the same pupil-edge entries bucketed by 16 x 16 pixel tiles of each
    // subaperture (sensors with k > 32): first entry of each tile, then pixels
    // and weights in tile order
    std::vector<int> tl_start, tl_pix;
    std::vector<int8_t> tl_w;
    int tl_n = 0;
    std::vector<int4> irrc;
    std::vector<int8_t> irr_w;
    std::vector<short> vsj;
    std::vector<float> fac;
    std::vector<uint8_t> P;
    int nv = 0;
};

bool build_wfs_tables(const synim_wfs_desc &d, WfsTables &t, std::string &why) {
    const int M = d.grid_m, n = d.n_sub, k = M / n;
    std::vector<uint8_t> P((size_t)M * M);
    if (d.pupil_mask) {
        for (size_t q = 0; q < P.size(); ++q) P[q] = d.pupil_mask[q] ? 1 : 0;
    } else {
        const double c = (M - 1) * 0.5, ro = M * 0.5, ri = d.obstruction * M * 0.5;
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                // exact squares and sum of half-integer offsets, correctly
                // rounded sqrt: the no-allocation path gives the same mask
                const double dx = (double)j - c, dy = (double)i - c;
                const double r = std::sqrt(dx * dx + dy * dy);
                P[(size_t)i * M + j] = (r <= ro && r >= ri) ? 1 : 0;
            }
    }
    std::vector<int> lit((size_t)n * n, 0);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) lit[(i / k) * n + j / k] += P[(size_t)i * M + j];
    std::vector<uint8_t> V((size_t)n * n);
    t.vsub.clear();
    t.fac.clear();
    t.vrow.assign(n + 1, 0);
    const double dw = d.pupil_diam_m / M;
    for (int si = 0; si < n; ++si) {
        t.vrow[si] = (int)t.vsub.size();
        for (int sj = 0; sj < n; ++sj) {
            const int l = lit[si * n + sj];
            bool ok = d.subap_valid ? d.subap_valid[si * n + sj] != 0 : (2 * l >= k * k);
            if (l == 0) ok = false;
            V[si * n + sj] = ok;
            if (ok) {
                t.vsub.push_back((si << 16) | sj);
                t.fac.push_back((float)(d.slope_scale / (2.0 * dw * l)));
            }
        }
    }
    t.vrow[n] = (int)t.vsub.size();
    t.nv = (int)t.vsub.size();
    t.vidx.assign((size_t)n * n, -1);
    for (int r = 0; r < t.nv; ++r) t.vidx[(t.vsub[r] >> 16) * n + (t.vsub[r] & 0xffff)] = r;
    t.vsj.assign((size_t)t.nv + 4, (short)-1);
    for (int r = 0; r < t.nv; ++r) t.vsj[r] = (short)(t.vsub[r] & 0xffff);
    if (t.nv == 0) {
        why = "sensor has no valid subaperture";
        return false;
    }
    auto Pv = [&](int i, int j) -> int {
        return (i >= 0 && j >= 0 && i < M && j < M) ? P[(size_t)i * M + j] : 0;
    };
    auto Vv = [&](int si, int sj) -> int {
        return (si >= 0 && sj >= 0 && si < n && sj < n) ? V[si * n + sj] : 0;
    };
    // Column pair (b k - 1, b k) at row i.  bit0/bit1: pixel b k - 1 adds
    // +phi to subaperture (si, b-1) / -phi to (si, b); bit2/bit3: pixel b k.
    t.xcode.assign((size_t)(n + 1) * M, 0);
    t.ycode.assign((size_t)(n + 1) * M, 0);
    for (int b = 0; b <= n; ++b) {
        const int c0 = b * k - 1, c1 = b * k;
        for (int i = 0; i < M; ++i) {
            const int si = i / k;
            int code = 0;
            if (c0 >= 0) {
                if (Pv(i, c0 - 1) && Vv(si, b - 1)) code |= 1;
                if (Pv(i, c0 + 1) && Vv(si, b)) code |= 2;
            }
            if (c1 < M) {
                if (Pv(i, c1 - 1) && Vv(si, b - 1)) code |= 4;
                if (Pv(i, c1 + 1) && Vv(si, b)) code |= 8;
            }
            t.xcode[(size_t)b * M + i] = (uint8_t)code;
        }
        for (int j = 0; j < M; ++j) {
            const int sj = j / k;
            int code = 0;
            if (c0 >= 0) {
                if (Pv(c0 - 1, j) && Vv(b - 1, sj)) code |= 1;
                if (Pv(c0 + 1, j) && Vv(b, sj)) code |= 2;
            }
            if (c1 < M) {
                if (Pv(c1 - 1, j) && Vv(b - 1, sj)) code |= 4;
                if (Pv(c1 + 1, j) && Vv(b, sj)) code |= 8;
            }
            t.ycode[(size_t)b * M + j] = (uint8_t)code;
        }
    }
    // Pixels off the boundary lines whose two neighbours (both inside the same
    // subaperture) differ in the pupil mask: weight P(q-e) - P(q+e).
    t.irr_pix.clear();
    t.irr_w.clear();
    t.irr_sub.assign((size_t)n * n + 1, 0);
    t.irr_sr.assign((size_t)n * n * k + 1, 0);
    for (int si = 0; si < n; ++si)
        for (int sj = 0; sj < n; ++sj) {
            t.irr_sub[si * n + sj] = (int)t.irr_pix.size();
            for (int r = 0; r < k; ++r) t.irr_sr[(size_t)(si * n + sj) * k + r] = (int)t.irr_pix.size();
            if (!V[si * n + sj]) continue;
            for (int i = si * k; i < (si + 1) * k; ++i) {
                t.irr_sr[(size_t)(si * n + sj) * k + (i - si * k)] = (int)t.irr_pix.size();
                for (int j = sj * k; j < (sj + 1) * k; ++j) {
                    const int jm = j - sj * k, im = i - si * k;
                    const int wx = (jm != 0 && jm != k - 1) ? Pv(i, j - 1) - Pv(i, j + 1) : 0;
                    const int wy = (im != 0 && im != k - 1) ? Pv(i - 1, j) - Pv(i + 1, j) : 0;
                    if (wx || wy) {
                        t.irr_pix.push_back((i << 16) | j);
                        t.irr_w.push_back((int8_t)wx);
                        t.irr_w.push_back((int8_t)wy);
                    }
                }
            }
        }
    t.irr_sub[(size_t)n * n] = (int)t.irr_pix.size();
    t.irr_sr[(size_t)n * n * k] = (int)t.irr_pix.size();
    // subapertures that have pupil-edge pixels, per subaperture row
    t.irrc.clear();
    t.irrc_row.assign(n + 1, 0);
    for (int si = 0; si < n; ++si) {
        t.irrc_row[si] = (int)t.irrc.size();
        for (int sj = 0; sj < n; ++sj) {
            const int e0 = t.irr_sub[si * n + sj], e1 = t.irr_sub[si * n + sj + 1];
            if (e1 > e0) t.irrc.push_back(make_int4(sj, e0, e1, 0));
        }
    }
    t.irrc_row[n] = (int)t.irrc.size();
    if (k > 32) {
        const int T = (k + 15) / 16;
        t.tl_n = T;
        const size_t nt = (size_t)n * n * T * T;
        std::vector<int> cnt(nt + 1, 0), tile_of(t.irr_pix.size());
        for (size_t e = 0; e < t.irr_pix.size(); ++e) {
            const int i = t.irr_pix[e] >> 16, j = t.irr_pix[e] & 0xffff;
            const int si = i / k, sj = j / k;
            const int q = ((si * n + sj) * T + (i - si * k) / 16) * T + (j - sj * k) / 16;
            tile_of[e] = q;
            ++cnt[q + 1];
        }
        for (size_t q = 0; q < nt; ++q) cnt[q + 1] += cnt[q];
        t.tl_start = cnt;
        t.tl_pix.assign(t.irr_pix.size(), 0);
        t.tl_w.assign(t.irr_w.size(), 0);
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (size_t e = 0; e < t.irr_pix.size(); ++e) {   // stable: entry order within a tile
            const int d = fill[tile_of[e]]++;
            t.tl_pix[d] = t.irr_pix[e];
            t.tl_w[2 * d] = t.irr_w[2 * e];
            t.tl_w[2 * d + 1] = t.irr_w[2 * e + 1];
        }
    }
    t.P = std::move(P);
    return true;
}

// Edge tables of the telescoping-sum engine (Sec. 2.2): per valid row, the
// half-pixel ends of the lit pixel runs inside the subaperture along x
// (pixel rows) and along y (pixel columns), packed as DevTele describes,
// and the scale slope_scale / (dw lit).  A run end on the boundary between
// two valid subapertures whose pixels on both sides are lit is the end of
// one run and the start of the next: it is stored once, as the start event
// of the right (x) or lower (y) subaperture, flagged to credit +phi to the
// neighbour as well.
struct TeleTables {
    std::vector<int> es, ev, vfirst;
    std::vector<float> fac;
};

void build_tele_tables(const synim_wfs_desc &d, const WfsTables &t, TeleTables &e) {
    const int M = d.grid_m, n = d.n_sub, k = M / n;
    const double dw = d.pupil_diam_m / M;
    auto Pv = [&](int i, int j) -> int {
        return (i >= 0 && j >= 0 && i < M && j < M) ? t.P[(size_t)i * M + j] : 0;
    };
    auto Vv = [&](int si, int sj) -> bool {
        return si >= 0 && sj >= 0 && si < n && sj < n && t.vidx[si * n + sj] >= 0;
    };
    auto pack = [](int end, int axis, int credit, int i2, int j2) {
        return (int)(((unsigned)end << 31) | ((unsigned)i2 << 16) | ((unsigned)axis << 15) |
                     ((unsigned)credit << 14) | (unsigned)j2);
    };
    e.es.assign(1, 0);
    e.ev.clear();
    e.fac.clear();
    for (int r = 0; r < t.nv; ++r) {
        const int si = t.vsub[r] >> 16, sj = t.vsub[r] & 0xffff;
        const int i0 = si * k, j0 = sj * k;
        const bool vl = Vv(si, sj - 1), vr = Vv(si, sj + 1), vt = Vv(si - 1, sj), vb = Vv(si + 1, sj);
        int lit = 0;
        for (int i = i0; i < i0 + k; ++i)
            for (int j = j0; j < j0 + k; ++j) {
                if (!Pv(i, j)) continue;
                ++lit;
                const int i2 = 2 * i + 1, j2 = 2 * j + 1;   // doubled, offset by one
                if (j == j0 || !Pv(i, j - 1)) e.ev.push_back(pack(0, 0, j == j0 && vl && Pv(i, j - 1), i2, j2 - 1));
                if (j == j0 + k - 1 || !Pv(i, j + 1))
                    if (!(j == j0 + k - 1 && vr && Pv(i, j + 1))) e.ev.push_back(pack(1, 0, 0, i2, j2 + 1));
                if (i == i0 || !Pv(i - 1, j)) e.ev.push_back(pack(0, 1, i == i0 && vt && Pv(i - 1, j), i2 - 1, j2));
                if (i == i0 + k - 1 || !Pv(i + 1, j))
                    if (!(i == i0 + k - 1 && vb && Pv(i + 1, j))) e.ev.push_back(pack(1, 1, 0, i2 + 1, j2));
            }
        e.es.push_back((int)e.ev.size());
        e.fac.push_back((float)(d.slope_scale / (dw * lit)));
    }
    e.vfirst.assign((size_t)n * (n + 1), 0);
    for (int si = 0; si < n; ++si) {
        int r = t.vrow[si + 1];
        e.vfirst[(size_t)si * (n + 1) + n] = r;
        for (int sj = n - 1; sj >= 0; --sj) {
            if (t.vidx[si * n + sj] >= 0) r = t.vidx[si * n + sj];
            e.vfirst[(size_t)si * (n + 1) + sj] = r;
        }
    }
}

}  // namespace

namespace synim {

// Upper bound of the per-sensor accumulator floats for one pair (any
// actuator), mirroring the kernel's box arithmetic.
long long seg_need(const DmHost &D, const WfsHost &W, const double Ai[4], int NV) {
    const double ej = (D.W + 1.0) * (std::fabs(Ai[0]) + std::fabs(Ai[1])) + 9.0;
    const double ei = (D.W + 1.0) * (std::fabs(Ai[2]) + std::fabs(Ai[3])) + 9.0;
    const long long pj = std::min<long long>((long long)std::ceil(ej), W.M);
    const long long pi = std::min<long long>((long long)std::ceil(ei), W.M);
    const long long nsj = std::min<long long>((pj + 2) / W.k + 2, W.n_sub);
    const long long nsi = std::min<long long>((pi + 2) / W.k + 2, W.n_sub);
    // one box row: nsj + 1 x segments, two rows of nsj y segments, nsj pupil-edge
    // sums, two values each
    (void)nsi;
    return (long long)NV * 2 * (4 * nsj + 1);
}

}  // namespace synim

namespace {
}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
namespace synim {
// One warp; lane 0 waits on an mbarrier that nothing arrives at, through the
// bounded wait of the tensor-core kernels, and raises ERR_TIMEOUT when it
// gives up.
__global__ void k_wait_selftest(long long limit, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc_mbar_init(tc_smem(&bar), 1);
        tc_fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0 && !tc_mbar_wait(tc_smem(&bar), 0, limit)) atomicOr(err, ERR_TIMEOUT);
}
}  // namespace synim

namespace {

// Window origin of each actuator from its support box (x0, x1, y0, y1): the
// box corner clamped so that the W x W window stays on the N x N grid; (0, 0)
// for an empty box.
__global__ void k_org_from_box(const int *__restrict__ box, int n_act, int N, int W, int *__restrict__ org) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_act) return;
    const int *bx = box + 4 * (size_t)a;
    int ox = 0, oy = 0;
    if (bx[1] >= bx[0]) {
        ox = max(0, min(bx[0], N - W));
        oy = max(0, min(bx[2], N - W));
    }
    org[2 * (size_t)a] = ox;
    org[2 * (size_t)a + 1] = oy;
}

}  // namespace

extern "C" {

const char *synim_status_string(synim_status s) {
    switch (s) {
        case SYNIM_OK: return "ok";
        case SYNIM_ERR_INVALID_ARG: return "invalid argument";
        case SYNIM_ERR_SHAPE: return "inconsistent shapes";
        case SYNIM_ERR_OOM: return "device out of memory";
        case SYNIM_ERR_CUDA: return "CUDA runtime error";
        case SYNIM_ERR_TIMEOUT: return "bounded device wait timed out";
        case SYNIM_ERR_NOT_CONVERGED: return "did not converge";
        case SYNIM_ERR_NOT_TRAINED: return "estimator not trained";
    }
    return "unknown status";
}

const char *synim_last_error(const synim_ctx *ctx) {
    if (ctx) return ctx->err.c_str();
    return g_create_error.empty() ? synim::noalloc_last_error() : g_create_error.c_str();
}

void synim_im_destroy(synim_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard guard(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    for (int q = 0; q < NPROF; ++q) {
        if (ctx->prof_a[q]) cudaEventDestroy(ctx->prof_a[q]);
        if (ctx->prof_b[q]) cudaEventDestroy(ctx->prof_b[q]);
    }
    for (int s = 0; s < NSLOT; ++s)
        if (ctx->slot_ev[s]) cudaEventDestroy(ctx->slot_ev[s]);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->prep) cudaStreamDestroy(ctx->prep);
    for (int t = 0; t < 2; ++t) {
        if (ctx->ev_prep[t]) cudaEventDestroy(ctx->ev_prep[t]);
        if (ctx->ev_im[t]) cudaEventDestroy(ctx->ev_im[t]);
    }
    cnn_destroy(ctx->cnn);
    est_destroy(ctx->est);
    probe_destroy(ctx->probe);
    for (void *p : ctx->dev_allocs) cudaFree(p);
    for (void *p : ctx->host_allocs) cudaFreeHost(p);
    delete ctx;
}

synim_status synim_im_create(const synim_dm_desc *dms, int32_t n_dm, const synim_wfs_desc *wfs,
                             int32_t n_wfs, const synim_opts *opts, synim_ctx **out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, SYNIM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!dms || !wfs || n_dm < 1 || n_dm > SYNIM_MAX_DM || n_wfs < 1 || n_wfs > SYNIM_MAX_WFS)
        return fail(nullptr, SYNIM_ERR_INVALID_ARG, "need 1..8 DMs and 1..16 sensors");
    for (int d = 0; d < n_dm; ++d) {
        const synim_dm_desc &D = dms[d];
        if (D.n_act < 1 || D.grid_n < 4 || !(D.pixel_pitch_m > 0) || !(D.altitude_m >= 0) ||
            !D.ifs || !(D.support_eps >= 0) || D.grid_n > 32767)
            return fail(nullptr, SYNIM_ERR_INVALID_ARG, "invalid DM descriptor " + std::to_string(d));
    }
    for (int w = 0; w < n_wfs; ++w) {
        const synim_wfs_desc &W = wfs[w];
        if (W.n_sub < 1 || W.grid_m < 2 || !(W.pupil_diam_m > 0) || !(W.mag[0] != 0) ||
            !(W.mag[1] != 0) || W.grid_m > 32767)
            return fail(nullptr, SYNIM_ERR_INVALID_ARG, "invalid sensor descriptor " + std::to_string(w));
        if (W.grid_m % W.n_sub != 0 || W.grid_m / W.n_sub < 2)
            return fail(nullptr, SYNIM_ERR_SHAPE,
                        "sensor " + std::to_string(w) + ": grid_m must be k * n_sub with k >= 2");
    }
    synim_ctx *c = new synim_ctx();
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    c->n_dm = n_dm;
    c->n_wfs = n_wfs;
    if (opts) {
        if (opts->threads_per_cta > 0) c->threads = opts->threads_per_cta;
        c->ctas_per_sm = std::max(0, opts->ctas_per_sm);
        c->use_graph = opts->use_graph != 0;
        c->autotune = opts->autotune != 0;
        c->profile = opts->profile != 0;
        c->mem_cap = std::max<int64_t>(0, opts->device_mem_cap);
        c->slope_engine = opts->slope_engine;
    }
    if (c->slope_engine != SYNIM_ENGINE_NUMERICAL && c->slope_engine != SYNIM_ENGINE_TELESCOPING) {
        delete c;
        return fail(nullptr, SYNIM_ERR_INVALID_ARG, "slope_engine must be 0 (numerical) or 1 (telescoping)");
    }
    for (int w = 0; w < n_wfs && c->slope_engine == SYNIM_ENGINE_TELESCOPING; ++w)
        if (wfs[w].grid_m > 8191) {
            delete c;
            return fail(nullptr, SYNIM_ERR_SHAPE, "the telescoping engine takes sensor grids up to 8191 pixels");
        }
    if (c->threads % 32 != 0 || c->threads < 64 || c->threads > 256) {
        delete c;
        return fail(nullptr, SYNIM_ERR_INVALID_ARG, "threads_per_cta must be a multiple of 32 in 64..256");
    }
    auto bail = [&](synim_status s) {
        std::string m = c->err;
        synim_im_destroy(c);
        g_create_error = m;
        return s;
    };
    // ---- DMs, part 1: the host cubes start their way to the device ----
    // Two staging buffers in turn: the copy of cube d + 1 (copy stream) runs
    // while cube d is scanned and packed (work stream), and both overlap the
    // host-side sensor tables below.  A buffer is refilled once the packing
    // that read it has finished.
    struct Upload {
        cudaStream_t cs = nullptr, ks = nullptr;
        cudaEvent_t copied[SYNIM_MAX_DM] = {}, packed[SYNIM_MAX_DM] = {};
        float *buf[2] = {nullptr, nullptr};
        int *box = nullptr;   // support boxes of one DM (the largest n_act)
        size_t bytes = 0;
        // (a failed create has destroyed the context by the time this runs:
        // the successful path returns the buffers' bytes to its count itself)
        ~Upload() {
            if (cs) cudaStreamSynchronize(cs);
            if (ks) cudaStreamSynchronize(ks);
            for (int q = 0; q < 2; ++q)
                if (buf[q]) cudaFree(buf[q]);
            if (box) cudaFree(box);
            for (int d = 0; d < SYNIM_MAX_DM; ++d) {
                if (copied[d]) cudaEventDestroy(copied[d]);
                if (packed[d]) cudaEventDestroy(packed[d]);
            }
            if (cs) cudaStreamDestroy(cs);
            if (ks) cudaStreamDestroy(ks);
        }
    } up;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&up.cs, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&up.ks, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(c, e, "upload streams"));
    int n_host = 0;
    for (int d = 0; d < n_dm; ++d) {
        if ((e = cudaEventCreateWithFlags(&up.copied[d], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&up.packed[d], cudaEventDisableTiming)) != cudaSuccess)
            return bail(cuda_fail(c, e, "upload events"));
        if (!dms[d].ifs_on_device) {
            up.bytes = std::max(up.bytes, (size_t)dms[d].grid_n * dms[d].grid_n * dms[d].n_act * sizeof(float));
            ++n_host;
        }
    }
    for (int q = 0; q < std::min(n_host, 2); ++q)
        if ((e = capped_malloc(c, reinterpret_cast<void **>(&up.buf[q]), up.bytes)) != cudaSuccess)
            return bail(cuda_fail(c, e, "cube staging"));
    // Nothing below waits on the copy stream until the last cube is packed:
    // the masks go up before the cubes, the support boxes stay in one scratch
    // (no cudaFree, which would wait for the copies), the window origins are
    // computed on the device, and the sensor tables are uploaded afterwards.
    uint8_t *d_masks[SYNIM_MAX_DM] = {};
    int max_act = 1;
    for (int d = 0; d < n_dm; ++d) {
        max_act = std::max(max_act, dms[d].n_act);
        if (!dms[d].mask) continue;
        const size_t NN = (size_t)dms[d].grid_n * dms[d].grid_n;
        std::vector<uint8_t> m(NN);
        for (size_t q = 0; q < NN; ++q) m[q] = dms[d].mask[q] ? 1 : 0;
        if ((e = dev_upload(c, &d_masks[d], m)) != cudaSuccess) return bail(cuda_fail(c, e, "mask upload"));
    }
    if ((e = cudaMalloc(&up.box, (4 * (size_t)max_act + 1) * sizeof(int))) != cudaSuccess)
        return bail(cuda_fail(c, e, "support boxes"));
    // host cube d goes to staging buffer slot[d] (host cubes alternate between the two)
    int slot[SYNIM_MAX_DM];
    for (int d = 0, h = 0; d < n_dm; ++d) slot[d] = dms[d].ifs_on_device ? -1 : (h++ & 1);
    auto issue_copy = [&](int d) -> cudaError_t {
        const size_t nb = (size_t)dms[d].grid_n * dms[d].grid_n * dms[d].n_act * sizeof(float);
        cudaError_t ec = cudaMemcpyAsync(up.buf[slot[d]], dms[d].ifs, nb, cudaMemcpyHostToDevice, up.cs);
        if (ec == cudaSuccess) ec = cudaEventRecord(up.copied[d], up.cs);
        return ec;
    };
    // the first two host cubes now; each later one after the packing of the cube two before it
    int next_copy = 0, issued = 0;
    for (; next_copy < n_dm && issued < 2; ++next_copy)
        if (slot[next_copy] >= 0) {
            if ((e = issue_copy(next_copy)) != cudaSuccess) return bail(cuda_fail(c, e, "cube upload"));
            ++issued;
        }
    // ---- sensors: tables, built on the host while the cubes travel (uploaded after the DMs) ----
    std::vector<WfsTables> tabs((size_t)n_wfs);
    for (int w = 0; w < n_wfs; ++w) {
        const synim_wfs_desc &Wd = wfs[w];
        WfsHost &H = c->wh[w];
        H.n_sub = Wd.n_sub; H.M = Wd.grid_m; H.k = Wd.grid_m / Wd.n_sub;
        H.CH = largest_divisor_le(H.k, 32);
        H.D = Wd.pupil_diam_m; H.H = Wd.src_height_m;
        H.th[0] = Wd.field_rad[0]; H.th[1] = Wd.field_rad[1];
        H.rot = Wd.rot_deg; H.mag[0] = Wd.mag[0]; H.mag[1] = Wd.mag[1];
        H.shift[0] = Wd.shift_m[0]; H.shift[1] = Wd.shift_m[1]; H.scale = Wd.slope_scale;
        WfsTables &T = tabs[w];
        std::string why;
        if (!build_wfs_tables(Wd, T, why)) {
            fail(c, SYNIM_ERR_SHAPE, "sensor " + std::to_string(w) + ": " + why);
            return bail(SYNIM_ERR_SHAPE);
        }
        H.nv = T.nv;
        c->pupil[w] = T.P;
        c->vidx_h[w] = T.vidx;
        c->max_mm = std::max(c->max_mm, H.M * H.M);
        c->max_lines = std::max(c->max_lines, H.M * (H.n_sub + 1));
    }
    // (a DM gets the 9-pixel-bordered windows when some sensor has subapertures
    // small enough for the weight boxes; the DM loop below builds them)
    bool want_k_any = false;
    for (int w = 0; w < n_wfs; ++w)
        want_k_any |= c->wh[w].k <= KF_MAX_K && (long)c->wh[w].n_sub * (c->wh[w].n_sub + 1) <= KPS;
    // ---- per-pair state maps, parameter blocks, counters ----
    long long tot = 0, tot_lines = 0;
    for (int d = 0; d < n_dm; ++d)
        for (int w = 0; w < n_wfs; ++w) {
            c->pst_off[d * n_wfs + w] = tot;
            tot += (long long)c->wh[w].M * c->wh[w].M;
            c->line_off[d * n_wfs + w] = tot_lines;
            tot_lines += 2LL * c->wh[w].M * (c->wh[w].n_sub + 1);
        }
    const int np = n_dm * n_wfs;
    // two table sets (alternate calls); the telescoping engine takes set 0 only
    const int n_sets = c->slope_engine == SYNIM_ENGINE_TELESCOPING ? 1 : 2;
    e = cudaSuccess;
    // one allocation per set, carved at 256-byte boundaries (a hundred-odd
    // separate buffers cost milliseconds to allocate and free)
    auto carve = [](size_t &off, size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) / 256 * 256;
        return at;
    };
    for (int t = 0; t < n_sets && e == cudaSuccess; ++t) {
        size_t off = 0;
        const size_t o_pst = carve(off, (size_t)tot), o_lines = carve(off, (size_t)tot_lines);
        const size_t o_pairs = carve(off, sizeof(DevPair) * np);
        size_t o_k[SYNIM_MAX_PAIRS][3] = {};
        bool has_k[SYNIM_MAX_PAIRS] = {};
        for (int d = 0; d < n_dm; ++d)
            for (int w = 0; w < n_wfs; ++w) {
                const WfsHost &H = c->wh[w];
                if (H.k > KF_MAX_K || (long)H.n_sub * (H.n_sub + 1) > KPS || !want_k_any) continue;
                const int p = d * n_wfs + w;
                has_k[p] = true;
                o_k[p][0] = carve(off, sizeof(int) * 4 * KPS);
                o_k[p][1] = carve(off, sizeof(float) * 2 * KNC * KTAPS * KPS);
                o_k[p][2] = carve(off, sizeof(float) * 2 * KNC * KTAPS * KPS);
            }
        uint8_t *blk = nullptr;
        if ((e = dev_alloc(c, &blk, off)) != cudaSuccess) break;
        c->d_pst[t] = blk + o_pst;
        c->d_lines[t] = blk + o_lines;
        c->d_pairs[t] = reinterpret_cast<DevPair *>(blk + o_pairs);
        for (int p = 0; p < np; ++p)
            if (has_k[p]) {
                c->k_org[t][p] = reinterpret_cast<int *>(blk + o_k[p][0]);
                c->k_w[t][p] = reinterpret_cast<float *>(blk + o_k[p][1]);
                c->k_wb[t][p] = reinterpret_cast<float *>(blk + o_k[p][2]);
            }
    }
    if (e == cudaSuccess) e = dev_alloc(c, &c->d_err, 1);
    if (e == cudaSuccess) e = dev_alloc(c, &c->d_gp, (size_t)np * 4);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "context buffers"));
    for (int s = 0; s < NSLOT; ++s) {
        void *h = nullptr;
        if ((e = cudaMallocHost(&h, sizeof(DevPair) * np)) != cudaSuccess)
            return bail(cuda_fail(c, e, "pinned parameter block"));
        c->host_allocs.push_back(h);
        c->h_pairs[s] = static_cast<DevPair *>(h);
        std::memset(h, 0, sizeof(DevPair) * np);
        if ((e = cudaEventCreateWithFlags(&c->slot_ev[s], cudaEventDisableTiming)) != cudaSuccess)
            return bail(cuda_fail(c, e, "event"));
    }
    {
        void *h = nullptr;
        if ((e = cudaMallocHost(&h, sizeof(int))) != cudaSuccess) return bail(cuda_fail(c, e, "pinned flag"));
        c->host_allocs.push_back(h);
        c->h_err = static_cast<int *>(h);
    }
    if ((e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(c, e, "capture stream"));
    if ((e = cudaStreamCreateWithFlags(&c->prep, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(c, e, "prep stream"));
    for (int t = 0; t < 2; ++t)
        if ((e = cudaEventCreateWithFlags(&c->ev_prep[t], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c->ev_im[t], cudaEventDisableTiming)) != cudaSuccess)
            return bail(cuda_fail(c, e, "event"));
    if (c->profile)
        for (int q = 0; q < NPROF; ++q)
            if ((e = cudaEventCreate(&c->prof_a[q])) != cudaSuccess ||
                (e = cudaEventCreate(&c->prof_b[q])) != cudaSuccess)
                return bail(cuda_fail(c, e, "profiling events"));
    // ---- DMs, part 2: support scan + window packing ----
    for (int d = 0; d < n_dm; ++d) {
        const synim_dm_desc &Dd = dms[d];
        DmHost &H = c->dmh[d];
        H.n_act = Dd.n_act; H.N = Dd.grid_n; H.dd = Dd.pixel_pitch_m; H.h = Dd.altitude_m;
        const float *cube = Dd.ifs;
        if (slot[d] >= 0) {
            if ((e = cudaStreamWaitEvent(up.ks, up.copied[d], 0)) != cudaSuccess)
                return bail(cuda_fail(c, e, "cube upload"));
            cube = up.buf[slot[d]];
        }
        int *d_box = up.box;
        std::vector<int> box(4 * (size_t)H.n_act);
        e = launch_support(cube, H.n_act, H.N, Dd.support_eps, d_box, up.ks);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(box.data(), d_box, box.size() * sizeof(int), cudaMemcpyDeviceToHost, up.ks);
        if (e == cudaSuccess) e = cudaStreamSynchronize(up.ks);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "support scan"));
        int W = 1;
        for (int a = 0; a < H.n_act; ++a) {
            const int *bx = &box[4 * (size_t)a];
            if (bx[1] < bx[0]) continue;
            W = std::max(W, std::max(bx[1] - bx[0] + 1, bx[3] - bx[2] + 1));
        }
        W = std::min(W, H.N);
        int Wp = W + 2;
        if ((Wp & 1) == 0) ++Wp;  // odd pitch: rows of the window fall in distinct banks
        const int stride = (Wp * Wp + 3) / 4 * 4;
        H.W = W; H.Wp = Wp;
        DevDM &G = c->geo.dm[d];
        int *d_org = nullptr;
        float *d_win = nullptr;
        e = dev_alloc(c, &d_org, 2 * (size_t)H.n_act);
        if (e == cudaSuccess) {
            k_org_from_box<<<(H.n_act + 255) / 256, 256, 0, up.ks>>>(d_box, H.n_act, H.N, W, d_org);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = dev_alloc(c, &d_win, (size_t)H.n_act * stride);
        if (e == cudaSuccess) e = launch_pack(cube, H.n_act, H.N, d_org, W, Wp, stride, d_win, up.ks);
        // the same windows with a KPAD-pixel zero border for the boundary-segment
        // weight boxes, when a sensor has subapertures small enough for them
        bool want_k = false;
        for (int w = 0; w < n_wfs; ++w)
            want_k |= c->wh[w].k <= KF_MAX_K && (long)c->wh[w].n_sub * (c->wh[w].n_sub + 1) <= KPS;
        float *d_wink = nullptr;
        int WpK = 0, strideK = 0;
        if (want_k && e == cudaSuccess) {
            WpK = W + 2 * KPAD;
            if ((WpK & 1) == 0) ++WpK;
            strideK = (WpK * WpK + 3) / 4 * 4;
            e = dev_alloc(c, &d_wink, (size_t)H.n_act * strideK);
            if (e == cudaSuccess)
                e = launch_pack(cube, H.n_act, H.N, d_org, W, WpK, strideK, d_wink, up.ks, KPAD);
        }
        if (e == cudaSuccess) e = cudaEventRecord(up.packed[d], up.ks);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "window packing"));
        // the staging buffer of cube d takes the next host cube once the packing has read it
        if (slot[d] >= 0) {
            while (next_copy < n_dm && slot[next_copy] < 0) ++next_copy;
            if (next_copy < n_dm) {
                if ((e = cudaStreamWaitEvent(up.cs, up.packed[d], 0)) != cudaSuccess ||
                    (e = issue_copy(next_copy)) != cudaSuccess)
                    return bail(cuda_fail(c, e, "cube upload"));
                ++next_copy;
            }
        }
        uint8_t *d_mask = d_masks[d];
        uint8_t *d_mcls = nullptr;
        e = dev_alloc(c, &d_mcls, (size_t)(H.N + 1) * (H.N + 1));
        if (e == cudaSuccess) e = launch_mcls(d_mask, H.N, d_mcls, up.ks);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "mask interior map"));
        G.win = d_win; G.org = d_org; G.mask = d_mask; G.mcls = d_mcls;
        G.n_act = H.n_act; G.N = H.N; G.W = W; G.Wp = Wp; G.win_stride = stride;
        G.winK = d_wink; G.WpK = WpK; G.strideK = strideK;
    }
    if ((e = cudaStreamSynchronize(up.ks)) != cudaSuccess) return bail(cuda_fail(c, e, "window packing"));
    for (int q = 0; q < 2; ++q)
        if (up.buf[q]) {
            cudaFree(up.buf[q]);
            up.buf[q] = nullptr;
            c->mem_used -= up.bytes;
        }
    // ---- sensors: device tables (the copy engine is idle now) ----
    for (int w = 0; w < n_wfs; ++w) {
        const synim_wfs_desc &Wd = wfs[w];
        const WfsHost &H = c->wh[w];
        const WfsTables &T = tabs[w];
        DevWFS &G = c->geo.wfs[w];
        uint8_t *xc, *yc;
        int *ip, *is, *vs, *vr;
        int8_t *iw;
        float *fa;
        e = dev_upload(c, &xc, T.xcode);
        if (e == cudaSuccess) e = dev_upload(c, &yc, T.ycode);
        if (e == cudaSuccess) e = dev_upload(c, &ip, T.irr_pix);
        if (e == cudaSuccess) e = dev_upload(c, &iw, T.irr_w);
        if (e == cudaSuccess) e = dev_upload(c, &is, T.irr_sub);
        if (e == cudaSuccess) e = dev_upload(c, &fa, T.fac);
        if (e == cudaSuccess) e = dev_upload(c, &vs, T.vsub);
        if (e == cudaSuccess) e = dev_upload(c, &vr, T.vrow);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "sensor tables"));
        int4 *cd = nullptr;
        int *cr = nullptr, *sr = nullptr;
        short *vj = nullptr;
        int *vx = nullptr;
        if (e == cudaSuccess) e = dev_upload(c, &vj, T.vsj);
        if (e == cudaSuccess) e = dev_upload(c, &vx, T.vidx);
        if (e == cudaSuccess) e = dev_upload(c, &sr, T.irr_sr);
        if (e == cudaSuccess) e = dev_upload(c, &cd, T.irrc);
        if (e == cudaSuccess) e = dev_upload(c, &cr, T.irrc_row);
        int *ts = nullptr, *tp = nullptr;
        int8_t *tw = nullptr;
        if (T.tl_n > 0) {
            if (e == cudaSuccess) e = dev_upload(c, &ts, T.tl_start);
            if (e == cudaSuccess && !T.tl_pix.empty()) e = dev_upload(c, &tp, T.tl_pix);
            if (e == cudaSuccess && !T.tl_w.empty()) e = dev_upload(c, &tw, T.tl_w);
        }
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "sensor tables"));
        G.tl_start = ts; G.tl_pix = tp; G.tl_w = tw; G.tl_n = tp ? T.tl_n : 0;
        G.irrc = cd; G.irrc_row = cr; G.irr_sr = sr; G.vsj = vj; G.vidx = vx;
        G.xcode = xc; G.ycode = yc; G.irr_pix = ip; G.irr_w = iw; G.irr_sub = is;
        G.fac = fa; G.vsub = vs; G.vrow = vr;
        G.n_sub = H.n_sub; G.M = H.M; G.k = H.k; G.nv = H.nv; G.CH = H.CH;
        G.n_irr = (int)T.irr_pix.size();
        if (c->slope_engine == SYNIM_ENGINE_TELESCOPING) {
            TeleTables TT;
            build_tele_tables(Wd, T, TT);
            DevTele &DT = c->tele.w[w];
            int *es = nullptr, *ev = nullptr, *vf = nullptr;
            float *tf = nullptr;
            e = dev_upload(c, &es, TT.es);
            if (e == cudaSuccess) e = dev_upload(c, &ev, TT.ev);
            if (e == cudaSuccess) e = dev_upload(c, &vf, TT.vfirst);
            if (e == cudaSuccess) e = dev_upload(c, &tf, TT.fac);
            if (e != cudaSuccess) return bail(cuda_fail(c, e, "telescoping edge tables"));
            DT.es = es; DT.ev = ev; DT.fac = tf; DT.vfirst = vf;
            DT.n_ev = (int)TT.ev.size();
            // a full subaperture has 4 k events: at most sixteen per lane
            int L = 1;
            while (L < 32 && 4 * L < H.k) L *= 2;
            DT.lanes = L;
        }
    }
    tabs.clear();
    // processing order: largest windows first (longest items scheduled early)
    std::vector<int> order(n_dm);
    for (int d = 0; d < n_dm; ++d) order[d] = d;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return c->geo.dm[x].win_stride > c->geo.dm[y].win_stride;
    });
    int acc = 0;
    for (int q = 0; q < n_dm; ++q) {
        c->geo.order_dm[q] = order[q];
        c->geo.order_start[q] = acc;
        acc += c->dmh[order[q]].n_act;
    }
    c->geo.order_start[n_dm] = acc;
    c->geo.n_items = acc;
    {
        int q = 0;
        for (int w = 0; w < n_wfs; ++w)
            if (c->wh[w].k <= 32) c->geo.wfs_order[q++] = w;
        c->geo.n_wfs_a = q;
        for (int w = 0; w < n_wfs; ++w)
            if (c->wh[w].k > 32) c->geo.wfs_order[q++] = w;
    }
    if ((e = dev_alloc(c, &c->d_vjp_part, (size_t)acc * n_wfs * 4)) != cudaSuccess)
        return bail(cuda_fail(c, e, "adjoint partials"));
    c->geo.n_dm = n_dm;
    c->geo.n_wfs = n_wfs;
    *out = c;
    return SYNIM_OK;
}

synim_status synim_im_query(const synim_ctx *ctx, int32_t dm, int32_t wfs, int64_t *n_rows,
                            int64_t *n_cols) {
    if (!ctx || !n_rows || !n_cols || dm < 0 || dm >= ctx->n_dm || wfs < 0 || wfs >= ctx->n_wfs)
        return SYNIM_ERR_INVALID_ARG;
    *n_rows = 2LL * ctx->wh[wfs].nv;
    *n_cols = ctx->dmh[dm].n_act;
    return SYNIM_OK;
}

synim_status synim_dm_window(const synim_ctx *ctx, int32_t dm, int32_t *W) {
    if (!ctx || !W || dm < 0 || dm >= ctx->n_dm) return SYNIM_ERR_INVALID_ARG;
    *W = ctx->dmh[dm].W;
    return SYNIM_OK;
}

synim_status synim_im_kernel_ms(synim_ctx *ctx, double *total_ms, int32_t *n_launches) {
    if (!ctx || !total_ms || !n_launches || !ctx->profile) return SYNIM_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    double ms = ctx->prof_acc_ms;
    int n = ctx->prof_acc_n;
    for (; ctx->prof_tail < ctx->prof_head; ++ctx->prof_tail) {
        const int q = (int)(ctx->prof_tail % NPROF);
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(ctx->prof_b[q]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ctx->prof_a[q], ctx->prof_b[q]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel timing");
        ms += t;
        ++n;
    }
    ctx->prof_acc_ms = 0.0;
    ctx->prof_acc_n = 0;
    *total_ms = ms;
    *n_launches = n;
    return SYNIM_OK;
}

synim_status synim_pair_affine(const synim_ctx *ctx, int32_t dm, int32_t wfs,
                               const synim_misreg *mis, double *A, double *b) {
    if (!ctx || !mis || !A || !b || dm < 0 || dm >= ctx->n_dm || wfs < 0 || wfs >= ctx->n_wfs)
        return SYNIM_ERR_INVALID_ARG;
    if (!(mis->mag > 0)) return SYNIM_ERR_INVALID_ARG;
    composite(ctx->dmh[dm], ctx->wh[wfs], *mis, A, b);
    return SYNIM_OK;
}

int32_t synim_debug_bounds(void) {
#ifdef SYNIM_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

synim_status synim_im_check(synim_ctx *ctx, void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    if ((e = cudaMemcpy(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(ctx, e, "error flag read");
    const int flag = *ctx->h_err;
    cudaMemset(ctx->d_err, 0, sizeof(int));
    if (flag & ERR_TIMEOUT) return fail(ctx, SYNIM_ERR_TIMEOUT, "a bounded device wait timed out");
    if (flag & ERR_ARENA) return fail(ctx, SYNIM_ERR_SHAPE, "slope values exceeded their shared-memory buffer");
    if (flag & ERR_BOUNDS) return fail(ctx, SYNIM_ERR_BOUNDS, "an IM kernel index left its buffer (access skipped)");
    return SYNIM_OK;
}

synim_status synim_wait_selftest(synim_ctx *ctx, int64_t limit_clocks, void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    const long long lim = std::min<long long>(std::max<long long>(limit_clocks, 1), 1LL << 31);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_wait_selftest<<<1, 32, 0, s>>>(lim, ctx->d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait self-test launch");
    return synim_im_check(ctx, cuda_stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// compute / sensitivity / vjp share one launch path
// ---------------------------------------------------------------------------
namespace {

synim_status run(synim_ctx *c, int mode, const synim_misreg *mis, float *const *im,
                 float *const *dim, const float *const *gim, double *grad_p, cudaStream_t s) {
    DeviceGuard guard(c->device);
    const int np = c->n_dm * c->n_wfs;
    const int NV = (mode == MODE_FWD) ? 1 : 5;
    const bool tele = c->slope_engine == SYNIM_ENGINE_TELESCOPING;
    if (tele && mode != MODE_FWD)
        return fail(c, SYNIM_ERR_INVALID_ARG, "the telescoping-sum engine computes IMs only (no tangents or vjp)");
    cudaError_t e;
    // parameter slot (pinned); wait for its previous copy to finish
    const int slot = c->slot;
    if (c->slot_used[slot] && (e = cudaEventSynchronize(c->slot_ev[slot])) != cudaSuccess)
        return cuda_fail(c, e, "slot wait");
    DevPair *hp = c->h_pairs[slot];
    // this call's table set: forward and tangent calls alternate between the
    // two; the adjoint, which synchronises at the end of each call, always
    // takes set 0 (alternating sets measured slower for it)
    const int ts = (tele || mode == MODE_VJP) ? 0 : c->tset;
    DevPair *dp = c->d_pairs[ts];
    std::vector<long long> need((size_t)np);
    int max_seg = 0;   // segments per axis of the largest sensor with weight boxes this call
    for (int d = 0; d < c->n_dm; ++d)
        for (int w = 0; w < c->n_wfs; ++w) {
            const int p = d * c->n_wfs + w;
            const synim_misreg &m = mis[p];
            if (!(m.mag > 0) || !std::isfinite(m.shift_x_px) || !std::isfinite(m.shift_y_px) ||
                !std::isfinite(m.rot_deg) || !std::isfinite(m.mag))
                return fail(c, SYNIM_ERR_INVALID_ARG, "misregistration of pair " + std::to_string(p));
            DevPair &P = hp[p];
            std::memset(&P, 0, sizeof(P));
            composite(c->dmh[d], c->wh[w], m, P.A, P.b);
            if (!invert2(P.A, P.Ai)) return fail(c, SYNIM_ERR_INVALID_ARG, "singular composite affine");
            composite_jac(c->dmh[d], m, P.A, P.b, P.dA, P.db);
            split_pair(P);
            P.pst = c->d_pst[ts] + c->pst_off[p];
            P.xcc = c->d_lines[ts] + c->line_off[p];
            P.ycc = P.xcc + (size_t)c->wh[w].M * (c->wh[w].n_sub + 1);
            if (mode == MODE_FWD) P.im = im ? im[p] : nullptr;
            if (mode == MODE_TAN) {
                P.im = im ? im[p] : nullptr;
                for (int q = 0; q < 4; ++q) P.dim[q] = dim ? dim[4 * p + q] : nullptr;
            }
            if (mode == MODE_VJP) P.gim = gim ? gim[p] : nullptr;
            // the numerical engine's boundary-segment weight boxes: values for
            // forward IMs, values and tangents for the sensitivities and the adjoint
            if (!tele && c->k_org[ts][p]) {
                const int s0 = kseg_shape(P.A, c->wh[w].k, 0), s1 = kseg_shape(P.A, c->wh[w].k, 1);
                if (s0 >= 0 && s1 >= 0) {
                    P.kf = 1;
                    P.kcomp = (mode == MODE_FWD) ? 1 : KNC;
                    P.kshape[0] = s0;
                    P.kshape[1] = s1;
                    for (int ax = 0; ax < 2; ++ax) {
                        P.korg[ax] = c->k_org[ts][p] + (size_t)ax * KPS;
                        P.kring[ax] = c->k_org[ts][p] + (size_t)(2 + ax) * KPS;
                        P.kw[ax] = c->k_w[ts][p] + (size_t)ax * KNC * KTAPS * KPS;
                        P.kwb[ax] = c->k_wb[ts][p] + (size_t)ax * KNC * KTAPS * KPS;
                    }
                }
            }
            {
                // 16-byte column stores need aligned outputs and 2 nv % 4 == 0
                auto al = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
                bool v4 = (2 * c->wh[w].nv) % 4 == 0;
                if (P.im && !al(P.im)) v4 = false;
                for (int q = 0; q < 4; ++q)
                    if (P.dim[q] && !al(P.dim[q])) v4 = false;
                P.vec4 = v4 ? 1 : 0;
            }
            need[p] = (seg_need(c->dmh[d], c->wh[w], P.Ai, NV) + 3) / 4 * 4;
            if (P.kf) {
                // chunks of box rows (X, Y, E of the rows, the carried Y row and the
                // ring buffer, NV values each) in at most 768 NV floats (forward) or
                // 3072 (tangents), and at least four rows: small boxes take one
                // chunk, large ones several, and the per-warp buffer stays small
                // enough for the occupancy the registers allow
                const long long nsj = (need[p] / (2 * NV) - 1) / 4;
                const long long whole = 2 * NV * ((nsj + 1) * (3 * nsj + 1) + nsj) + 64 * NV;
                const long long four = 2 * NV * (4 * (3 * nsj + 1) + nsj) + 64 * NV;
                const long long top = (NV == 1) ? 768 : 3072;
                need[p] = std::max(need[p], (std::max(four, std::min(whole, top)) + 3) / 4 * 4);
                max_seg = std::max(max_seg, c->wh[w].n_sub * (c->wh[w].n_sub + 1));
            }
        }
    // Per-warp segment buffer (one warp per column): the largest need over the pairs.
    Geo g = c->geo;
    long long cap = 4;
    for (int p = 0; p < np; ++p) cap = std::max(cap, need[p]);
    cap = std::max<long long>(cap, c->seg_floats);  // never shrink: keeps the captured graph
    int dev_max = 0;
    cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (!tele && (long long)8 * 4 * cap > dev_max)
        return fail(c, SYNIM_ERR_SHAPE,
                    "boundary segments need " + std::to_string(8 * 4 * cap) +
                        " bytes of shared memory per CTA; lower the grid or raise support_eps");
    int tele_cap4 = 0;   // the telescoping kernel's per-warp buffer (float4 subaperture sums)
    if (tele) {
        // a chunk of box rows plus the carried row: at least two rows, 256 float4 by default
        tele_cap4 = 256;
        for (int w = 0; w < c->n_wfs; ++w) tele_cap4 = std::max(tele_cap4, 2 * c->wh[w].n_sub);
        cap = 4;
        if ((long long)tele_smem_bytes(256, tele_cap4) > dev_max)
            return fail(c, SYNIM_ERR_SHAPE, "telescoping engine: too many subapertures per side for shared memory");
    }
    c->seg_floats = (int)cap;
    g.seg_floats = c->seg_floats;
    // launch shape: the tuned one once the autotuner has run for this mode
    int threads = c->threads;
    g.seg_lanes = 0;
    if (c->tuned[mode]) {
        threads = c->tune_threads[mode];
        g.seg_lanes = c->tune_lanes[mode];
    }
    size_t smem = im_smem_bytes(g, threads);
    const long long units = (long long)c->geo.n_items * c->n_wfs;
    auto grid_for = [&](int th) {
        const long long warps = th / 32;
        return (int)std::max<long long>(1, std::min<long long>((units + warps - 1) / warps, 1LL << 30));
    };
    int bps = 1;
    if (!tele && (e = im_prepare(mode, threads, smem, &bps)) != cudaSuccess)
        return cuda_fail(c, e, "kernel attributes");
    if (bps < 1) return fail(c, SYNIM_ERR_SHAPE, "IM kernel does not fit on an SM");
    int grid = grid_for(threads);
    // k_im when no pair has weight boxes, else k_imk for every column
    bool any_plain = false, any_k = false;
    for (int p = 0; p < np; ++p) {
        const DevPair &P = hp[p];
        const bool active = (mode == MODE_FWD) ? P.im != nullptr
                            : (mode == MODE_TAN) ? (P.im || P.dim[0] || P.dim[1] || P.dim[2] || P.dim[3])
                                                 : P.gim != nullptr;
        if (active && !P.kf) any_plain = true;
        if (active && P.kf) any_k = true;
    }
    if (!any_plain && !any_k) any_plain = true;   // nothing to compute: the plain kernel's empty launch
    // one launch: k_imk takes every forward column when some pair has weight boxes
    auto grids = [&](int th, int &g0, int &g1) {
        g0 = (any_plain && !any_k) ? grid_for(th) : 0;
        g1 = any_k ? grid_for(th) : 0;
    };
    // forward IMs and tangents build this call's tables on the prep stream,
    // once the IM launch that last read the set has finished; the adjoint
    // (which synchronises at the end of each call) builds them on the
    // caller's stream, and the telescoping engine has no tables to build
    const bool overlap = !tele && mode != MODE_VJP;
    cudaStream_t up = overlap ? c->prep : s;
    if (!tele && c->im_used[ts] && (e = cudaStreamWaitEvent(up, c->ev_im[ts], 0)) != cudaSuccess)
        return cuda_fail(c, e, "table set wait");
    if ((e = cudaMemcpyAsync(dp, hp, sizeof(DevPair) * np, cudaMemcpyHostToDevice, up)) != cudaSuccess)
        return cuda_fail(c, e, "parameter upload");
    cudaEventRecord(c->slot_ev[slot], up);
    c->slot_used[slot] = true;
    if (overlap && c->autotune && !c->tuned[mode]) {
        // the autotuner runs on the caller's stream: after the upload, and the
        // prep stream after it
        if ((e = cudaEventRecord(c->ev_prep[ts], up)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, c->ev_prep[ts], 0)) != cudaSuccess)
            return cuda_fail(c, e, "autotune order");
    }
    c->slot = (slot + 1) % NSLOT;
    if (c->autotune && !c->tuned[mode] && tele) {
        // autotuner of the telescoping kernel: lanes per subaperture (each
        // sensor's create-time choice times 1/2, 1, 2 or 4, within 1..32) x
        // 128 or 256 threads, timed like the IM kernel's candidates
        static const int cand_threads[] = {128, 256};
        static const int cand_shift[] = {-1, 0, 1, 2};
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess)
            return cuda_fail(c, e, "autotune events");
        const TeleSet base = c->tele;
        TeleSet best_set = base;
        float best = 3e38f;
        int best_th = threads;
        for (int th : cand_threads)
            for (int sh : cand_shift) {
                TeleSet t = base;
                for (int w = 0; w < c->n_wfs; ++w) {
                    const int L = base.w[w].lanes;
                    t.w[w].lanes = std::min(32, std::max(1, sh < 0 ? (L >> -sh) : (L << sh)));
                }
                const int gr = grid_for(th);
                float ms = 0.f;
                e = launch_tele(g, t, dp, tele_cap4, c->d_err, gr, th, s);
                if (e == cudaSuccess) e = cudaEventRecord(t0, s);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r)
                    e = launch_tele(g, t, dp, tele_cap4, c->d_err, gr, th, s);
                if (e == cudaSuccess) e = cudaEventRecord(t1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e != cudaSuccess) break;
                if (ms < best) {
                    best = ms;
                    best_th = th;
                    best_set = t;
                }
            }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
        c->tele = best_set;
        c->tuned[mode] = true;
        c->tune_threads[mode] = best_th;
        c->tune_lanes[mode] = best_set.w[0].lanes;
        c->tune_ms[mode] = best / 3.f;
        threads = best_th;
        grid = grid_for(threads);
    }
    bool ran_tuner = false;
    if (c->autotune && !c->tuned[mode] && !tele) {
        ran_tuner = true;
        // autotuner: time each candidate launch shape on this call's inputs
        // (three launches after a warm-up) and keep the fastest for the mode
        static const int cand_threads[] = {128, 256};
        static const int cand_lanes[] = {2, 4, 8};
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess)
            return cuda_fail(c, e, "autotune events");
        float best = 3e38f;
        int best_th = threads, best_l = 0;
        if ((e = launch_pst(g, dp, c->max_mm, c->max_lines, s)) != cudaSuccess ||
            (e = launch_kseg(g, dp, max_seg, mode == MODE_FWD ? 1 : KNC, s)) != cudaSuccess)
            return cuda_fail(c, e, "autotune");
        for (int th : cand_threads)
            for (int l : cand_lanes) {
                Geo gt = g;
                gt.seg_lanes = l;
                int b2 = 0;
                const size_t sm = im_smem_bytes(g, th);
                if ((e = im_prepare(mode, th, sm, &b2)) != cudaSuccess || b2 < 1) continue;
                int gr = 0, gk = 0;
                grids(th, gr, gk);
                float ms = 0.f;
                e = launch_im(mode, gt, dp, c->d_err, c->d_vjp_part, gr, th, sm, s, gk);
                if (e == cudaSuccess) e = cudaEventRecord(t0, s);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r)
                    e = launch_im(mode, gt, dp, c->d_err, c->d_vjp_part, gr, th, sm, s, gk);
                if (e == cudaSuccess) e = cudaEventRecord(t1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e != cudaSuccess) break;
                if (ms < best) {
                    best = ms;
                    best_th = th;
                    best_l = l;
                }
            }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
        c->tuned[mode] = true;
        c->tune_threads[mode] = best_th;
        c->tune_lanes[mode] = best_l;
        c->tune_ms[mode] = best / 3.f;
        threads = best_th;
        g.seg_lanes = best_l;
        smem = im_smem_bytes(g, threads);
        if ((e = im_prepare(mode, threads, smem, &bps)) != cudaSuccess) return cuda_fail(c, e, "kernel attributes");
        grid = grid_for(threads);
    }
    // profiling: pick the event pair of this launch (collect the oldest if the ring is full)
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    if (c->profile) {
        if (c->prof_head - c->prof_tail >= (unsigned long long)NPROF) {
            const int q = (int)(c->prof_tail % NPROF);
            float t = 0.f;
            if (cudaEventSynchronize(c->prof_b[q]) == cudaSuccess &&
                cudaEventElapsedTime(&t, c->prof_a[q], c->prof_b[q]) == cudaSuccess) {
                c->prof_acc_ms += t;
                ++c->prof_acc_n;
            }
            ++c->prof_tail;
        }
        const int q = (int)(c->prof_head % NPROF);
        ++c->prof_head;
        ev_a = c->prof_a[q];
        ev_b = c->prof_b[q];
    }
    // (inside a capture, only an "external" record becomes an event-record node)
    // part 0: the IM kernel (or the telescoping kernel), on the caller's
    // stream; part 1: the class kernels and weight boxes, on the prep stream
    auto enqueue = [&](int part, cudaStream_t q, cudaEvent_t a0, cudaEvent_t b0, bool capturing) -> cudaError_t {
        const unsigned int rf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (part == 1) {
            cudaError_t r = launch_pst(g, dp, c->max_mm, c->max_lines, q);
            if (r == cudaSuccess) r = launch_kseg(g, dp, max_seg, mode == MODE_FWD ? 1 : KNC, q);
            return r;
        }
        cudaError_t r = a0 ? cudaEventRecordWithFlags(a0, q, rf) : cudaSuccess;
        if (tele) {
            // telescoping sum: one kernel, no pixel classes
            if (r == cudaSuccess) r = launch_tele(g, c->tele, dp, tele_cap4, c->d_err, grid, threads, q);
        } else {
            int g0 = 0, g1 = 0;
            grids(threads, g0, g1);
            if (r == cudaSuccess) r = launch_im(mode, g, dp, c->d_err, c->d_vjp_part, g0, threads, smem, q, g1);
            if (r == cudaSuccess && mode == MODE_VJP) r = launch_vjp_reduce(g, c->d_vjp_part, c->d_gp, q);
        }
        if (r == cudaSuccess && b0) r = cudaEventRecordWithFlags(b0, q, rf);
        return r;
    };
    // one part, from its captured graph where graphs are on (one graph per
    // part, table set and launch shape)
    auto launch_part = [&](int part, cudaStream_t q) -> synim_status {
        const bool prof = c->profile && part == 0;
        if (!c->use_graph) {
            const cudaError_t r = enqueue(part, q, prof ? ev_a : nullptr, prof ? ev_b : nullptr, false);
            return r == cudaSuccess ? SYNIM_OK : cuda_fail(c, r, "launch");
        }
        // the weight-box kernel's grid (max_seg) is part of the captured launches
        const auto key = std::make_tuple(mode * 4 + (any_plain ? 1 : 0) + (any_k ? 2 : 0) + 16 * ts + 64 * part,
                                         smem, grid, threads * 16 + g.seg_lanes + max_seg * 65536);
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            GraphEntry ge;
            if ((e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(c, e, "graph capture begin");
            cudaError_t e1 = enqueue(part, c->cap, prof ? c->prof_a[0] : nullptr, prof ? c->prof_b[0] : nullptr, true);
            e = cudaStreamEndCapture(c->cap, &ge.graph);
            if (e1 != cudaSuccess) {
                if (ge.graph) cudaGraphDestroy(ge.graph);
                return cuda_fail(c, e1, "graph capture");
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "graph capture end");
            if (prof) {
                size_t nn = 0;
                cudaGraphGetNodes(ge.graph, nullptr, &nn);
                std::vector<cudaGraphNode_t> nodes(nn);
                cudaGraphGetNodes(ge.graph, nodes.data(), &nn);
                for (cudaGraphNode_t nd : nodes) {
                    cudaGraphNodeType ty;
                    cudaEvent_t ev = nullptr;
                    if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
                    if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
                    if (ev == c->prof_a[0]) ge.ev_start = nd;
                    if (ev == c->prof_b[0]) ge.ev_stop = nd;
                }
            }
            e = cudaGraphInstantiate(&ge.exec, ge.graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(ge.graph);
                return cuda_fail(c, e, "graph instantiate");
            }
            it = c->graphs.emplace(key, ge).first;
        }
        if (prof) {
            if (!it->second.ev_start || !it->second.ev_stop)
                return fail(c, SYNIM_ERR_CUDA, "profiling: event nodes missing from the captured graph");
            if ((e = cudaGraphExecEventRecordNodeSetEvent(it->second.exec, it->second.ev_start, ev_a)) != cudaSuccess ||
                (e = cudaGraphExecEventRecordNodeSetEvent(it->second.exec, it->second.ev_stop, ev_b)) != cudaSuccess)
                return cuda_fail(c, e, "profiling: event node update");
        }
        if ((e = cudaGraphLaunch(it->second.exec, q)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
        return SYNIM_OK;
    };
    synim_status st = SYNIM_OK;
    if (tele) {
        if ((st = launch_part(0, s)) != SYNIM_OK) return st;
    } else {
        // the autotuner's launches (caller's stream) read this set: the prep
        // stream rebuilds it after them
        if (overlap && ran_tuner &&
            ((e = cudaEventRecord(c->ev_im[ts], s)) != cudaSuccess ||
             (e = cudaStreamWaitEvent(c->prep, c->ev_im[ts], 0)) != cudaSuccess))
            return cuda_fail(c, e, "autotune order");
        if ((st = launch_part(1, up)) != SYNIM_OK) return st;
        if (overlap && ((e = cudaEventRecord(c->ev_prep[ts], up)) != cudaSuccess ||
                        (e = cudaStreamWaitEvent(s, c->ev_prep[ts], 0)) != cudaSuccess))
            return cuda_fail(c, e, "table set order");
        if ((st = launch_part(0, s)) != SYNIM_OK) return st;
        if ((e = cudaEventRecord(c->ev_im[ts], s)) != cudaSuccess) return cuda_fail(c, e, "table set release");
        c->im_used[ts] = true;
        if (mode != MODE_VJP) c->tset = ts ^ 1;
    }
    if (mode == MODE_VJP) {
        std::vector<double> tmp((size_t)np * 4);
        if ((e = cudaMemcpyAsync(tmp.data(), c->d_gp, sizeof(double) * np * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(c, e, "vjp readback");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "vjp sync");
        std::memcpy(grad_p, tmp.data(), sizeof(double) * np * 4);
    }
    return SYNIM_OK;
}

}  // namespace

extern "C" synim_status synim_im_tuning(const synim_ctx *ctx, int32_t mode, int32_t *threads, int32_t *seg_lanes,
                                        double *ms) {
    if (!ctx || mode < 0 || mode > 2) return SYNIM_ERR_INVALID_ARG;
    const bool t = ctx->tuned[mode];
    if (threads) *threads = t ? ctx->tune_threads[mode] : ctx->threads;
    if (seg_lanes) *seg_lanes = t ? ctx->tune_lanes[mode] : 0;
    if (ms) *ms = t ? (double)ctx->tune_ms[mode] : 0.0;
    return t ? SYNIM_OK : SYNIM_ERR_NOT_CONVERGED;
}

extern "C" synim_status synim_im_compute(synim_ctx *ctx, const synim_misreg *mis, float *const *im,
                                         void *cuda_stream) {
    if (!ctx || !mis || !im) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    return run(ctx, MODE_FWD, mis, im, nullptr, nullptr, nullptr, static_cast<cudaStream_t>(cuda_stream));
}

extern "C" synim_status synim_im_sensitivity(synim_ctx *ctx, const synim_misreg *mis, float *const *im,
                                             float *const *d_im, void *cuda_stream) {
    if (!ctx || !mis || !d_im) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    return run(ctx, MODE_TAN, mis, im, d_im, nullptr, nullptr, static_cast<cudaStream_t>(cuda_stream));
}

extern "C" synim_status synim_im_vjp(synim_ctx *ctx, const synim_misreg *mis, const float *const *grad_im,
                                     double *grad_p, void *cuda_stream) {
    if (!ctx || !mis || !grad_im || !grad_p) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    return run(ctx, MODE_VJP, mis, nullptr, nullptr, grad_im, grad_p, static_cast<cudaStream_t>(cuda_stream));
}
