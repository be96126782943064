// synim_probe.cu -- probe responses of one (DM, sensor) pair for many
// misregistrations at once: the input of the misregistration estimators.
//
// A probe mode is a DM shape S_m = sum_a cmd[m][a] IF_a.  The screens are
// formed once on the device and kept interleaved, [N + 2][N + 2][NMP] FP32
// with a zero border (NMP = modes rounded up to 4), so one bilinear tap of
// all modes is NMP consecutive floats.  They are small (config of the learned
// estimator: 322^2 x 16 x 4 B = 6.6 MB) and stay in L2 while every sample's
// resample gathers from them.
//
// k_probe: one CTA per (sample, subaperture row, chunk of Cs subapertures).
//   phase 1: strict core (Sec. 2.3 step 1) of the tile with a 3-pixel halo,
//            and the tile's pupil bytes, into shared memory;
//   phase 2: repaired phase of all modes (and tangents) at the k + 2 rows x
//            Cs k + 2 columns the central differences touch: core pixels are
//            one bilinear resample (Sec. 2.1), ring pixels the mean over the
//            valid cardinal directions of 2 P1 - P2 or P1 (Sec. 2.3 steps
//            2-3), the rest zero;
//   phase 3: pupil-weighted central differences summed per subaperture and
//            scaled by slope_scale / (2 dw lit) (Sec. 2.2), one coalesced
//            store of the chunk's Cs x C channels.
// Coordinates: each pixel's DM position is evaluated with an error-free
// split of A (j, i) + b about the integer part of a cheap estimate, so the
// bilinear weights carry no cancellation error from coordinates near 300 px.
#include <cfloat>
#include <climits>
#include <cstring>

#include <cuda_bf16.h>

#include "synim_internal.h"
#include "synim_device.cuh"

namespace synim {

constexpr double kCoreThreshold = 0.999999;  // Sec. 2.3, step 1
constexpr int kProbeThreads = 256;
constexpr int kMaxModes = 32;
constexpr size_t kProbeSmemCap = 64 * 1024;  // per CTA, for 3-4 resident CTAs per SM

// Per-sample transform.
struct ProbeAff {
    double A[4], b[2];                      // FP64 (mask cells that need the exact core test)
    float Ahi[4], Alo[4], bhi[2], blo[2];   // A, b as float pairs
    float dA[16], db[8];                    // d(A, b)/dp_k
};

struct ProbeGeo {
    const float *scr;        // [(N + 2)^2][NMP]
    const uint8_t *mask;     // DM mask [N][N] or nullptr (all ones)
    const uint8_t *pupil;    // [M][M]
    const int *vidx;         // [n_sub^2] valid row or -1
    const float *fac;        // [nv] slope_scale / (2 dw lit)
    int N, M, k, n_sub, n_modes, NMP, C;
    int Cs, n_chunks;        // subapertures per CTA, chunks per subaperture row
};

struct ProbeSet {
    int dm = -1, wfs = -1, n_modes = 0, NMP = 0;
    double *cmd = nullptr;   // [NMP][n_act]
    float *scr = nullptr;
    uint8_t *pupil = nullptr;
    ProbeGeo geo{};
    size_t smem_fwd = 0, smem_tan = 0;
    int cs_fwd = 1, cs_tan = 1;
    // scratch
    ProbeAff *aff = nullptr;
    long long aff_cap = 0;
    float *clean = nullptr;
    unsigned *peak = nullptr;
    long long gen_cap = 0;   // samples the clean buffer holds
};

int probe_per_sample(const ProbeSet *p) { return p->geo.n_sub * p->geo.n_sub * p->geo.C; }

void probe_destroy(ProbeSet *p) {
    if (!p) return;
    cudaFree(p->cmd);
    cudaFree(p->scr);
    cudaFree(p->pupil);
    cudaFree(p->aff);
    cudaFree(p->clean);
    cudaFree(p->peak);
    delete p;
}

// ---------------------------------------------------------------------------
// Screens: S_m(x, y) = sum over actuators whose packed window covers (x, y)
// of cmd[m][a] IF_a(x, y), accumulated in FP64 in actuator order.
// ---------------------------------------------------------------------------
__global__ void k_form_screens(const DevDM D, const double *__restrict__ cmd, int NMP,
                               float *__restrict__ scr) {
    const int N = D.N, N2 = N + 2;
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)N2 * N2) return;
    const int py = (int)(q / N2), px = (int)(q - (long)py * N2);
    float *dst = scr + q * NMP;
    const int x = px - 1, y = py - 1;
    double acc[kMaxModes];
#pragma unroll
    for (int m = 0; m < kMaxModes; ++m) acc[m] = 0.0;
    if (x >= 0 && y >= 0 && x < N && y < N) {
        for (int a = 0; a < D.n_act; ++a) {
            const int cx = x - D.org[2 * a] + 1, cy = y - D.org[2 * a + 1] + 1;
            if (cx < 1 || cy < 1 || cx > D.W || cy > D.W) continue;
            const double v = (double)D.win[(size_t)a * D.win_stride + (size_t)cy * D.Wp + cx];
            if (v == 0.0) continue;
#pragma unroll
            for (int m = 0; m < kMaxModes; ++m)
                if (m < NMP) acc[m] += cmd[(size_t)m * D.n_act + a] * v;
        }
    }
#pragma unroll
    for (int m = 0; m < kMaxModes; ++m)
        if (m < NMP) dst[m] = (float)acc[m];
}

// The parts of the composite transform (Sec. 2.1) that depend on the pair
// alone, formed on the host: the sensor's rotation-magnification matrix X =
// R(theta_w) diag(mag_w), the conjugation factor times the sensor pixel,
// the pair's translation before the misregistration, and the grid centres.
struct AffPre {
    double X00, X01, X10, X11;   // X
    double cdw;                  // (1 - h / H) D_w / M
    double tx0, ty0;             // (1 - h / H) shift_w + h theta_w
    double dd, cN, cM;           // DM pitch; (N - 1) / 2, (M - 1) / 2
};

AffPre aff_pre(const DmHost &D, const WfsHost &W) {
    AffPre a;
    const double cone = (W.H > 0.0 && std::isfinite(W.H)) ? 1.0 - D.h / W.H : 1.0;
    const double tw = W.rot * kPi / 180.0, cw = std::cos(tw), sw = std::sin(tw);
    a.X00 = cw * W.mag[0];
    a.X01 = -sw * W.mag[1];
    a.X10 = sw * W.mag[0];
    a.X11 = cw * W.mag[1];
    a.cdw = cone * (W.D / W.M);
    a.tx0 = cone * W.shift[0] + D.h * W.th[0];
    a.ty0 = cone * W.shift[1] + D.h * W.th[1];
    a.dd = D.dd;
    a.cN = (D.N - 1) * 0.5;
    a.cM = (W.M - 1) * 0.5;
    return a;
}

// Per-sample composite transform (Sec. 2.1) and, with with_jac, its
// parameter derivatives in closed form: the shifts translate by -R(-td) e /
// mag; the rotation turns the map about the DM centre (dA = -J A, db = -J (b
// - cN), J = [[0, -1], [1, 0]], per radian); the magnification scales it
// about the DM centre (dA = -A / mag, db = -(b - cN) / mag).  One FP64 sincos
// and one reciprocal per sample: FP64 is a narrow pipe on this part and the
// kernel runs once per fit pass.
__global__ void k_probe_affine(const AffPre Q, const double *__restrict__ params, long n, int with_jac,
                               ProbeAff *__restrict__ out) {
    const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double sx = params[4 * s + 0], sy = params[4 * s + 1], rot = params[4 * s + 2], mag = params[4 * s + 3];
    double st, ct;
    sincos(rot * (kPi / 180.0), &st, &ct);
    const double inv = 1.0 / (Q.dd * mag), sc = Q.cdw * inv;
    ProbeAff P;
    // A = sc R(-td) X, R(-td) = [[ct, st], [-st, ct]]
    P.A[0] = sc * (ct * Q.X00 + st * Q.X10);
    P.A[1] = sc * (ct * Q.X01 + st * Q.X11);
    P.A[2] = sc * (-st * Q.X00 + ct * Q.X10);
    P.A[3] = sc * (-st * Q.X01 + ct * Q.X11);
    const double tx = Q.tx0 - sx * Q.dd, ty = Q.ty0 - sy * Q.dd;
    P.b[0] = Q.cN + inv * (ct * tx + st * ty) - (P.A[0] + P.A[1]) * Q.cM;
    P.b[1] = Q.cN + inv * (-st * tx + ct * ty) - (P.A[2] + P.A[3]) * Q.cM;
    for (int q = 0; q < 4; ++q) {
        P.Ahi[q] = (float)P.A[q];
        P.Alo[q] = (float)(P.A[q] - (double)P.Ahi[q]);
    }
    for (int q = 0; q < 2; ++q) {
        P.bhi[q] = (float)P.b[q];
        P.blo[q] = (float)(P.b[q] - (double)P.bhi[q]);
    }
    for (int q = 0; q < 16; ++q) P.dA[q] = 0.f;
    for (int q = 0; q < 8; ++q) P.db[q] = 0.f;
    if (with_jac) {
        const double rm = 1.0 / mag, rad = kPi / 180.0;
        P.db[0] = (float)(-ct * rm);
        P.db[1] = (float)(st * rm);
        P.db[2] = (float)(-st * rm);
        P.db[3] = (float)(-ct * rm);
        P.dA[8] = (float)(rad * P.A[2]);
        P.dA[9] = (float)(rad * P.A[3]);
        P.dA[10] = (float)(-rad * P.A[0]);
        P.dA[11] = (float)(-rad * P.A[1]);
        P.db[4] = (float)(rad * (P.b[1] - Q.cN));
        P.db[5] = (float)(-rad * (P.b[0] - Q.cN));
        for (int q = 0; q < 4; ++q) P.dA[12 + q] = (float)(-P.A[q] * rm);
        P.db[6] = (float)(-(P.b[0] - Q.cN) * rm);
        P.db[7] = (float)(-(P.b[1] - Q.cN) * rm);
    }
    out[s] = P;
}

// Integer cell and fraction of one DM coordinate: ah, al / bh, bl / ch, cl are
// the float pairs of the coefficient of j, of i and of the offset.
__device__ __forceinline__ void cell_coord(float ah, float al, float bh, float bl, float ch,
                                           float cl, int j, int i, int &ic, float &f) {
    float e = fmaf(ah, (float)j, fmaf(bh, (float)i, ch));
    e = fminf(fmaxf(e, -1.0e6f), 1.0e6f);
    const int off = (int)floorf(e);
    const float r = exact_affine(ah, al, bh, bl, ch, cl, j, i, off);
    const float fr = floorf(r);
    ic = off + (int)fr;
    f = r - fr;
}

__device__ __forceinline__ int mask_tap_p(const uint8_t *__restrict__ mask, int N, int x, int y) {
    if (x < 0 || y < 0 || x >= N || y >= N) return 0;
    return mask ? (mask[(size_t)y * N + x] != 0) : 1;
}

// Strict core test (Sec. 2.3 step 1) at sensor pixel (i, j): all four mask
// taps of the cell one -> core, all zero -> not; otherwise the FP64
// definition (no contraction), as the oracle evaluates it.
__device__ __forceinline__ bool core_at(const ProbeGeo &G, const ProbeAff &P, int i, int j) {
    int ix, iy;
    float fx, fy;
    cell_coord(P.Ahi[0], P.Alo[0], P.Ahi[1], P.Alo[1], P.bhi[0], P.blo[0], j, i, ix, fx);
    cell_coord(P.Ahi[2], P.Alo[2], P.Ahi[3], P.Alo[3], P.bhi[1], P.blo[1], j, i, iy, fy);
    const int s = mask_tap_p(G.mask, G.N, ix, iy) + mask_tap_p(G.mask, G.N, ix + 1, iy) +
                  mask_tap_p(G.mask, G.N, ix, iy + 1) + mask_tap_p(G.mask, G.N, ix + 1, iy + 1);
    if (s == 4) return true;
    if (s == 0) return false;
    const double x = __dadd_rn(__dadd_rn(__dmul_rn(P.A[0], (double)j), __dmul_rn(P.A[1], (double)i)), P.b[0]);
    const double y = __dadd_rn(__dadd_rn(__dmul_rn(P.A[2], (double)j), __dmul_rn(P.A[3], (double)i)), P.b[1]);
    const double x0 = floor(x), y0 = floor(y);
    const double ex = __dadd_rn(x, -x0), ey = __dadd_rn(y, -y0);
    const int cx = (int)x0, cy = (int)y0;
    const double gx = __dadd_rn(1.0, -ex), gy = __dadd_rn(1.0, -ey);
    double m = __dmul_rn(__dmul_rn(gx, gy), (double)mask_tap_p(G.mask, G.N, cx, cy));
    m = __dadd_rn(m, __dmul_rn(__dmul_rn(ex, gy), (double)mask_tap_p(G.mask, G.N, cx + 1, cy)));
    m = __dadd_rn(m, __dmul_rn(__dmul_rn(gx, ey), (double)mask_tap_p(G.mask, G.N, cx, cy + 1)));
    m = __dadd_rn(m, __dmul_rn(__dmul_rn(ex, ey), (double)mask_tap_p(G.mask, G.N, cx + 1, cy + 1)));
    return m >= kCoreThreshold;
}

// One bilinear tap set (Sec. 2.1) of sensor pixel (i, j): base pointers of the
// cell's two rows in the interleaved screens, the fractions and, with NV = 5,
// the coordinate derivatives d(x, y)/dp_k.
template <int NV>
struct Tap {
    const float *t0, *t1;
    float fx, fy;
    float dx[4], dy[4];
    bool zero;

    __device__ __forceinline__ void at(const ProbeGeo &G, const ProbeAff &P, int i, int j, int NMP) {
        int ix, iy;
        cell_coord(P.Ahi[0], P.Alo[0], P.Ahi[1], P.Alo[1], P.bhi[0], P.blo[0], j, i, ix, fx);
        cell_coord(P.Ahi[2], P.Alo[2], P.Ahi[3], P.Alo[3], P.bhi[1], P.blo[1], j, i, iy, fy);
        zero = (ix < -1 || iy < -1 || ix > G.N - 1 || iy > G.N - 1);
        const int N2 = G.N + 2;
        t0 = zero ? G.scr : G.scr + ((size_t)(iy + 1) * N2 + (ix + 1)) * NMP;
        t1 = t0 + (zero ? 0 : (size_t)N2 * NMP);
        if (NV == 5) {
            const float fj = (float)j, fi = (float)i;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dx[k] = fmaf(P.dA[4 * k + 0], fj, fmaf(P.dA[4 * k + 1], fi, P.db[2 * k + 0]));
                dy[k] = fmaf(P.dA[4 * k + 2], fj, fmaf(P.dA[4 * k + 3], fi, P.db[2 * k + 1]));
            }
        }
    }

    // Modes m4 .. m4 + 3: out[v * 4 + u] (v = 0 phase, 1 + k tangent k).
    __device__ __forceinline__ void group(int m4, int NMP, float *out) const {
        if (zero) {
#pragma unroll
            for (int q = 0; q < NV * 4; ++q) out[q] = 0.f;
            return;
        }
        const float4 a00 = __ldg(reinterpret_cast<const float4 *>(t0 + m4));
        const float4 a10 = __ldg(reinterpret_cast<const float4 *>(t0 + NMP + m4));
        const float4 a01 = __ldg(reinterpret_cast<const float4 *>(t1 + m4));
        const float4 a11 = __ldg(reinterpret_cast<const float4 *>(t1 + NMP + m4));
        const float v00[4] = {a00.x, a00.y, a00.z, a00.w}, v10[4] = {a10.x, a10.y, a10.z, a10.w};
        const float v01[4] = {a01.x, a01.y, a01.z, a01.w}, v11[4] = {a11.x, a11.y, a11.z, a11.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float ex = v10[u] - v00[u], ex1 = v11[u] - v01[u];
            const float top = fmaf(fx, ex, v00[u]), bot = fmaf(fx, ex1, v01[u]);
            out[u] = fmaf(fy, bot - top, top);
            if (NV == 5) {
                const float gx = fmaf(fy, ex1 - ex, ex), gy = bot - top;
#pragma unroll
                for (int k = 0; k < 4; ++k) out[(1 + k) * 4 + u] = fmaf(gx, dx[k], gy * dy[k]);
            }
        }
    }
};

// Shared-memory tile pixel layout: [v][NMP] floats (v = phase, tangents).
template <int NV, int NMP>
__device__ __forceinline__ void store_group(float *dst, int m4, const float *g) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
        *reinterpret_cast<float4 *>(dst + v * NMP + m4) = make_float4(g[4 * v], g[4 * v + 1], g[4 * v + 2], g[4 * v + 3]);
}

template <int NV, int NMP>
__global__ void __launch_bounds__(kProbeThreads)
k_probe(const __grid_constant__ ProbeGeo G, const ProbeAff *__restrict__ aff, long n,
        float *__restrict__ maps, float *__restrict__ dmaps, unsigned *__restrict__ peak) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int k = G.k, Cs = G.Cs;
    const long blk = blockIdx.x;
    const long per_sample = (long)G.n_sub * G.n_chunks;
    const long s = blk / per_sample;
    if (s >= n) return;
    const int rem = (int)(blk - s * per_sample);
    const int si = rem / G.n_chunks, ch = rem - si * G.n_chunks;
    const int sj0 = ch * Cs, ncs = min(Cs, G.n_sub - sj0);
    const int i0 = si * k, j0 = sj0 * k;
    // tile geometry: phase rows i0-1 .. i0+k, columns j0-1 .. j0+Cs k
    const int TR = k + 2, TC = Cs * k + 2;
    const int CR = k + 6, CC = Cs * k + 6;  // core map: 2 more on each side
    constexpr int PV = NV * NMP;            // floats per tile pixel
    float *phi = reinterpret_cast<float *>(smem);
    uint8_t *core = smem + (size_t)TR * TC * PV * 4;
    uint8_t *pup = core + CR * CC;
    __shared__ ProbeAff sP;
    __shared__ float s_red[kProbeThreads / 32];
    if (threadIdx.x == 0) sP = aff[s];
    __syncthreads();
    const ProbeAff &P = sP;

    // ---- phase 1: core map with halo, pupil bytes of the chunk ----
    for (int q = threadIdx.x; q < CR * CC; q += blockDim.x) {
        const int r = q / CC, c = q - r * CC;
        const int i = i0 - 3 + r, j = j0 - 3 + c;
        bool v = false;
        if (i >= 0 && j >= 0 && i < G.M && j < G.M) v = core_at(G, P, i, j);
        core[q] = v ? 1 : 0;
    }
    for (int q = threadIdx.x; q < k * Cs * k; q += blockDim.x) {
        const int r = q / (Cs * k), c = q - r * (Cs * k);
        const int i = i0 + r, j = j0 + c;
        pup[q] = (j < G.M) ? G.pupil[(size_t)i * G.M + j] : 0;
    }
    __syncthreads();

    // ---- phase 2: repaired phase (and tangents) on the tile ----
    auto is_core = [&](int i, int j) -> bool {
        return core[(i - i0 + 3) * CC + (j - j0 + 3)] != 0;
    };
    for (int q = threadIdx.x; q < TR * TC; q += blockDim.x) {
        const int r = q / TC, c = q - r * TC;
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        float *dst = phi + (size_t)q * PV;
        float g[NV * 4];
        if (i < 0 || j < 0 || i >= G.M || j >= G.M || (!is_core(i, j) &&
            !((j + 1 < G.M && is_core(i, j + 1)) || (j > 0 && is_core(i, j - 1)) ||
              (i + 1 < G.M && is_core(i + 1, j)) || (i > 0 && is_core(i - 1, j))))) {
#pragma unroll
            for (int t = 0; t < NV * 4; ++t) g[t] = 0.f;
#pragma unroll
            for (int m4 = 0; m4 < NMP; m4 += 4) store_group<NV, NMP>(dst, m4, g);
            continue;
        }
        if (is_core(i, j)) {
            Tap<NV> T;
            T.at(G, P, i, j, NMP);
#pragma unroll
            for (int m4 = 0; m4 < NMP; m4 += 4) {
                T.group(m4, NMP, g);
                store_group<NV, NMP>(dst, m4, g);
            }
            continue;
        }
        // ring pixel: mean over valid directions of 2 P1 - P2 (or P1)
#pragma unroll 1
        for (int m4 = 0; m4 < NMP; m4 += 4) {
            float acc[NV * 4];
#pragma unroll
            for (int t = 0; t < NV * 4; ++t) acc[t] = 0.f;
            int nd = 0;
#pragma unroll 1
            for (int d = 0; d < 4; ++d) {
                const int di = (d == 2) ? 1 : (d == 3 ? -1 : 0);
                const int dj = (d == 0) ? 1 : (d == 1 ? -1 : 0);
                const int i1 = i + di, j1 = j + dj, i2 = i1 + di, j2 = j1 + dj;
                if (i1 < 0 || j1 < 0 || i1 >= G.M || j1 >= G.M || !is_core(i1, j1)) continue;
                Tap<NV> T;
                T.at(G, P, i1, j1, NMP);
                T.group(m4, NMP, g);
                if (i2 >= 0 && j2 >= 0 && i2 < G.M && j2 < G.M && is_core(i2, j2)) {
#pragma unroll
                    for (int t = 0; t < NV * 4; ++t) acc[t] += 2.f * g[t];
                    T.at(G, P, i2, j2, NMP);
                    T.group(m4, NMP, g);
#pragma unroll
                    for (int t = 0; t < NV * 4; ++t) acc[t] -= g[t];
                } else {
#pragma unroll
                    for (int t = 0; t < NV * 4; ++t) acc[t] += g[t];
                }
                ++nd;
            }
            const float inv = nd ? 1.f / (float)nd : 0.f;
#pragma unroll
            for (int t = 0; t < NV * 4; ++t) acc[t] *= inv;
            store_group<NV, NMP>(dst, m4, acc);
        }
    }
    __syncthreads();

    // ---- phase 3: pupil-weighted central differences per subaperture ----
    float mx = 0.f;
    const int items = ncs * G.n_modes * NV;
    for (int q = threadIdx.x; q < items; q += blockDim.x) {
        const int m = q % G.n_modes;
        const int t2 = q / G.n_modes;
        const int cc = t2 % ncs, vv = t2 / ncs;
        const int sj = sj0 + cc;
        const int vr = G.vidx[si * G.n_sub + sj];
        float sx = 0.f, sy = 0.f;
        if (vr >= 0) {
            const int off = vv * NMP + m;
            for (int r = 0; r < k; ++r) {
                const int tr = r + 1;
                for (int c = 0; c < k; ++c) {
                    if (!pup[r * (Cs * k) + cc * k + c]) continue;
                    const int tc = cc * k + c + 1;
                    sx += phi[((size_t)tr * TC + tc + 1) * PV + off] - phi[((size_t)tr * TC + tc - 1) * PV + off];
                    sy += phi[((size_t)(tr + 1) * TC + tc) * PV + off] - phi[((size_t)(tr - 1) * TC + tc) * PV + off];
                }
            }
            const float f = G.fac[vr];
            sx *= f;
            sy *= f;
        }
        const size_t o = (((size_t)s * G.n_sub + si) * G.n_sub + sj) * G.C + 2 * m;
        float2 w2;
        w2.x = sx;
        w2.y = sy;
        if (vv == 0) {
            *reinterpret_cast<float2 *>(maps + o) = w2;
            mx = fmaxf(mx, fmaxf(fabsf(sx), fabsf(sy)));
        } else {
            *reinterpret_cast<float2 *>(dmaps + (size_t)(vv - 1) * n * G.n_sub * G.n_sub * G.C + o) = w2;
        }
    }
    if (peak) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, s_red[w]);
            atomicMax(peak + s, __float_as_uint(b));
        }
    }
}

// ---------------------------------------------------------------------------
// Noise: Philox4x32-10 (Salmon et al., SC 2011) from its published
// definition, Box-Muller (1958) to normal deviates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__global__ void k_probe_noise(const float *__restrict__ clean, const unsigned *__restrict__ peak,
                              const int *__restrict__ vidx, long n, int per_sample, int C,
                              uint64_t seed, uint64_t sample0, float noise_rel,
                              __nv_bfloat16 *__restrict__ out) {
    const int groups = (per_sample + 3) / 4;
    const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n * groups) return;
    const long s = g / groups;
    const int e0 = (int)(g - s * groups) * 4;
    const uint64_t smp = sample0 + (uint64_t)s;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(e0 / 4), (uint32_t)smp, (uint32_t)(smp >> 32), 0u),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const float sigma = noise_rel * __uint_as_float(peak[s]);
    const float two32inv = 2.3283064365386963e-10f;  // 2^-32
    float z[4];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const uint32_t a = t ? w.z : w.x, b = t ? w.w : w.y;
        const float u1 = ((float)a + 1.0f) * two32inv;
        const float u2 = (float)b * two32inv;
        const float rr = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        z[2 * t] = rr * cs;
        z[2 * t + 1] = rr * sn;
    }
    const float *src = clean + s * (long)per_sample;
    __nv_bfloat16 *dst = out + s * (long)per_sample;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int e = e0 + l;
        if (e >= per_sample) break;
        const bool valid = vidx[e / C] >= 0;
        const float v = valid ? fmaf(sigma, z[l], src[e]) : 0.f;
        dst[e] = __float2bfloat16_rn(v);
    }
}

namespace {

synim_status pfail(synim_ctx *c, synim_status s, const std::string &m) {
    c->err = m;
    return s;
}

synim_status pcuda(synim_ctx *c, cudaError_t e, const char *what) {
    return pfail(c, e == cudaErrorMemoryAllocation ? SYNIM_ERR_OOM : SYNIM_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

size_t probe_smem(int k, int Cs, int NV, int NMP) {
    const size_t tile = (size_t)(k + 2) * (Cs * k + 2) * NV * NMP * 4;
    return tile + (size_t)(k + 6) * (Cs * k + 6) + (size_t)k * Cs * k + 16;
}

// Subapertures per CTA: the largest count (<= n_sub) whose tile fits the cap.
int pick_cs(int k, int n_sub, int NV, int NMP) {
    int best = 0;
    for (int cs = 1; cs <= n_sub; ++cs)
        if (probe_smem(k, cs, NV, NMP) <= kProbeSmemCap) best = cs;
    return best;
}

template <int NV>
cudaError_t set_smem(int NMP, size_t bytes) {
    auto f = NMP == 8 ? k_probe<NV, 8> : (NMP == 16 ? k_probe<NV, 16> : k_probe<NV, 32>);
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t ensure_aff(synim_ctx *c, ProbeSet *p, long long n) {
    if (n <= p->aff_cap) return cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    cudaFree(p->aff);
    p->aff = nullptr;
    p->aff_cap = 0;
    const long long cap = std::max<long long>(n, 1024);
    e = cudaMalloc(&p->aff, sizeof(ProbeAff) * cap);
    if (e == cudaSuccess) p->aff_cap = cap;
    ++c->est_gen;
    return e;
}

}  // namespace

cudaError_t probe_reserve(synim_ctx *c, long long n) { return ensure_aff(c, c->probe, n); }

// Launch the per-sample transforms and the probe kernel for n samples.
cudaError_t probe_launch(synim_ctx *c, const double *params, long long n, float *maps, float *dmaps,
                         unsigned *peak, cudaStream_t st) {
    ProbeSet *p = c->probe;
    cudaError_t e = ensure_aff(c, p, n);
    if (e != cudaSuccess) return e;
    const int d = p->dm, w = p->wfs;
    k_probe_affine<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(aff_pre(c->dmh[d], c->wh[w]), params, n,
                                                               dmaps != nullptr ? 1 : 0, p->aff);
    ProbeGeo G = p->geo;
    const bool tan = dmaps != nullptr;
    G.Cs = tan ? p->cs_tan : p->cs_fwd;
    // a few samples (a single estimate) would leave most SMs idle: narrower
    // chunks until there are about two CTAs per SM
    const long long rows = n * G.n_sub, target = 2LL * c->n_sm;
    if (rows * ((G.n_sub + G.Cs - 1) / G.Cs) < target) {
        const long long chunks = std::min<long long>(G.n_sub, (target + rows - 1) / rows);
        G.Cs = std::min(G.Cs, (int)((G.n_sub + chunks - 1) / chunks));
    }
    G.n_chunks = (G.n_sub + G.Cs - 1) / G.Cs;
    const long long blocks = n * G.n_sub * G.n_chunks;
    if (blocks > INT_MAX) return cudaErrorInvalidValue;
    const size_t sm = probe_smem(G.k, G.Cs, tan ? 5 : 1, G.NMP);
    const unsigned nb = (unsigned)blocks;
#define SYNIM_PROBE_LAUNCH(NV_, NMP_) \
    k_probe<NV_, NMP_><<<nb, kProbeThreads, sm, st>>>(G, p->aff, n, maps, NV_ == 5 ? dmaps : nullptr, peak)
    if (tan) {
        if (G.NMP == 8) SYNIM_PROBE_LAUNCH(5, 8);
        else if (G.NMP == 16) SYNIM_PROBE_LAUNCH(5, 16);
        else SYNIM_PROBE_LAUNCH(5, 32);
    } else {
        if (G.NMP == 8) SYNIM_PROBE_LAUNCH(1, 8);
        else if (G.NMP == 16) SYNIM_PROBE_LAUNCH(1, 16);
        else SYNIM_PROBE_LAUNCH(1, 32);
    }
#undef SYNIM_PROBE_LAUNCH
    return cudaGetLastError();
}

}  // namespace synim

using namespace synim;

extern "C" {

synim_status synim_probe_attach(synim_ctx *ctx, int32_t dm, int32_t wfs, const double *cmd,
                                int32_t n_modes) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (dm < 0 || dm >= ctx->n_dm || wfs < 0 || wfs >= ctx->n_wfs || !cmd || n_modes < 1 ||
        n_modes > kMaxModes)
        return pfail(ctx, SYNIM_ERR_INVALID_ARG, "probe_attach: bad pair index, cmd or n_modes (1..32)");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    struct Restore {
        int p, d;
        ~Restore() {
            if (p >= 0 && p != d) cudaSetDevice(p);
        }
    } restore{prev, ctx->device};
    const DmHost &D = ctx->dmh[dm];
    const WfsHost &W = ctx->wh[wfs];
    const int NMP = n_modes <= 8 ? 8 : (n_modes <= 16 ? 16 : 32);
    const int cs_fwd = pick_cs(W.k, W.n_sub, 1, NMP), cs_tan = pick_cs(W.k, W.n_sub, 5, NMP);
    if (cs_fwd < 1 || cs_tan < 1)
        return pfail(ctx, SYNIM_ERR_SHAPE, "probe_attach: one subaperture's tile (k = " +
                                               std::to_string(W.k) + ") exceeds the shared-memory cap");
    probe_destroy(ctx->probe);
    ctx->probe = nullptr;
    ++ctx->est_gen;
    ProbeSet *p = new ProbeSet();
    p->dm = dm;
    p->wfs = wfs;
    p->n_modes = n_modes;
    p->NMP = NMP;
    p->cs_fwd = cs_fwd;
    p->cs_tan = cs_tan;
    p->smem_fwd = probe_smem(W.k, cs_fwd, 1, NMP);
    p->smem_tan = probe_smem(W.k, cs_tan, 5, NMP);
    cudaError_t e = cudaSuccess;
    std::vector<double> hc((size_t)NMP * D.n_act, 0.0);
    std::memcpy(hc.data(), cmd, sizeof(double) * (size_t)n_modes * D.n_act);
    const size_t N2 = (size_t)(D.N + 2) * (D.N + 2);
    const size_t MM = (size_t)W.M * W.M;
    if (e == cudaSuccess) e = cudaMalloc(&p->cmd, hc.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->scr, N2 * NMP * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&p->pupil, MM);
    if (e == cudaSuccess) e = cudaMemcpy(p->cmd, hc.data(), hc.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->pupil, ctx->pupil[wfs].data(), MM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_form_screens<<<(unsigned)((N2 + 127) / 128), 128>>>(ctx->geo.dm[dm], p->cmd, NMP, p->scr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = set_smem<1>(NMP, p->smem_fwd);
    if (e == cudaSuccess) e = set_smem<5>(NMP, p->smem_tan);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        probe_destroy(p);
        return pcuda(ctx, e, "probe_attach");
    }
    ProbeGeo &G = p->geo;
    G.scr = p->scr;
    G.mask = ctx->geo.dm[dm].mask;
    G.pupil = p->pupil;
    G.vidx = ctx->geo.wfs[wfs].vidx;
    G.fac = ctx->geo.wfs[wfs].fac;
    G.N = D.N;
    G.M = W.M;
    G.k = W.k;
    G.n_sub = W.n_sub;
    G.n_modes = n_modes;
    G.NMP = NMP;
    G.C = 2 * n_modes;
    ctx->probe = p;
    return SYNIM_OK;
}

synim_status synim_probe_query(const synim_ctx *ctx, int32_t *n_sub, int32_t *n_channels,
                               uint8_t *valid) {
    if (!ctx || !ctx->probe) return SYNIM_ERR_INVALID_ARG;
    const ProbeSet *p = ctx->probe;
    if (n_sub) *n_sub = p->geo.n_sub;
    if (n_channels) *n_channels = p->geo.C;
    if (valid) {
        const std::vector<int> &v = ctx->vidx_h[p->wfs];
        for (size_t q = 0; q < v.size(); ++q) valid[q] = v[q] >= 0 ? 1 : 0;
    }
    return SYNIM_OK;
}

synim_status synim_probe_response(synim_ctx *ctx, const double *params, int64_t n, float *maps,
                                  float *d_maps, void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->probe) return pfail(ctx, SYNIM_ERR_INVALID_ARG, "probe_response: no probes attached");
    if (n < 0 || (n > 0 && (!params || !maps)))
        return pfail(ctx, SYNIM_ERR_INVALID_ARG, "probe_response: bad n, params or maps");
    if (n == 0) return SYNIM_OK;
    cudaError_t e = probe_launch(ctx, params, n, maps, d_maps, nullptr, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? SYNIM_OK : pcuda(ctx, e, "probe_response");
}

synim_status synim_probe_generate(synim_ctx *ctx, const double *params, int64_t n, uint64_t seed,
                                  uint64_t sample0, float noise_rel, uint16_t *out,
                                  void *cuda_stream) {
    if (!ctx) return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->probe) return pfail(ctx, SYNIM_ERR_INVALID_ARG, "probe_generate: no probes attached");
    if (n < 0 || (n > 0 && (!params || !out)) || !(noise_rel >= 0.f))
        return pfail(ctx, SYNIM_ERR_INVALID_ARG, "probe_generate: bad n, params, out or noise_rel");
    ProbeSet *p = ctx->probe;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int per_sample = p->geo.n_sub * p->geo.n_sub * p->geo.C;
    const long long chunk = 1024;
    cudaError_t e = cudaSuccess;
    if (p->gen_cap < chunk) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return pcuda(ctx, e, "probe_generate");
        cudaFree(p->clean);
        cudaFree(p->peak);
        p->clean = nullptr;
        p->peak = nullptr;
        p->gen_cap = 0;
        e = cudaMalloc(&p->clean, sizeof(float) * per_sample * chunk);
        if (e == cudaSuccess) e = cudaMalloc(&p->peak, sizeof(unsigned) * chunk);
        if (e != cudaSuccess) return pcuda(ctx, e, "probe_generate scratch");
        p->gen_cap = chunk;
    }
    for (long long s0 = 0; s0 < n; s0 += chunk) {
        const long long b = std::min(chunk, n - s0);
        if ((e = cudaMemsetAsync(p->peak, 0, sizeof(unsigned) * b, st)) != cudaSuccess) break;
        if ((e = probe_launch(ctx, params + 4 * s0, b, p->clean, nullptr, p->peak, st)) != cudaSuccess) break;
        const long long groups = b * ((per_sample + 3) / 4);
        k_probe_noise<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(
            p->clean, p->peak, p->geo.vidx, b, per_sample, p->geo.C, seed, sample0 + (uint64_t)s0, noise_rel,
            reinterpret_cast<__nv_bfloat16 *>(out) + s0 * per_sample);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
    }
    return e == cudaSuccess ? SYNIM_OK : pcuda(ctx, e, "probe_generate");
}

}  // extern "C"
