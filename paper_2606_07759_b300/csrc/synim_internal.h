// synim_internal.h -- device-side data layout shared by the library's .cu files.
//
// HBM layout (all owned by a synim_ctx):
//   per DM     packed support windows [n_act][win_stride] FP32: each window is
//              Wp x Wp (Wp = W + 2 or W + 3, odd) with a one-pixel zero border,
//              so one 1-D bulk copy stages it into shared memory as-is; the
//              window origin (wx0, wy0) in DM pixels per actuator.
//   per sensor subaperture tables (valid rows, lit-pixel scale factors) and the
//              telescoped derivative stencil: xcode/ycode per subaperture
//              boundary line pair, and the irregular pixels where the pupil
//              edge crosses a subaperture.
//   per pair   strict-core map [M][M] (0/1) and, for the two pixel lines at
//              every subaperture boundary, one byte per (line pixel pair)
//              holding the stencil bits and both pixels' classes (zero /
//              core / ring), stored [pixel][boundary] so that the threads of
//              a warp (consecutive subapertures) read consecutive bytes; both
//              rebuilt every call because they depend on the misregistration.
#pragma once

#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "synim.h"
#include "synim_geom.h"

#define SYNIM_MAX_DM 16
#define SYNIM_MAX_WFS 16
#define SYNIM_MAX_PAIRS (SYNIM_MAX_DM * SYNIM_MAX_WFS)

namespace synim {

// Boundary-segment weight boxes (the IM kernel's dot-product form of the
// telescoped segment sums, see k_kseg): windows for them carry a KPAD-pixel
// zero border so that any box that touches an IF's support lies inside its
// window; a box spans at most KBA_MAX DM pixels along the segment and
// KBC_MAX across it; the weight tables are [KTAPS][KPS] planes per axis.
constexpr int KPAD = 9;
constexpr int KBA_MAX = 10, KBC_MAX = 4, KTAPS = KBA_MAX * KBC_MAX;
constexpr int KPS = 8192;    // plane stride (floats): n_sub (n_sub + 1) <= KPS
constexpr int KF_MAX_K = 12; // largest subaperture side (pixels) given weight tables
constexpr int KNC = 5;       // weight-box components: the value and its four misregistration tangents
// segment flags (bits 24-31 of the origin word): no core sample in the box,
// A and B differ (kwb holds B), resample pixel by pixel, ring pixels listed
// in kring (repaired by the lane that takes the segment)
enum { KF_NOCORE = 1, KF_ASYM = 2, KF_FALLBACK = 4, KF_RING = 8 };

struct DevDM {
    const float *win;     // [n_act][win_stride]
    const int *org;       // [n_act][2] window origin (wx0, wy0), DM pixels
    const uint8_t *mask;  // [N][N] 0/1, or nullptr = all ones
    const uint8_t *mcls;  // [(N+1)][(N+1)] taps of the 3x3 cells around cell (x-1, y-1):
                          // 0 all zero, 1 all one, 2 mixed (interior test of the core)
    int n_act, N, W, Wp;
    int win_stride;       // floats per packed window, multiple of 4 (16-byte bulk copies)
    const float *winK;    // [n_act][strideK] the same windows with a KPAD-pixel zero border, or nullptr
    int WpK, strideK;
};

struct DevWFS {
    const uint8_t *xcode;  // [(n_sub + 1)][M]: column pair (b k - 1, b k), row i
    const uint8_t *ycode;  // [(n_sub + 1)][M]: row pair (b k - 1, b k), column j
    const int *irr_pix;    // [n_irr] (i << 16) | j, grouped by subaperture (row-major)
    const int8_t *irr_w;   // [n_irr][2] weights (wx, wy) in {-1, 0, 1}
    const int *irr_sub;    // [n_sub * n_sub + 1] first entry of each subaperture
    const int *irr_sr;     // [n_sub * n_sub * k + 1] first entry of each (subaperture, pixel row)
    const int4 *irrc;      // subapertures that have irregular pixels: (sj, e0, e1, 0)
    const int *irrc_row;   // [n_sub + 1] first candidate of each subaperture row
    const float *fac;      // [nv] slope_scale / (2 dw lit)
    const int *vsub;       // [nv] (si << 16) | sj of each valid row
    const short *vsj;      // [nv + 4] sj of each valid row (padded with -1: 4-row loads)
    const int *vidx;       // [n_sub * n_sub] valid row of each subaperture, -1 if invalid
    const int *vrow;       // [n_sub + 1] first valid row of each subaperture row
    // the pupil-edge entries by 16 x 16 pixel tiles of each subaperture (k > 32 only):
    // tile (si, sj, ti, tj) at ((si n_sub + sj) tl_n + ti) tl_n + tj, its entries
    // [tl_start[tile], tl_start[tile + 1]) of tl_pix / tl_w (as irr_pix / irr_w)
    const int *tl_start;
    const int *tl_pix;
    const int8_t *tl_w;
    int tl_n;              // tiles per subaperture side, 0 = no tiles
    int n_sub, M, k, nv, CH;
    int n_irr;             // entries of irr_pix (an upper bound where the tables are built on the device)
};

// Edge tables of the telescoping-sum engine (Sec. 2.2), per sensor.  Each
// event is one half-pixel end of a lit pixel run inside a valid subaperture,
// packed as (end << 31) | ((2 i + 1 + e_i) << 16) | (axis << 15) |
// (credit << 14) | (2 j + 1 + e_j), with (e_i, e_j) the half-pixel offset
// doubled (-1, 0 or 1), axis 0 for runs along x (pixel rows) and 1 along y
// (pixel columns), end = 1 for the run's last pixel (+phi), 0 for its first
// (-phi), and credit = 1 for a run start on the left (x) or upper (y)
// boundary whose point is also the end of a run of the valid neighbour
// there: that neighbour's event is not stored, and this one adds +phi to
// the neighbour's sum.  Grouped by valid row.
struct DevTele {
    const int *es;       // [nv + 1] first event of each valid row
    const int *ev;       // events
    const float *fac;    // [nv] slope_scale / (dw lit)
    const int *vfirst;   // [n_sub][n_sub + 1] valid row of the first valid subaperture at
                         // or right of column sj in row si (vrow[si + 1] if none)
    int lanes;           // lanes that share one subaperture's events (1 .. 32, a power of 2)
    int n_ev;            // entries of ev
};

struct TeleSet {
    DevTele w[SYNIM_MAX_WFS];
};

// Per (DM, sensor) pair, rewritten by the host every call.
struct DevPair {
    double A[4], b[2];   // DM pixel = A (j, i) + b
    double Ai[4];        // inverse of A
    double dA[16], db[8];  // d(A, b)/dp_k, p = (shift x px, shift y px, rot deg, mag)
    float Ahi[4], Alo[4], bhi[2], blo[2];  // A, b as float pairs (compensated origins)
    float Aif[4];        // inverse of A, float (pixel boxes, with a margin)
    uint8_t *xcc, *ycc;  // [M][n_sub + 1] boundary-line bytes (see above)
    int vec4;            // output columns are 16-byte aligned and a multiple of 4 floats
    float *im;           // output [n_act][2 nv] or nullptr (skip)
    float *dim[4];       // tangent outputs or nullptr
    const float *gim;    // VJP input [n_act][2 nv] or nullptr
    uint8_t *pst;        // [M][M] strict core (0/1)
    // Boundary-segment weight boxes, per axis (0: x segments, index si (n_sub + 1) + b;
    // 1: y segments, index b n_sub + sj), rebuilt every call by k_kseg when kf != 0:
    // korg = box origin (gx, gy) in DM pixels as signed 12-bit fields (bits 0-11,
    // 12-23) and the segment flags (bits 24-31); kw / kwb = [KNC][KTAPS][KPS] weights of
    // the A / B sums (kwb only for KF_ASYM segments), component q (0 the value,
    // 1..4 its tangents) and tap (along a, across c) at plane q KTAPS + a KBC_MAX
    // + c; kshape = (ori << 8) | (BA << 4) | BC: box of BA x BC taps,
    // along the DM's y (ori 0) or x (ori 1) axis.
    // kring: bit 2 q + t set when line pixel t of pair q of the segment is a
    // ring pixel with a stencil bit (KF_RING segments only)
    int kf;
    int kcomp;           // weight-box components built this call: 1 (values) or KNC (values and tangents)
    int kshape[2];
    int *korg[2], *kring[2];
    float *kw[2], *kwb[2];
};

struct Geo {
    DevDM dm[SYNIM_MAX_DM];
    DevWFS wfs[SYNIM_MAX_WFS];
    int n_dm, n_wfs, n_items;
    int order_dm[SYNIM_MAX_DM];         // DM processed at each position (costliest first)
    int order_start[SYNIM_MAX_DM + 1];  // item prefix in processing order
    // k_imk's column order within each DM: the actuators on the sensors
    // wfs_order[0 .. n_wfs_a) (subapertures of at most 32 pixels), then the
    // actuators on the others, so that a CTA's warps take columns of one kind
    int wfs_order[SYNIM_MAX_WFS];
    int n_wfs_a;
    int seg_floats;      // per-warp shared-memory buffer of the IM kernel (floats)
    int seg_lanes;       // lanes per boundary segment for k <= 32 (2, 4 or 8); 0 = by k
};

enum { ERR_TIMEOUT = 1, ERR_ARENA = 2, ERR_BOUNDS = 4 };

// Debug builds (-DSYNIM_DEBUG_BOUNDS) test the index of each global and
// shared-memory access of the IM kernels against its buffer: an index
// outside sets ERR_BOUNDS in the context's error flag (surfaced by
// synim_im_check) and the access is skipped.  Release builds compile the
// tests away (the error pointer is not even evaluated).
#ifdef SYNIM_DEBUG_BOUNDS
#define SYNIM_IDX_OK(cond, errp) ((cond) ? true : (atomicOr((errp), ERR_BOUNDS), false))
#else
#define SYNIM_IDX_OK(cond, errp) true
#endif

enum Mode { MODE_FWD = 0, MODE_TAN = 1, MODE_VJP = 2 };

// Host helpers (synim_api.cu).
bool invert2(const double A[4], double Ai[4]);
int largest_divisor_le(int k, int cap);
// Per-warp buffer (floats) of the IM kernel for the pair: one box row's
// boundary segments and pupil-edge sums, NV values each.
long long seg_need(const DmHost &D, const WfsHost &W, const double Ai[4], int NV);
void split_pair(DevPair &P);  // float pairs of A, b and the float inverse
void clear_create_error();         // synim_api.cu (no allocation)
void set_global_error(const std::string &m);   // message of synim_last_error(NULL)
// Valid-row tables of sensor w of a context (device pointers): vsub[r] =
// (si << 16) | sj of valid row r; returns nv.
int ctx_valid_rows(const synim_ctx *ctx, int w, const int **vsub, int *n_sub);
const char *noalloc_last_error();  // synim_noalloc.cu

// Launch wrappers (synim_kernels.cu).
// box: 4 * n_act + 1 ints (the extra one is scratch for the DM peak)
cudaError_t launch_support(const float *cube, int n_act, int N, float eps, int *box,
                           cudaStream_t s);
// pad: zero border of the packed windows (1, or KPAD for the weight-box windows)
cudaError_t launch_pack(const float *cube, int n_act, int N, const int *org, int W, int Wp,
                        int stride, float *win, cudaStream_t s, int pad = 1);
cudaError_t launch_mcls(const uint8_t *mask, int N, uint8_t *mcls, cudaStream_t s);
cudaError_t launch_pst(const Geo &g, const DevPair *pairs, int max_mm, int max_lines, cudaStream_t s);
// Boundary-segment weight boxes of the pairs with kf != 0 (after launch_pst),
// ncomp components (1, or KNC with the tangents) in parallel.
cudaError_t launch_kseg(const Geo &g, const DevPair *pairs, int max_seg, int ncomp, cudaStream_t s);
// Box shape code of one axis for the composite A and subaperture side k, or -1.
int kseg_shape(const double A[4], int k, int axis);
// dynamic shared memory of the IM kernels: one seg_floats buffer per warp
size_t im_smem_bytes(const Geo &g, int threads);
cudaError_t im_prepare(int mode, int threads, size_t smem, int *blocks_per_sm);
// gp: MODE_VJP only, the per-column partials [n_items * n_wfs][4] that
// launch_vjp_reduce sums per pair into grad_p [n_pairs][4].
// k_im<mode> (grid CTAs, none if 0) when no pair has weight boxes, else
// k_imk<mode> over every column (kgrid CTAs).
cudaError_t launch_im(int mode, const Geo &g, const DevPair *pairs, int *err, double *gp, int grid, int threads,
                      size_t smem, cudaStream_t s, int kgrid = 0);
cudaError_t launch_vjp_reduce(const Geo &g, const double *part, double *gp, cudaStream_t s);
// The telescoping-sum IM kernel: one warp per (actuator, sensor) column, a
// per-warp buffer of cap4 float4 subaperture sums (a chunk of box rows and
// the row above it; cap4 >= 2 n_sub).
size_t tele_smem_bytes(int threads, int cap4);
cudaError_t launch_tele(const Geo &g, const TeleSet &t, const DevPair *pairs, int cap4, int *err, int grid,
                        int threads, cudaStream_t s);

// Dense FP32-accurate linear algebra on tcgen05 (synim_dense.cu); row-major
// matrices with leading dimensions.  C = beta C + alpha A B with A(m, k) =
// A[m lda + k], B(k, n) = B[n ldb + k] or, b_kn, B[k ldb + n]; lower: only
// the lower triangle (n <= m) of C is written.  *err gets ERR_TIMEOUT if a
// bounded tensor-core wait gives up.
cudaError_t dense_gemm(const float *A, long lda, const float *B, long ldb, bool b_kn, float *C, long ldc, int M,
                       int N, int K, float alpha, float beta, bool lower, int *err, cudaStream_t s);
int dense_blocks(int n);   // diagonal blocks of the blocked factorization (128 rows each)
cudaError_t dense_potrf(float *S, long lds, int n, float *linvs, float *work, int *info, int *err, cudaStream_t s);
cudaError_t dense_posolve_right(const float *S, long lds, int n, const float *linvs, float *Y, long ldy, int m,
                                float *work, int *err, cudaStream_t s);

struct ProbeSet;   // synim_probe.cu
void probe_destroy(ProbeSet *p);
// Probe responses of n samples (params device [n][4]): maps [n][per_sample],
// tangents dmaps [4][n][per_sample] when not null, per-sample peak |slope|
// (float bits) when peak is not null.
cudaError_t probe_launch(synim_ctx *c, const double *params, long long n, float *maps, float *dmaps,
                         unsigned *peak, cudaStream_t st);
int probe_per_sample(const ProbeSet *p);   // n_sub^2 x channels
// Grow the probe scratch for n samples outside any stream capture.
cudaError_t probe_reserve(synim_ctx *c, long long n);
struct EstState;   // synim_estimate.cu
void est_destroy(EstState *e);
struct CnnState;   // synim_cnn.cu
void cnn_destroy(CnnState *s);

constexpr int NSLOT = 4;
constexpr int NPROF = 256;

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ev_start = nullptr, ev_stop = nullptr;  // event-record nodes (profiling)
};

}  // namespace synim

// One context (opaque to callers): everything create() packed, the per-call
// parameter slots, captured graphs and profiling events.
struct synim_ctx {
    int device = 0, n_sm = 0, n_dm = 0, n_wfs = 0;
    synim::DmHost dmh[SYNIM_MAX_DM];
    synim::WfsHost wh[SYNIM_MAX_WFS];
    synim::Geo geo{};
    std::vector<void *> dev_allocs;
    int64_t mem_cap = 0;      // device bytes create may take (0 = no cap)
    int slope_engine = 0;     // SYNIM_ENGINE_NUMERICAL or SYNIM_ENGINE_TELESCOPING
    synim::TeleSet tele{};
    size_t mem_used = 0;      // device bytes taken by create so far
    std::vector<void *> host_allocs;
    // Two sets of per-call tables (pair records, core maps, boundary-line
    // classes, weight boxes), taken by alternate calls: a call's class kernels
    // and weight boxes run on the context's prep stream and overlap the
    // previous call's IM kernel on the caller's stream.  ev_prep[t]: set t is
    // built; ev_im[t]: the IM launch that read set t has finished.
    synim::DevPair *d_pairs[2] = {};
    int tset = 0;
    cudaStream_t prep = nullptr;
    cudaEvent_t ev_prep[2] = {}, ev_im[2] = {};
    bool im_used[2] = {};
    synim::DevPair *h_pairs[synim::NSLOT] = {};
    cudaEvent_t slot_ev[synim::NSLOT] = {};
    bool slot_used[synim::NSLOT] = {};
    int slot = 0;
    int *d_err = nullptr, *h_err = nullptr;
    double *d_gp = nullptr;     // grad_p [n_pairs][4] of the adjoint
    double *d_vjp_part = nullptr;   // per-column adjoint partials [n_items * n_wfs][4]
    long long pst_off[SYNIM_MAX_PAIRS] = {};
    long long line_off[SYNIM_MAX_PAIRS] = {};
    uint8_t *d_pst[2] = {}, *d_lines[2] = {};
    // boundary-segment weight boxes per table set and pair (nullptr where the
    // sensor's subapertures are too large for them): origins and ring lists
    // [2][2][KPS], weights [2][KNC][KTAPS][KPS] for A and for B
    int *k_org[2][SYNIM_MAX_PAIRS] = {};
    float *k_w[2][SYNIM_MAX_PAIRS] = {}, *k_wb[2][SYNIM_MAX_PAIRS] = {};
    int max_mm = 0, max_lines = 0;
    int threads = 256, ctas_per_sm = 0;
    bool autotune = false;
    bool tuned[3] = {false, false, false};
    int tune_threads[3] = {0, 0, 0}, tune_lanes[3] = {0, 0, 0};
    float tune_ms[3] = {0.f, 0.f, 0.f};
    bool use_graph = true;
    int seg_floats = 0;
    std::map<std::tuple<int, size_t, int, int>, synim::GraphEntry> graphs;
    cudaStream_t cap = nullptr;
    bool profile = false;
    cudaEvent_t prof_a[synim::NPROF] = {}, prof_b[synim::NPROF] = {};
    unsigned long long prof_head = 0, prof_tail = 0;
    double prof_acc_ms = 0.0;
    int prof_acc_n = 0;
    std::string err;
    // host copies of each sensor's pupil and valid-row index (probe responses)
    std::vector<uint8_t> pupil[SYNIM_MAX_WFS];
    std::vector<int> vidx_h[SYNIM_MAX_WFS];
    synim::ProbeSet *probe = nullptr;
    synim::EstState *est = nullptr;
    synim::CnnState *cnn = nullptr;
    // bumped whenever a buffer or setting the estimator's captured graphs
    // hold changes (probe attach or scratch growth, network init, GN config)
    unsigned long long est_gen = 0;
};
