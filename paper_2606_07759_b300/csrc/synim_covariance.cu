// synim_covariance.cu -- tomographic covariances and the MMSE reconstructor
// (Sec. 2.4: von Karman C_atm projected onto a modal basis, C_noise from
// detector parameters with LGS spot elongation, MMSE after Fusco et al.).
//
// Readings (the paper names the models without formulas):
//   B(r)   = c (L0/r0)^(5/3) x^(5/6) K_5/6(x), x = 2 pi r / L0, the von Karman
//            phase covariance, c = Gamma(11/6)/(2^(5/6) pi^(8/3)) (24/5
//            Gamma(6/5))^(5/6); K_5/6 from its integral representation
//            K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt by the
//            trapezoidal rule (exponentially convergent for this integrand),
//            evaluated once per distinct pixel separation on the device (FP64).
//   C_atm  = G^-1 F^T C_phi F G^-1, F the DM basis averaged over bin x bin
//            pixel blocks (columns = modes), G = F^T F: the covariance of the
//            least-squares coefficients of the layer phase sampled at the
//            binned pixel centres.
//   C_n    = per valid subaperture, R(theta) diag(v_along, v_across)
//            R(theta)^T / d^2 * slope_scale^2 with the Shack-Hartmann photon
//            and read-out centroid variances (Rousset) of a spot elongated
//            by eps = t rho / H^2 along the direction from the launch
//            telescope (LGS), or round (NGS).
//   R      = C_atm D^T (D C_atm D^T + C_n)^-1 with D^T = the IM (one row per
//            mode).
// Kernels: k_bin_basis (F^T from the packed windows), k_vk_fill (C_phi from
// the separation table), k_noise_blocks, k_transpose; the contractions and
// the SPD solves are the tensor-core routines of synim_dense.cu.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "synim.h"
#include "synim_internal.h"

namespace synim {

namespace {

// x^nu K_nu(x) (x >= 0, nu in (0, 1)) by the trapezoidal rule on
// int_0^inf exp(-x cosh t) cosh(nu t) dt with step h, up to where the
// integrand is below 1e-300 of its value at t = 0; one thread per pixel separation
// (dx, dy) of the binned grid: tab[dy Nb + dx] = amp x^nu K_nu(x), x = 2 pi
// pitch |(dx, dy)| / L0, in FP64.
__global__ void k_vk_table(int Nb, double pitch, double L0, double amp, double nu, float *__restrict__ tab) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Nb * Nb) return;
    const int dy = q / Nb, dx = q - dy * Nb;
    const double x = 2.0 * 3.14159265358979323846 * pitch * sqrt((double)dx * dx + (double)dy * dy) / L0;
    double v;
    if (x <= 0.0) {
        v = tgamma(nu) * pow(2.0, nu - 1.0);
    } else {
        const double h = 0.02;
        double s = 0.5 * exp(-x);
        for (int i = 1; i < 200000; ++i) {
            const double t = i * h;
            const double ct = cosh(t);
            if (-x * ct + nu * t + x < -700.0 && t > 1.0) break;
            s += exp(-x * ct) * cosh(nu * t);
        }
        v = pow(x, nu) * h * s;
    }
    tab[q] = (float)(amp * v);
}

double vk_const() {
    const double pi = 3.14159265358979323846;
    return std::tgamma(11.0 / 6.0) / (std::pow(2.0, 5.0 / 6.0) * std::pow(pi, 8.0 / 3.0)) *
           std::pow(24.0 / 5.0 * std::tgamma(6.0 / 5.0), 5.0 / 6.0);
}

// F^T[a][p] = mean over the bin x bin block of binned pixel p (row-major on
// the Nb x Nb grid) of IF_a, read from the packed window (zero outside it).
__global__ void k_bin_basis(const DevDM D, int bin, int Nb, float *__restrict__ Ft) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long npix = (long)Nb * Nb;
    if (q >= (long)D.n_act * npix) return;
    const int a = (int)(q / npix);
    const int p = (int)(q - (long)a * npix);
    const int py = p / Nb, px = p - py * Nb;
    const int wx0 = D.org[2 * a], wy0 = D.org[2 * a + 1];
    const float *win = D.win + (size_t)a * D.win_stride;
    float s = 0.f;
    for (int v = 0; v < bin; ++v) {
        const int ly = py * bin + v - wy0 + 1;   // padded-window row
        if (ly < 0 || ly >= D.Wp) continue;
        for (int u = 0; u < bin; ++u) {
            const int lx = px * bin + u - wx0 + 1;
            if (lx >= 0 && lx < D.Wp) s += win[ly * D.Wp + lx];
        }
    }
    Ft[q] = s / (float)(bin * bin);
}

// C_phi[p][q] = B(|p - q|) from tab[|dy| Nb + |dx|].
__global__ void k_vk_fill(const float *__restrict__ tab, int Nb, float *__restrict__ C) {
    const long npix = (long)Nb * Nb;
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npix * npix) return;
    const int i = (int)(q / npix), j = (int)(q - (long)i * npix);
    const int dy = abs(i / Nb - j / Nb), dx = abs(i % Nb - j % Nb);
    C[q] = tab[dy * Nb + dx];
}

// Transpose r x c (row-major, lds) into c x r (ldd) through shared tiles.
__global__ void k_transpose(const float *__restrict__ src, long lds, float *__restrict__ dst, long ldd, int r, int c) {
    __shared__ float t[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int y = y0 + k, x = x0 + threadIdx.x;
        if (y < r && x < c) t[k][threadIdx.x] = src[(long)y * lds + x];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int x = x0 + k, y = y0 + threadIdx.x;   // dst row x, column y
        if (x < c && y < r) dst[(long)x * ldd + y] = t[threadIdx.x][k];
    }
}

// (C + C^T) / 2 of an n x n matrix into dst (both row-major, ld n).
__global__ void k_symmetrize(const float *__restrict__ C, float *__restrict__ dst, int n) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)n * n) return;
    const int i = (int)(q / n), j = (int)(q - (long)i * n);
    dst[q] = 0.5f * (C[q] + C[(long)j * n + i]);
}

// The 2 x 2 block of valid row r: xx, xy, yy at (r, r), (r, nv + r),
// (nv + r, r), (nv + r, nv + r) of the zeroed 2 nv x 2 nv matrix.
__global__ void k_noise_blocks(const float *__restrict__ blk, int nv, float *__restrict__ C) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nv) return;
    const long n2 = 2L * nv;
    C[(long)r * n2 + r] = blk[3 * r];
    C[(long)r * n2 + nv + r] = blk[3 * r + 1];
    C[(long)(nv + r) * n2 + r] = blk[3 * r + 1];
    C[(long)(nv + r) * n2 + nv + r] = blk[3 * r + 2];
}

cudaError_t transpose(const float *src, long lds, float *dst, long ldd, int r, int c, cudaStream_t s) {
    dim3 grid((unsigned)((c + 31) / 32), (unsigned)((r + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(src, lds, dst, ldd, r, c);
    return cudaGetLastError();
}

}  // namespace

}  // namespace synim

using namespace synim;

namespace {

synim_status cv_fail(synim_ctx *c, synim_status st, const std::string &m) {
    if (c) c->err = m;
    else synim::set_global_error(m);
    return st;
}

struct CvScratch {
    std::vector<void *> p;
    ~CvScratch() {
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

unsigned blocks_for(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" synim_status synim_atm_covariance(synim_ctx *ctx, int32_t dm, int32_t bin, double r0_m, double L0_m,
                                             float *c_atm, void *cuda_stream) {
    if (!ctx || dm < 0 || dm >= ctx->n_dm || bin < 1 || !(r0_m > 0) || !(L0_m > 0) || !c_atm)
        return SYNIM_ERR_INVALID_ARG;
    ctx->err.clear();
    const DmHost &H = ctx->dmh[dm];
    const DevDM &D = ctx->geo.dm[dm];
    if (H.N % bin != 0) return cv_fail(ctx, SYNIM_ERR_SHAPE, "atm_covariance: the DM grid is not a multiple of bin");
    const int Nb = H.N / bin, na = H.n_act;
    const long npix = (long)Nb * Nb;
    if (npix > 46340) return cv_fail(ctx, SYNIM_ERR_SHAPE, "atm_covariance: more than 46340 binned pixels (raise bin)");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // separation table (device, FP64): B at (dx, dy) pixel offsets of pitch dd bin
    const double c = vk_const();
    const double amp = c * std::pow(L0_m / r0_m, 5.0 / 3.0), pitch = H.dd * bin;
    const size_t ntab = (size_t)Nb * Nb;
    CvScratch sc;
    float *d_tab = nullptr, *Ft = nullptr, *C = nullptr, *W = nullptr, *T = nullptr, *G = nullptr, *X = nullptr;
    float *linvs = nullptr, *work = nullptr;
    int *flags = nullptr;
    cudaError_t e = sc.alloc(&d_tab, ntab);
    if (e == cudaSuccess) e = sc.alloc(&Ft, (size_t)na * npix);
    if (e == cudaSuccess) e = sc.alloc(&C, (size_t)npix * npix);
    if (e == cudaSuccess) e = sc.alloc(&W, (size_t)npix * na);
    if (e == cudaSuccess) e = sc.alloc(&T, (size_t)na * na);
    if (e == cudaSuccess) e = sc.alloc(&G, (size_t)na * na);
    if (e == cudaSuccess) e = sc.alloc(&X, (size_t)na * na);
    if (e == cudaSuccess) e = sc.alloc(&linvs, (size_t)dense_blocks(na) * 128 * 128);
    if (e == cudaSuccess) e = sc.alloc(&work, (size_t)na * 128);
    if (e == cudaSuccess) e = sc.alloc(&flags, 2);
    if (e != cudaSuccess) return cv_fail(ctx, SYNIM_ERR_OOM, "atm_covariance: scratch");
    e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) {
        k_vk_table<<<blocks_for((long)ntab, 128), 128, 0, st>>>(Nb, pitch, L0_m, amp, 5.0 / 6.0, d_tab);
        k_bin_basis<<<blocks_for((long)na * npix, 256), 256, 0, st>>>(D, bin, Nb, Ft);
        k_vk_fill<<<blocks_for(npix * npix, 256), 256, 0, st>>>(d_tab, Nb, C);
        e = cudaGetLastError();
    }
    int *err = flags + 1;
    // W = C_phi F, T = F^T W, G = F^T F
    if (e == cudaSuccess)
        e = dense_gemm(C, npix, Ft, npix, false, W, na, (int)npix, na, (int)npix, 1.f, 0.f, false, err, st);
    if (e == cudaSuccess) e = dense_gemm(Ft, npix, W, na, true, T, na, na, na, (int)npix, 1.f, 0.f, false, err, st);
    if (e == cudaSuccess) e = dense_gemm(Ft, npix, Ft, npix, false, G, na, na, na, (int)npix, 1.f, 0.f, false, err, st);
    // C_atm = G^-1 T G^-1: X = T G^-1, then (X^T) G^-1 = G^-1 T G^-1
    if (e == cudaSuccess) e = dense_potrf(G, na, na, linvs, work, flags, err, st);
    if (e == cudaSuccess) e = dense_posolve_right(G, na, na, linvs, T, na, na, work, err, st);
    if (e == cudaSuccess) e = transpose(T, na, X, na, na, na, st);
    if (e == cudaSuccess) e = dense_posolve_right(G, na, na, linvs, X, na, na, work, err, st);
    if (e == cudaSuccess) {
        k_symmetrize<<<blocks_for((long)na * na, 256), 256, 0, st>>>(X, c_atm, na);
        e = cudaGetLastError();
    }
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cv_fail(ctx, SYNIM_ERR_CUDA, std::string("atm_covariance: ") + cudaGetErrorString(e));
    if (h[1]) return cv_fail(ctx, SYNIM_ERR_TIMEOUT, "atm_covariance: a tensor-core wait gave up");
    if (h[0]) return cv_fail(ctx, SYNIM_ERR_NOT_CONVERGED, "atm_covariance: the basis Gram matrix is singular at this bin");
    return SYNIM_OK;
}

extern "C" synim_status synim_noise_covariance(synim_ctx *ctx, int32_t wfs, const synim_noise_desc *nd,
                                               float *c_noise, void *cuda_stream) {
    if (!ctx || wfs < 0 || wfs >= ctx->n_wfs || !nd || !c_noise) return SYNIM_ERR_INVALID_ARG;
    if (!(nd->n_photons > 0) || !(nd->ron_e >= 0) || !(nd->pixel_scale_rad > 0) || nd->n_pix < 1 ||
        !(nd->fwhm_rad > 0) || !(nd->wavelength_m > 0) ||
        (nd->lgs && (!(nd->na_altitude_m > 0) || !(nd->na_thickness_m >= 0) || !(std::cos(nd->zenith_rad) > 0))))
        return cv_fail(ctx, SYNIM_ERR_INVALID_ARG, "noise_covariance: invalid noise descriptor");
    ctx->err.clear();
    const WfsHost &W = ctx->wh[wfs];
    const int nv = W.nv, n = W.n_sub;
    const double d = W.D / n, pi = 3.14159265358979323846;
    const double N_D = (nd->wavelength_m / d) / nd->pixel_scale_rad;
    const double ron_var = (pi * pi / 3.0) * nd->ron_e * nd->ron_e / (nd->n_photons * nd->n_photons) *
                           std::pow((double)nd->n_pix * nd->n_pix / N_D, 2.0);
    auto axis_var = [&](double fwhm) {
        return (pi * pi / 2.0) / nd->n_photons * std::pow(fwhm / nd->pixel_scale_rad / N_D, 2.0) + ron_var;
    };
    const double sc2 = W.scale * W.scale / (d * d);
    std::vector<float> blk((size_t)3 * nv);
    const std::vector<int> &vidx = ctx->vidx_h[wfs];
    for (int si = 0; si < n; ++si)
        for (int sj = 0; sj < n; ++sj) {
            const int r = vidx[(size_t)si * n + sj];
            if (r < 0) continue;
            double xx, xy, yy;
            if (!nd->lgs) {
                xx = yy = axis_var(nd->fwhm_rad);
                xy = 0.0;
            } else {
                const double sec = 1.0 / std::cos(nd->zenith_rad);
                const double cx = (sj + 0.5) * d - W.D / 2.0, cy = (si + 0.5) * d - W.D / 2.0;
                const double dx = cx - nd->llt_xy_m[0], dy = cy - nd->llt_xy_m[1];
                const double rho = std::hypot(dx, dy);
                const double Hs = nd->na_altitude_m * sec;
                const double eps = nd->na_thickness_m * sec * rho / (Hs * Hs);
                const double va = axis_var(std::hypot(nd->fwhm_rad, eps)), vc = axis_var(nd->fwhm_rad);
                const double th = std::atan2(dy, dx), c = std::cos(th), s = std::sin(th);
                xx = c * c * va + s * s * vc;
                yy = s * s * va + c * c * vc;
                xy = c * s * (va - vc);
            }
            blk[3 * (size_t)r] = (float)(xx * sc2);
            blk[3 * (size_t)r + 1] = (float)(xy * sc2);
            blk[3 * (size_t)r + 2] = (float)(yy * sc2);
        }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CvScratch sc;
    float *d_blk = nullptr;
    cudaError_t e = sc.alloc(&d_blk, blk.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_blk, blk.data(), blk.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c_noise, 0, sizeof(float) * 4 * (size_t)nv * nv, st);
    if (e == cudaSuccess) {
        k_noise_blocks<<<blocks_for(nv, 128), 128, 0, st>>>(d_blk, nv, c_noise);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cv_fail(ctx, SYNIM_ERR_CUDA, std::string("noise_covariance: ") + cudaGetErrorString(e));
    return SYNIM_OK;
}

extern "C" synim_status synim_mmse_reconstructor(int32_t n_modes, int32_t n_slopes, const float *im, const float *c_atm,
                                                 const float *c_noise, float *R, void *cuda_stream) {
    synim::clear_create_error();
    if (n_modes < 1 || n_slopes < 1 || !im || !c_atm || !c_noise || !R)
        return cv_fail(nullptr, SYNIM_ERR_INVALID_ARG, "mmse_reconstructor: invalid sizes or pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nm = n_modes, ns = n_slopes;
    CvScratch sc;
    float *imT = nullptr, *S = nullptr, *linvs = nullptr, *work = nullptr;
    int *flags = nullptr;
    cudaError_t e = sc.alloc(&imT, (size_t)ns * nm);
    if (e == cudaSuccess) e = sc.alloc(&S, (size_t)ns * ns);
    if (e == cudaSuccess) e = sc.alloc(&linvs, (size_t)dense_blocks(ns) * 128 * 128);
    if (e == cudaSuccess) e = sc.alloc(&work, (size_t)std::max(ns, nm) * 128);
    if (e == cudaSuccess) e = sc.alloc(&flags, 2);
    if (e != cudaSuccess) return cv_fail(nullptr, SYNIM_ERR_OOM, "mmse_reconstructor: scratch");
    int *err = flags + 1;
    e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st);
    // Y = C_atm D^T into R (n_modes x n_slopes); S = D C_atm D^T + C_n
    if (e == cudaSuccess) e = dense_gemm(c_atm, nm, im, ns, true, R, ns, nm, ns, nm, 1.f, 0.f, false, err, st);
    if (e == cudaSuccess) e = transpose(im, ns, imT, nm, nm, ns, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S, c_noise, sizeof(float) * (size_t)ns * ns, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = dense_gemm(imT, nm, R, ns, true, S, ns, ns, ns, nm, 1.f, 1.f, false, err, st);
    // R = Y S^-1
    if (e == cudaSuccess) e = dense_potrf(S, ns, ns, linvs, work, flags, err, st);
    if (e == cudaSuccess) e = dense_posolve_right(S, ns, ns, linvs, R, ns, nm, work, err, st);
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cv_fail(nullptr, SYNIM_ERR_CUDA, std::string("mmse_reconstructor: ") + cudaGetErrorString(e));
    if (h[1]) return cv_fail(nullptr, SYNIM_ERR_TIMEOUT, "mmse_reconstructor: a tensor-core wait gave up");
    if (h[0]) return cv_fail(nullptr, SYNIM_ERR_NOT_CONVERGED, "mmse_reconstructor: D C_atm D^T + C_n is not positive definite");
    return SYNIM_OK;
}
