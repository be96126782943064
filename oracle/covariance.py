"""FP64 oracle of the tomographic covariances and the MMSE reconstructor
(Sec. 2.4) -- test infrastructure.

Only ``tests/`` and the CPU legs of ``bench.py`` may use it; the product path
never imports it.  Sec. 2.4 names the models (von Karman turbulence with r0
and L0 projected onto the modal bases, a noise covariance from the detector's
read-out noise and photon flux with LGS spot elongation, the MMSE
reconstructor after Fusco et al. 2001) but prints no formula; the readings
taken here are the standard published forms, written out:

- Phase covariance of one von Karman layer (phase in radians at the
  wavelength r0 refers to), separation r:
      B(r) = c (L0 / r0)^(5/3) x^(5/6) K_(5/6)(x),   x = 2 pi r / L0,
      c = Gamma(11/6) / (2^(5/6) pi^(8/3)) * (24/5 Gamma(6/5))^(5/6),
  B(0) = c (L0 / r0)^(5/3) Gamma(5/6) 2^(-1/6).  Its structure function
  2 (B(0) - B(r)) tends to 6.88 (r / r0)^(5/3) for r << L0 (Kolmogorov).
- A layer with C_n^2 fraction f of the integrated profile has
  r0_layer = r0 f^(-3/5) (r0^(-5/3) is linear in C_n^2).
- "Projected onto the modal basis": the basis functions (the DM's influence
  functions) are averaged over bin x bin pixel blocks of the DM grid, F
  [n_pix, n_modes]; the least-squares coefficients of the layer phase
  sampled at the binned pixel centres are a = G^-1 F^T phi, G = F^T F, so
      C_atm = G^-1 F^T C_phi F G^-1,   C_phi[p, q] = B(|p - q|).
- Shack-Hartmann centroid noise (Rousset 1999), variance of the phase
  difference across a subaperture of diameter d, per spot axis:
      photon:    (pi^2 / 2) / N_ph * (N_T / N_D)^2
      read-out:  (pi^2 / 3) * ron^2 / N_ph^2 * (N_s^2 / N_D)^2
  with N_D = (lambda / d) / pixel scale, N_T = spot FWHM / pixel scale, N_s
  the window width in pixels; the slope variance is that over d^2, times
  slope_scale^2 (slopes in radians per metre).
- LGS elongation: a subaperture at distance rho from the launch telescope
  sees the sodium layer (thickness t, altitude H, both over cos(zenith))
  elongated by eps = t rho / H^2 radians along the direction from the
  launch telescope; the spot FWHM along it is sqrt(fwhm^2 + eps^2), across
  it fwhm.  The subaperture's (x, y) block is R(theta) diag(var_along,
  var_across) R(theta)^T; different subapertures are uncorrelated.
- MMSE reconstructor, slopes y = D a + n: R = C_atm D^T (D C_atm D^T + C_n)^-1
  (equal to (D^T C_n^-1 D + C_atm^-1)^-1 D^T C_n^-1).  The IM of the library
  is D^T ([n_modes, n_slopes], one row per mode).

Pins: tests/test_oracle_covariance.py.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import gamma, kv

VK_C = gamma(11.0 / 6.0) / (2.0 ** (5.0 / 6.0) * math.pi ** (8.0 / 3.0)) * (24.0 / 5.0 * gamma(6.0 / 5.0)) ** (5.0 / 6.0)
KOLMOGOROV = 2.0 * (24.0 / 5.0 * gamma(6.0 / 5.0)) ** (5.0 / 6.0)   # 6.8839


def vk_cov(r, r0: float, L0: float):
    """von Karman phase covariance B(r) [rad^2]."""
    r = np.asarray(r, np.float64)
    x = 2.0 * math.pi * r / L0
    out = np.empty_like(x)
    small = x == 0.0
    out[small] = gamma(5.0 / 6.0) * 2.0 ** (-1.0 / 6.0)
    xs = x[~small]
    out[~small] = xs ** (5.0 / 6.0) * kv(5.0 / 6.0, xs)
    return VK_C * (L0 / r0) ** (5.0 / 3.0) * out


def vk_structure(r, r0: float, L0: float):
    return 2.0 * (vk_cov(0.0, r0, L0) - vk_cov(r, r0, L0))


def layer_r0(r0: float, frac: float) -> float:
    return r0 * frac ** (-3.0 / 5.0)


def binned_basis(ifs: np.ndarray, bin: int) -> np.ndarray:
    """F [n_pix, n_modes]: each basis function averaged over bin x bin blocks."""
    n, N, _ = ifs.shape
    if N % bin:
        raise ValueError("grid not a multiple of bin")
    Nb = N // bin
    f = np.asarray(ifs, np.float64).reshape(n, Nb, bin, Nb, bin).mean(axis=(2, 4))
    return f.reshape(n, Nb * Nb).T


def phase_cov(Nb: int, pitch_m: float, r0: float, L0: float) -> np.ndarray:
    """C_phi between the centres of an Nb x Nb grid of pitch pitch_m."""
    yy, xx = np.mgrid[0:Nb, 0:Nb]
    p = np.stack([xx.ravel(), yy.ravel()], 1).astype(np.float64) * pitch_m
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    return vk_cov(d, r0, L0)


def atm_cov(ifs: np.ndarray, dd: float, bin: int, r0: float, L0: float) -> np.ndarray:
    """C_atm = G^-1 F^T C_phi F G^-1 of the DM basis on its grid binned by bin."""
    F = binned_basis(ifs, bin)
    Nb = ifs.shape[1] // bin
    C = phase_cov(Nb, dd * bin, r0, L0)
    G = F.T @ F
    T = F.T @ C @ F
    X = np.linalg.solve(G, T)            # G^-1 T
    return np.linalg.solve(G, X.T).T     # (G^-1 (G^-1 T)^T)^T = G^-1 T G^-1


def subap_centres(n_sub: int, D: float, ros) -> np.ndarray:
    """Pupil-plane centres [nv, 2] (x, y) of the valid subapertures, row order."""
    d = D / n_sub
    nv = int(ros.max()) + 1
    out = np.zeros((nv, 2))
    for si in range(n_sub):
        for sj in range(n_sub):
            r = ros[si, sj]
            if r >= 0:
                out[r] = ((sj + 0.5) * d - D / 2.0, (si + 0.5) * d - D / 2.0)
    return out


def noise_cov(centres: np.ndarray, d: float, n_ph: float, ron: float, pix_rad: float, n_pix: int, fwhm_rad: float,
              lam: float, slope_scale: float = 1.0, lgs=None) -> np.ndarray:
    """C_n [2 nv, 2 nv] (x slopes then y slopes).  lgs = (llt_x, llt_y, na_alt,
    na_thick, zenith) or None."""
    nv = centres.shape[0]
    N_D = (lam / d) / pix_rad
    ron_var = (math.pi ** 2 / 3.0) * ron ** 2 / n_ph ** 2 * (n_pix ** 2 / N_D) ** 2

    def axis_var(fwhm):
        return (math.pi ** 2 / 2.0) / n_ph * (fwhm / pix_rad / N_D) ** 2 + ron_var

    C = np.zeros((2 * nv, 2 * nv))
    for r in range(nv):
        if lgs is None:
            blk = np.eye(2) * axis_var(fwhm_rad)
        else:
            lx, ly, H, t, z = lgs
            sec = 1.0 / math.cos(z)
            dx, dy = centres[r, 0] - lx, centres[r, 1] - ly
            rho = math.hypot(dx, dy)
            eps = (t * sec) * rho / (H * sec) ** 2
            th = math.atan2(dy, dx)
            Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
            blk = Rm @ np.diag([axis_var(math.hypot(fwhm_rad, eps)), axis_var(fwhm_rad)]) @ Rm.T
        blk = blk * slope_scale ** 2 / d ** 2
        C[r, r], C[r, nv + r], C[nv + r, r], C[nv + r, nv + r] = blk[0, 0], blk[0, 1], blk[1, 0], blk[1, 1]
    return C


def mmse(im: np.ndarray, c_atm: np.ndarray, c_noise: np.ndarray) -> np.ndarray:
    """R [n_modes, n_slopes] = C_atm D^T (D C_atm D^T + C_n)^-1, im = D^T."""
    Y = c_atm @ im
    S = im.T @ Y + c_noise
    return np.linalg.solve(S, Y.T).T
