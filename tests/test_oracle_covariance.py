"""Pins of the covariance / MMSE oracle (oracle/covariance.py, Sec. 2.4).

- von Karman covariance: its structure function's leading small-separation
  term is the Kolmogorov law 6.8839 (r / r0)^(5/3) (the definition of r0);
  the phase variance is c Gamma(5/6) 2^(-1/6) (L0 / r0)^(5/3); the
  covariance is a positive definite function.
- Layers: structure functions of C_n^2 fractions add up to the total.
- Basis projection: a pixel basis (one unit impulse per pixel, bin 1) gives
  C_phi itself; a change of basis F' = F M gives M^-1 C M^-T (catches a
  transposed or missing G^-1); a scaled basis scales C by 1 / alpha^2.
- Noise: the photon-noise value of a diffraction-limited spot, the read-out
  term, the elongation geometry (a spot elongated along x, one at 45 degrees
  with equal diagonal terms and a positive x-y term, and the same
  elongation for a launch telescope mirrored through the subaperture).
- MMSE: the two textbook forms agree; with no noise and an invertible square
  D the reconstructor is D^-1; with overwhelming noise it vanishes.
"""
import math

import numpy as np
import pytest

from oracle import covariance as CV


def test_structure_function_has_the_kolmogorov_leading_term():
    r0, L0 = 0.15, 25.0
    assert abs(CV.KOLMOGOROV - 6.8839) < 1e-4
    # D(r) = a x^(5/3) + b x^2 + O(x^(11/3)), x = 2 pi r / L0: two separations
    # eliminate the x^2 term
    r1 = 1e-3 * L0 / (2 * math.pi)
    r2 = 2 * r1
    x1, x2 = 2 * math.pi * r1 / L0, 2 * math.pi * r2 / L0
    D1, D2 = CV.vk_structure(r1, r0, L0), CV.vk_structure(r2, r0, L0)
    M = np.array([[x1 ** (5 / 3), x1 ** 2], [x2 ** (5 / 3), x2 ** 2]])
    a, _ = np.linalg.solve(M, [D1, D2])
    kolmo = CV.KOLMOGOROV * (L0 / (2 * math.pi * r0)) ** (5 / 3)
    assert abs(a / kolmo - 1) < 1e-5


def test_variance_and_positive_definiteness():
    r0, L0 = 0.1, 30.0
    var = CV.vk_cov(0.0, r0, L0)
    from scipy.special import gamma
    assert abs(var - CV.VK_C * gamma(5 / 6) * 2 ** (-1 / 6) * (L0 / r0) ** (5 / 3)) < 1e-12 * var
    assert abs(CV.VK_C * gamma(5 / 6) * 2 ** (-1 / 6) - 0.0863) < 2e-4   # the textbook coefficient
    C = CV.phase_cov(7, 0.5, r0, L0)
    assert np.allclose(C, C.T)
    w = np.linalg.eigvalsh(C)
    assert w.min() > -1e-10 * w.max()
    # covariance decreases with separation
    r = np.linspace(0, 3 * L0, 50)
    assert np.all(np.diff(CV.vk_cov(r, r0, L0)) < 0)


def test_layer_structure_functions_add_up():
    r0, L0 = 0.12, 20.0
    fr = np.array([0.5, 0.3, 0.2])
    r = np.array([0.05, 0.4, 3.0])
    tot = sum(CV.vk_structure(r, CV.layer_r0(r0, f), L0) for f in fr)
    np.testing.assert_allclose(tot, CV.vk_structure(r, r0, L0), rtol=1e-12)


def _impulse_basis(N):
    ifs = np.zeros((N * N, N, N))
    for p in range(N * N):
        ifs[p, p // N, p % N] = 1.0
    return ifs


def test_pixel_basis_gives_the_phase_covariance():
    N, dd, r0, L0 = 6, 0.3, 0.2, 15.0
    C = CV.atm_cov(_impulse_basis(N), dd, 1, r0, L0)
    np.testing.assert_allclose(C, CV.phase_cov(N, dd, r0, L0), rtol=1e-10, atol=1e-12 * C.max())


def test_change_of_basis_and_scaling():
    rng = np.random.default_rng(3)
    N, dd, bin_, r0, L0 = 12, 0.1, 2, 0.15, 20.0
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    cents = rng.uniform(1, N - 2, (9, 2))
    ifs = np.stack([np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2) / 4.0) for c in cents])
    C = CV.atm_cov(ifs, dd, bin_, r0, L0)
    Mx = np.eye(9) + 0.3 * rng.standard_normal((9, 9))
    ifs2 = np.einsum("anm,ab->bnm", ifs, Mx)   # F' = F M
    C2 = CV.atm_cov(ifs2, dd, bin_, r0, L0)
    Mi = np.linalg.inv(Mx)
    np.testing.assert_allclose(C2, Mi @ C @ Mi.T, rtol=1e-7, atol=1e-9 * np.abs(C).max())
    np.testing.assert_allclose(CV.atm_cov(2.5 * ifs, dd, bin_, r0, L0), C / 6.25, rtol=1e-10)
    assert np.allclose(C, C.T, rtol=1e-9, atol=1e-12 * np.abs(C).max())


def test_noise_values_and_elongation_geometry():
    lam, d, pix = 600e-9, 0.5, 0.5e-6
    fwhm_dl = lam / d
    cen = np.array([[0.0, 0.0]])
    # diffraction-limited spot, photon noise only: (pi^2 / 2) / N_ph / d^2
    C = CV.noise_cov(cen, d, 100.0, 0.0, pix, 8, fwhm_dl, lam)
    np.testing.assert_allclose(np.diag(C), [math.pi ** 2 / 2 / 100 / d ** 2] * 2, rtol=1e-12)
    assert C[0, 1] == 0.0
    # read-out noise adds (pi^2 / 3) ron^2 / N_ph^2 (N_s^2 / N_D)^2 / d^2
    C2 = CV.noise_cov(cen, d, 100.0, 3.0, pix, 8, fwhm_dl, lam)
    N_D = fwhm_dl / pix
    np.testing.assert_allclose(C2[0, 0] - C[0, 0], (math.pi ** 2 / 3) * 9 / 1e4 * (64 / N_D) ** 2 / d ** 2,
                               rtol=1e-12)
    # LGS: subaperture on the +x axis of the launch telescope: elongated along x
    cen2 = np.array([[10.0, 0.0], [10 / math.sqrt(2), 10 / math.sqrt(2)]])
    lgs = (0.0, 0.0, 90e3, 10e3, 0.0)
    Cl = CV.noise_cov(cen2, d, 200.0, 1.0, pix, 8, 1e-6, lam, lgs=lgs)
    nv = 2
    assert Cl[0, 0] > Cl[nv, nv] and Cl[0, nv] == pytest.approx(0.0, abs=1e-12 * Cl[0, 0])
    assert Cl[1, 1] == pytest.approx(Cl[nv + 1, nv + 1], rel=1e-12) and Cl[1, nv + 1] > 0
    tr = np.trace(Cl)
    rot = CV.noise_cov(cen2, d, 200.0, 1.0, pix, 8, 1e-6, lam, lgs=(2 * cen2[0, 0], 0.0, 90e3, 10e3, 0.0))
    # the launch telescope mirrored through the first subaperture: same elongation there
    assert rot[0, 0] == pytest.approx(Cl[0, 0], rel=1e-12)
    assert tr > 0


def test_mmse_forms_and_limits():
    rng = np.random.default_rng(5)
    nm, ns = 7, 12
    im = rng.standard_normal((nm, ns))
    A = rng.standard_normal((nm, nm))
    Ca = A @ A.T + nm * np.eye(nm)
    B = rng.standard_normal((ns, ns))
    Cn = 0.3 * (B @ B.T + ns * np.eye(ns))
    R = CV.mmse(im, Ca, Cn)
    D = im.T
    R2 = np.linalg.solve(D.T @ np.linalg.solve(Cn, D) + np.linalg.inv(Ca), D.T @ np.linalg.inv(Cn))
    np.testing.assert_allclose(R, R2, rtol=1e-9, atol=1e-12)
    sq = rng.standard_normal((nm, nm)) + 3 * np.eye(nm)
    np.testing.assert_allclose(CV.mmse(sq, Ca, 1e-12 * np.eye(nm)), np.linalg.inv(sq.T), rtol=1e-6, atol=1e-8)
    assert np.abs(CV.mmse(im, Ca, 1e12 * np.eye(ns))).max() < 1e-9
