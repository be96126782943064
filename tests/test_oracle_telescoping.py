"""Pins of the telescoping-sum slope oracle (oracle/telescoping.py).

- A tilted plane: the difference of phi at the two ends of a run is the
  plane's slope along the run times its length, so every valid subaperture's
  slope is the exact gradient, whatever its lit shape (annular pupil,
  rotation).
- A wide Gaussian: the edge sums converge to the boundary integral of the
  continuous phase over each subaperture (evaluated with Gauss-Legendre),
  the same limit as the numerical-derivative engine, and agree with that
  engine's oracle on interior subapertures.
- A quadratic phase x^2 at unit pixel scale under a pure shift: the x slope
  is twice the lit-pixel centroid over dw (bilinear's error is the same
  constant at every run end and cancels).
"""
import numpy as np

import oracle
from oracle import telescoping as TS
from paper_2606_07759_b300 import workloads as W


def _setup(ifs, P, misreg, N=96, dd=0.05, M=48, n=6, D=3.6):
    dm = W.DM(ifs.astype(np.float32), None, dd, 0.0, np.array([[N / 2, N / 2]]), 1.0)
    wfs = W.WFS(n, M, D, 0.0, (0.0, 0.0), P)
    return W.Workload("pin", [dm], [wfs], [misreg])


def test_tilted_plane_gives_its_exact_gradient():
    N, M, n = 96, 48, 6
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    plane = (0.25 * xx - 0.5 * yy + 3.0)[None]
    P = W.disc_mask(M, M / 2.0, 0.2 * M / 2.0)
    for mis in (W.Misreg(0.3, -0.2, 0.0, 1.0), W.Misreg(-0.4, 0.1, 1.5, 1.01)):
        wl = _setup(plane, P, mis)
        out = TS.im(wl, 0, 0)[0]
        A, b = oracle.composite(oracle.pair_geom(wl.dms[0], wl.wfss[0]), mis.as_tuple())
        dw = wl.wfss[0].pupil_diam_m / M
        nv = out.size // 2
        np.testing.assert_allclose(out[:nv], (0.25 * A[0] - 0.5 * A[2]) / dw, rtol=1e-12)
        np.testing.assert_allclose(out[nv:], (0.25 * A[1] - 0.5 * A[3]) / dw, rtol=1e-12)


def test_low_frequency_matches_the_continuous_boundary_integral():
    N, dd, M, n, D = 96, 0.05, 48, 6, 3.6
    k, dw = M // n, D / M
    s = 4 * k * dw
    sx_px, sy_px, x0, y0 = 0.3, -0.45, 0.3, -0.2
    cN = (N - 1) / 2
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    X, Y = (xx - cN) * dd, (yy - cN) * dd
    f = np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2 * s * s))[None]
    P = np.ones((M, M), np.uint8)
    wl = _setup(f, P, W.Misreg(sx_px, sy_px, 0.0, 1.0))
    out = TS.im(wl, 0, 0)[0]
    ros, lit, nv = oracle.valid_subaps(P, n)
    gl, gw = np.polynomial.legendre.leggauss(24)

    def phi(u, v):
        return np.exp(-((u - sx_px * dd - x0) ** 2 + (v - sy_px * dd - y0) ** 2) / (2 * s * s))

    peak = np.abs(out).max()
    for si in range(1, n - 1):
        for sj in range(1, n - 1):
            u0, u1 = (sj * k - 0.5 - (M - 1) / 2) * dw, ((sj + 1) * k - 0.5 - (M - 1) / 2) * dw
            v0, v1 = (si * k - 0.5 - (M - 1) / 2) * dw, ((si + 1) * k - 0.5 - (M - 1) / 2) * dw
            vq = 0.5 * (v1 - v0) * gl + 0.5 * (v1 + v0)
            uq = 0.5 * (u1 - u0) * gl + 0.5 * (u1 + u0)
            area = (u1 - u0) * (v1 - v0)
            ex = 0.5 * (v1 - v0) * np.sum(gw * (phi(u1, vq) - phi(u0, vq))) / area
            ey = 0.5 * (u1 - u0) * np.sum(gw * (phi(uq, v1) - phi(uq, v0))) / area
            r = ros[si, sj]
            assert abs(out[r] - ex) < 2e-3 * peak
            assert abs(out[nv + r] - ey) < 2e-3 * peak


def test_quadratic_gives_the_lit_centroid_law():
    # phi = x^2 (DM pixel units), sensor pixel = DM pixel, pure shift: every
    # run end has the same fractional position, so bilinear's error
    # f (1 - f) is one constant that cancels between a run's two ends, and
    # the x slope is 2 * mean over the lit pixels of x / dw exactly (the y
    # slope vanishes)
    N, M, n, dd = 96, 48, 6, 0.05
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    quad = (xx ** 2)[None]
    P = W.disc_mask(M, M / 2.0, 0.3 * M / 2.0)
    mis = W.Misreg(0.37, -0.21, 0.0, 1.0)
    wl = _setup(quad, P, mis, N=N, dd=dd, M=M, n=n, D=M * dd)
    out = TS.im(wl, 0, 0)[0]
    A, b = oracle.composite(oracle.pair_geom(wl.dms[0], wl.wfss[0]), mis.as_tuple())
    assert abs(A[0] - 1.0) < 1e-12 and abs(A[1]) < 1e-12
    ros, lit, nv = oracle.valid_subaps(P, n)
    k, dw = M // n, dd
    for si in range(n):
        for sj in range(n):
            r = ros[si, sj]
            if r < 0:
                continue
            ii, jj = np.nonzero(P[si * k:(si + 1) * k, sj * k:(sj + 1) * k])
            xbar = np.mean(A[0] * (jj + sj * k) + b[0])
            np.testing.assert_allclose(out[r], 2.0 * xbar / dw, rtol=1e-11)
            assert abs(out[nv + r]) <= 1e-9 * abs(out[r]) + 1e-9


def test_low_frequency_matches_the_numerical_derivative_oracle():
    # both engines approximate the same boundary integral: for a wide IF
    # (sigma = 4 subapertures) they agree to O((k dw / sigma)^2) of the peak
    # on interior subapertures (on the outermost ring the central difference
    # reads phi = 0 beyond the grid edge, the run-end sums do not)
    N, dd, M, n, D = 96, 0.05, 48, 6, 3.6
    k, dw = M // n, D / M
    s = 4 * k * dw
    cN = (N - 1) / 2
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    X, Y = (xx - cN) * dd, (yy - cN) * dd
    f = np.exp(-((X - 0.3) ** 2 + (Y + 0.2) ** 2) / (2 * s * s))[None]
    P = np.ones((M, M), np.uint8)
    wl = _setup(f, P, W.Misreg(0.3, -0.45, 0.4, 1.002))
    tele = TS.im(wl, 0, 0)[0]
    num = oracle.pair_im(wl, 0, 0)[0]
    ros, lit, nv = oracle.valid_subaps(P, n)
    inner = np.array([ros[si, sj] for si in range(1, n - 1) for sj in range(1, n - 1)])
    rows = np.concatenate([inner, nv + inner])
    assert np.abs(tele[rows] - num[rows]).max() <= 2e-3 * np.abs(num).max()
