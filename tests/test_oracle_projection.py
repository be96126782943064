"""Pins of the FP64 projection oracle (oracle/projection.py) against
closed forms and limits that do not reuse its code path.

- A plane influence function: the bilinear resample of a plane is exact, and
  the mean of an affine function over a binning block is its value at the
  block centre.  So every entry is the plane at the mapped block centre; this
  pins the resample, the binning and the row order.
- A source at infinity: the direction's affine differs from the on-axis one
  by the footprint shift h * theta / (DM pixel pitch) and nothing else (no
  cone factor).
- lambda -> 0 with the same component on both sides: P_opt -> identity.
- lambda -> infinity: lambda * P_opt -> P_DM^T P_Layer.
"""
import dataclasses

import numpy as np
import pytest

from oracle import projection as PR
from paper_2606_07759_b300 import workloads as W


def _plane_setup(h=3000.0, b=2):
    D, N, M = 8.0, 40, 24
    dd = D / N
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    plane = (0.25 * xx - 0.75 * yy + 2.0).astype(np.float32)[None]   # exact in FP32
    dm = W.DM(plane, None, dd, h, np.array([[N / 2, N / 2]]), 1.0)
    wfs = W.WFS(3, M, D * 0.6, 0.0, (0.0, 0.0), np.ones((M, M), np.uint8))
    return dm, wfs, b


def test_plane_influence_function_closed_form():
    dm, wfs, b = _plane_setup()
    dirs = [(0.0, 0.0), (2e-5, -1e-5)]
    P = PR.projection_matrix(dm, wfs, dirs, b)
    Mb = wfs.grid_m // b
    for d, th in enumerate(dirs):
        A, bb = PR.direction_affine(dm, wfs, th)
        qi, qj = np.meshgrid(np.arange(Mb), np.arange(Mb), indexing="ij")
        jc, ic = qj * b + (b - 1) / 2.0, qi * b + (b - 1) / 2.0
        x = A[0] * jc + A[1] * ic + bb[0]
        y = A[2] * jc + A[3] * ic + bb[1]
        assert x.min() > 0 and y.min() > 0 and x.max() < dm.grid_n - 2 and y.max() < dm.grid_n - 2
        ref = 0.25 * x - 0.75 * y + 2.0
        np.testing.assert_allclose(P[d * Mb * Mb:(d + 1) * Mb * Mb, 0], ref.ravel(), rtol=0, atol=1e-12)


def test_direction_is_a_pure_footprint_shift():
    dm, wfs, _ = _plane_setup(h=5000.0)
    th = (3e-5, -2e-5)
    A0, b0 = PR.direction_affine(dm, wfs, (0.0, 0.0))
    A1, b1 = PR.direction_affine(dm, wfs, th)
    np.testing.assert_array_equal(A0, A1)
    shift = np.array(th) * dm.altitude_m / dm.pixel_pitch_m
    np.testing.assert_allclose(b1 - b0, shift, rtol=1e-12, atol=1e-12)


@pytest.fixture(scope="module")
def small():
    wl = W.mcao_dictionary(seed=9, scale=0.15)
    dirs = [(0.0, 0.0), (8e-5, 0.0), (0.0, -8e-5)]
    return wl, dirs


def test_same_component_at_vanishing_lambda_is_identity(small):
    wl, dirs = small
    P = PR.stack(wl, [0], 0, dirs, 2)
    G = P.T @ P
    X = PR.p_opt(P, P, 1e-12 * np.mean(np.diag(G)))
    np.testing.assert_allclose(X, np.eye(P.shape[1]), atol=1e-6)


def test_large_lambda_limit(small):
    wl, dirs = small
    Pd, Pl = PR.stack(wl, [0, 1], 0, dirs, 2), PR.stack(wl, [5, 9], 0, dirs, 2)
    lam = 1e9 * np.mean(np.diag(Pd.T @ Pd))
    X = PR.p_opt(Pd, Pl, lam)
    np.testing.assert_allclose(lam * X, Pd.T @ Pl, rtol=1e-6, atol=1e-9 * np.abs(Pd.T @ Pl).max())
