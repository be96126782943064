"""FP64 oracle of the tomographic projection matrix (test infrastructure).

Only ``tests/`` and the CPU legs of ``bench.py`` may use it; the product path
never imports it.

Sec. 2.5 (tomographic projection matrices) defines the projection as a
pseudo-inverse (P_DM^T P_DM + lambda I)^{-1} P_DM^T P_Layer.  P_DM and
P_Layer map each influence function over the optimisation directions.  The
readings taken here are written out in full:

- Direction j is a source at infinity (height 0 in the sensor description)
  at field angle theta_j.  Its view of a
  component at altitude h is the composite affine of the chosen sensor grid
  (Sec. 2.1), with that field angle, no cone, no sensor rotation,
  magnification or shift, and no misregistration.  The footprint moves by
  h theta_j.
- Entry P_X[(j, q), a] is the mean, over the b x b fine pixels p of binned
  pupil pixel q, of P(p) * bilinear(IF_a; A_j (p_col, p_row) + b_j).
  - P is the sensor's pupil mask.
  - The bilinear resample is zero outside the source grid.
  - There is no edge repair: it is a phase projection, not a slope.
- Rows are ordered direction-major: row = j * (M / b)^2 + q, with q
  row-major on the binned grid.

The geometry comes from this package's own C oracle (``composite``).  The
resample and the solve are plain NumPy FP64.

Pins (tests/test_oracle_projection.py): a plane IF gives closed-form
entries; the projection of a component onto itself at a vanishing lambda is
the identity; and lambda * P_opt tends to P_DM^T P_Layer as lambda grows.
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np

from . import composite, pair_geom


def bilinear(img: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Bilinear samples of img [N, N] (row = y) at (x, y); taps outside the grid are 0."""
    N = img.shape[0]
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = x - x0, y - y0
    ix, iy = x0.astype(np.int64), y0.astype(np.int64)

    def tap(xx, yy):
        ok = (xx >= 0) & (yy >= 0) & (xx < N) & (yy < N)
        out = np.zeros(xx.shape)
        out[ok] = img[yy[ok], xx[ok]]
        return out

    return ((1.0 - fx) * (1.0 - fy) * tap(ix, iy) + fx * (1.0 - fy) * tap(ix + 1, iy) +
            (1.0 - fx) * fy * tap(ix, iy + 1) + fx * fy * tap(ix + 1, iy + 1))


def direction_affine(dm, wfs, theta: Sequence[float]):
    """(A [4], b [2]) of component dm seen from direction theta (rad) on wfs's grid."""
    view = dataclasses.replace(wfs, field_rad=(float(theta[0]), float(theta[1])), src_height_m=0.0,
                               rot_deg=0.0, mag=(1.0, 1.0), shift_m=(0.0, 0.0))
    return composite(pair_geom(dm, view), (0.0, 0.0, 0.0, 1.0))


def projection_matrix(dm, wfs, dirs: Sequence[Sequence[float]], b: int) -> np.ndarray:
    """P [n_dir * (M / b)^2, n_act] of one component (FP64)."""
    M = wfs.grid_m
    if M % b:
        raise ValueError("the sensor grid must be a multiple of the binning")
    Mb = M // b
    P = np.asarray(wfs.pupil_mask, np.float64) if wfs.pupil_mask is not None else np.ones((M, M))
    ii, jj = np.meshgrid(np.arange(M, dtype=np.float64), np.arange(M, dtype=np.float64), indexing="ij")
    ifs = np.asarray(dm.ifs, np.float64)
    out = np.zeros((len(dirs) * Mb * Mb, dm.n_act))
    for d, th in enumerate(dirs):
        A, bb = direction_affine(dm, wfs, th)
        x = A[0] * jj + A[1] * ii + bb[0]
        y = A[2] * jj + A[3] * ii + bb[1]
        for a in range(dm.n_act):
            fine = P * bilinear(ifs[a], x, y)
            out[d * Mb * Mb:(d + 1) * Mb * Mb, a] = fine.reshape(Mb, b, Mb, b).mean(axis=(1, 3)).ravel()
    return out


def p_opt(p_dm: np.ndarray, p_layer: np.ndarray, lam: float) -> np.ndarray:
    """(P_DM^T P_DM + lam I)^{-1} P_DM^T P_Layer (FP64)."""
    G = p_dm.T @ p_dm + lam * np.eye(p_dm.shape[1])
    return np.linalg.solve(G, p_dm.T @ p_layer)


def stack(workload, comps: Sequence[int], w: int, dirs, b: int) -> np.ndarray:
    """Projection matrices of several components side by side (columns in component order)."""
    return np.concatenate([projection_matrix(workload.dms[c], workload.wfss[w], dirs, b) for c in comps], axis=1)
