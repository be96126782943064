"""FP64 oracle of the telescoping-sum slope engine (test infrastructure).

Only ``tests/`` and the CPU legs of ``bench.py`` may use it; the product path
never imports it.

Sec. 2.2 names two slope engines: the numerical derivative (the default; the
rest of this package) and the telescoping sum, which takes phase differences
only at the subaperture edges.  The reading taken here is written out:

- The x slope of valid subaperture s is its gradient tilt over the lit area.
  The fundamental theorem of calculus gives it, per pixel row, as the phase
  at the end of each lit run minus the phase at its start, where the run
  edges are the half-pixel points j - 1/2 and j + 1/2:
      s_x = slope_scale * sum_edges sign * phi(edge) / (dw * n_lit(s))
- An edge is the left (sign -1) or right (+1) side of a lit pixel whose
  neighbour on that side is unlit or outside s.  The y slope is the same
  along pixel columns (edges at i -/+ 1/2).
- phi(edge) is the influence function resampled once at the composite-affine
  image of the edge point (Sec. 2.1): bilinear, zero outside the source grid,
  with no edge repair.  The phase is evaluated at the edge itself rather than
  at pixels, and the cube already carries the DM mask.
- Valid subapertures, the row order, slope_scale and dw = D / M are those of
  the numerical-derivative engine.

Pins (tests/test_oracle_telescoping.py):
- a tilted plane gives its exact gradient, whatever the lit shape;
- a quadratic (unit pixel scale, pure shift) gives the lit-pixel centroid
  law exactly;
- a low-frequency influence function converges to the continuous boundary
  integral, and agrees with the numerical-derivative oracle on interior
  subapertures to O((k dw / sigma)^2).
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import composite, pair_geom, valid_subaps
from .projection import bilinear


def edges(P: np.ndarray, n_sub: int, valid_in: Optional[np.ndarray] = None):
    """Per valid subaperture (row order): x edges (i, j_edge, sign), y edges and n_lit."""
    P = np.asarray(P, np.uint8)
    M = P.shape[0]
    k = M // n_sub
    ros, lit, nv = valid_subaps(P, n_sub, valid_in)
    out = [None] * nv
    for si in range(n_sub):
        for sj in range(n_sub):
            r = ros[si, sj]
            if r < 0:
                continue
            ex, ey = [], []
            for i in range(si * k, si * k + k):
                for j in range(sj * k, sj * k + k):
                    if not P[i, j]:
                        continue
                    if j == sj * k or not P[i, j - 1]:
                        ex.append((i, j - 0.5, -1.0))
                    if j == sj * k + k - 1 or not P[i, j + 1]:
                        ex.append((i, j + 0.5, 1.0))
                    if i == si * k or not P[i - 1, j]:
                        ey.append((i - 0.5, j, -1.0))
                    if i == si * k + k - 1 or not P[i + 1, j]:
                        ey.append((i + 0.5, j, 1.0))
            out[r] = (np.array(ex, np.float64).reshape(-1, 3), np.array(ey, np.float64).reshape(-1, 3),
                      int(lit[si, sj]))
    return out


def im(workload, d: int, w: int, cols: Optional[Sequence[int]] = None, misreg=None) -> np.ndarray:
    """Telescoping-sum IM columns [ncols, 2 nv] of pair (d, w) (x slopes, then y)."""
    dm, wfs = workload.dms[d], workload.wfss[w]
    mis = misreg if misreg is not None else workload.pair(d, w)
    A, b = composite(pair_geom(dm, wfs), mis.as_tuple())
    ev = edges(wfs.pupil_mask, wfs.n_sub, wfs.subap_valid)
    nv = len(ev)
    dw = wfs.pupil_diam_m / wfs.grid_m
    cols = range(dm.n_act) if cols is None else cols
    ifs = np.asarray(dm.ifs, np.float64)
    out = np.zeros((len(cols), 2 * nv))
    for c, a in enumerate(cols):
        for r, (ex, ey, nlit) in enumerate(ev):
            fac = wfs.slope_scale / (dw * nlit)
            for axis, e in ((0, ex), (1, ey)):
                if e.size == 0:
                    continue
                i, j, sgn = e[:, 0], e[:, 1], e[:, 2]
                x = A[0] * j + A[1] * i + b[0]
                y = A[2] * j + A[3] * i + b[1]
                out[c, axis * nv + r] = fac * np.sum(sgn * bilinear(ifs[a], x, y))
    return out
