"""FP64 CPU oracle for synthetic interaction matrices (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2606_07759_b300``) never imports it, and the two share
no code: the C source here re-derives every step from the paper (Sec. 2.1
composite affine and single bilinear resample, Sec. 2.2 aligned numerical
derivative and subaperture mean, Sec. 2.3 edge repair).

``build()`` compiles ``synim_oracle.c`` with gcc (FP64, no FMA contraction,
OpenMP over independent columns).

Probe responses (the learned estimator's input) are the method applied to
modal screens; their counter-based noise is Philox4x32-10 with a Box-Muller
transform, both written from their published definitions.

Parity status: the forward IM, the composite affine and its Jacobian, the
tangents, the edge repair and the valid-subaperture rule are pinned by the
``-m "not gpu"`` tests (closed forms, invariants, telescoping identity,
continuous-gradient limit, hand-worked cases, finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synim_oracle.c")
_LIB = os.path.join(_HERE, "libsynim_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/libsynim_oracle.so (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        fp = ctypes.POINTER(ctypes.c_float)
        ci, cd = ctypes.c_int, ctypes.c_double
        L.synor_composite.argtypes = [dp, dp, dp, dp]
        L.synor_composite_jac.argtypes = [dp, dp, dp, dp]
        L.synor_valid_subaps.argtypes = [ci, ci, u8p, u8p, i32p, i32p]
        L.synor_valid_subaps.restype = ci
        L.synor_core.argtypes = [ci, u8p, ci, dp, dp, u8p, dp]
        L.synor_phase.argtypes = [fp, ci, u8p, ci, dp, dp, dp, u8p]
        L.synor_im.argtypes = [fp, ci, ci, u8p, ci, ci, u8p, u8p, dp, dp, cd, cd, i32p, ci, dp, ci]
        L.synor_im.restype = ci
        L.synor_im_tangent.argtypes = [fp, ci, ci, u8p, ci, ci, u8p, u8p, dp, dp, dp, dp, cd, cd,
                                       i32p, ci, dp, ci]
        L.synor_im_tangent.restype = ci
        L.synor_probe.argtypes = [dp, ci, ci, u8p, ci, ci, u8p, u8p, dp, dp, dp, dp, cd, cd, dp, dp]
        L.synor_probe.restype = ci
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.synor_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.synor_gauss.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64),
                                  ctypes.c_long, dp]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray], ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _u8(a) -> Optional[np.ndarray]:
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


# ---------------------------------------------------------------------------
# Geometry (Sec. 2.1)
# ---------------------------------------------------------------------------
def pair_geom(dm, wfs) -> np.ndarray:
    """The 13 geometric numbers of one (DM, WFS) pair, in the C oracle's order."""
    return _f64([dm.grid_n, dm.pixel_pitch_m, dm.altitude_m, wfs.grid_m, wfs.pupil_diam_m,
                 wfs.src_height_m, wfs.field_rad[0], wfs.field_rad[1], wfs.rot_deg,
                 wfs.mag[0], wfs.mag[1], wfs.shift_m[0], wfs.shift_m[1]])


def composite(geom: Sequence[float], p: Sequence[float]):
    """Composite affine: DM pixel (x, y) = A @ (j, i) + b for sensor pixel (row i, col j)."""
    g, pp = _f64(geom), _f64(p)
    A, b = np.zeros(4), np.zeros(2)
    lib().synor_composite(_p(g, ctypes.c_double), _p(pp, ctypes.c_double),
                          _p(A, ctypes.c_double), _p(b, ctypes.c_double))
    return A, b


def composite_jac(geom: Sequence[float], p: Sequence[float]):
    """d(A, b)/dp_k for p = (shift_x_px, shift_y_px, rot_deg, mag): dA [4, 4], db [4, 2]."""
    g, pp = _f64(geom), _f64(p)
    dA, db = np.zeros(16), np.zeros(8)
    lib().synor_composite_jac(_p(g, ctypes.c_double), _p(pp, ctypes.c_double),
                              _p(dA, ctypes.c_double), _p(db, ctypes.c_double))
    return dA.reshape(4, 4), db.reshape(4, 2)


def valid_subaps(P: np.ndarray, n_sub: int, valid_in: Optional[np.ndarray] = None):
    """(row_of_sub [n_sub, n_sub] int32, lit [n_sub, n_sub] int32, nv)."""
    P = _u8(P)
    M = P.shape[0]
    ros = np.zeros(n_sub * n_sub, np.int32)
    lit = np.zeros(n_sub * n_sub, np.int32)
    vi = _u8(valid_in)
    nv = lib().synor_valid_subaps(M, n_sub, _p(P, ctypes.c_uint8), _p(vi, ctypes.c_uint8),
                                  _p(ros, ctypes.c_int32), _p(lit, ctypes.c_int32))
    if nv < 0:
        raise ValueError("grid_m must be a multiple of n_sub")
    return ros.reshape(n_sub, n_sub), lit.reshape(n_sub, n_sub), nv


def core(dm_mask: Optional[np.ndarray], N: int, M: int, A, b):
    """Strict core of the interpolated DM mask (Sec. 2.3 step 1) and its closest margin."""
    m = _u8(dm_mask)
    A, b = _f64(A), _f64(b)
    out = np.zeros((M, M), np.uint8)
    margin = np.zeros(1)
    lib().synor_core(N, _p(m, ctypes.c_uint8), M, _p(A, ctypes.c_double), _p(b, ctypes.c_double),
                     _p(out, ctypes.c_uint8), _p(margin, ctypes.c_double))
    return out, float(margin[0])


def phase(if_a: np.ndarray, dm_mask: Optional[np.ndarray], M: int, A, b):
    """Repaired phase of one influence function on the M x M grid and the pixel classes."""
    img = np.ascontiguousarray(if_a, dtype=np.float32)
    N = img.shape[0]
    m = _u8(dm_mask)
    A, b = _f64(A), _f64(b)
    phi = np.zeros((M, M))
    cls = np.zeros((M, M), np.uint8)
    lib().synor_phase(_p(img, ctypes.c_float), N, _p(m, ctypes.c_uint8), M,
                      _p(A, ctypes.c_double), _p(b, ctypes.c_double), _p(phi, ctypes.c_double),
                      _p(cls, ctypes.c_uint8))
    return phi, cls


def im(ifs: np.ndarray, dm_mask, M: int, n_sub: int, P: np.ndarray, valid_in, A, b, dw: float,
       slope_scale: float = 1.0, cols: Optional[Sequence[int]] = None, nthreads: int = 0):
    """IM columns [ncols, 2 nv] (x slopes of valid subaps, then y slopes)."""
    ifs = np.ascontiguousarray(ifs, dtype=np.float32)
    n_act, N = ifs.shape[0], ifs.shape[1]
    cols = np.arange(n_act, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, np.int32)
    P = _u8(P)
    _, _, nv = valid_subaps(P, n_sub, valid_in)
    out = np.zeros((len(cols), 2 * nv))
    nthreads = nthreads or (os.cpu_count() or 1)
    vi, m = _u8(valid_in), _u8(dm_mask)
    A, b = _f64(A), _f64(b)
    lib().synor_im(_p(ifs, ctypes.c_float), n_act, N, _p(m, ctypes.c_uint8), M, n_sub,
                   _p(P, ctypes.c_uint8), _p(vi, ctypes.c_uint8), _p(A, ctypes.c_double),
                   _p(b, ctypes.c_double), dw, slope_scale, _p(cols, ctypes.c_int32), len(cols),
                   _p(out, ctypes.c_double), nthreads)
    return out


def im_tangent(ifs: np.ndarray, dm_mask, M: int, n_sub: int, P: np.ndarray, valid_in, A, b, dA,
               db, dw: float, slope_scale: float = 1.0, cols=None, nthreads: int = 0):
    """Tangents dIM/dp_k [4, ncols, 2 nv] with the core set held fixed."""
    ifs = np.ascontiguousarray(ifs, dtype=np.float32)
    n_act, N = ifs.shape[0], ifs.shape[1]
    cols = np.arange(n_act, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, np.int32)
    P = _u8(P)
    _, _, nv = valid_subaps(P, n_sub, valid_in)
    out = np.zeros((4, len(cols), 2 * nv))
    nthreads = nthreads or (os.cpu_count() or 1)
    vi, m = _u8(valid_in), _u8(dm_mask)
    A, b, dA, db = _f64(A), _f64(b), _f64(dA).ravel(), _f64(db).ravel()
    lib().synor_im_tangent(_p(ifs, ctypes.c_float), n_act, N, _p(m, ctypes.c_uint8), M, n_sub,
                           _p(P, ctypes.c_uint8), _p(vi, ctypes.c_uint8), _p(A, ctypes.c_double),
                           _p(b, ctypes.c_double), _p(dA, ctypes.c_double), _p(db, ctypes.c_double),
                           dw, slope_scale, _p(cols, ctypes.c_int32), len(cols),
                           _p(out, ctypes.c_double), nthreads)
    return out


# ---------------------------------------------------------------------------
# Workload-level helpers (marshalling only)
# ---------------------------------------------------------------------------
def pair_im(workload, d: int, w: int, cols=None, misreg=None, nthreads: int = 0):
    dm, wfs = workload.dms[d], workload.wfss[w]
    p = (misreg if misreg is not None else workload.pair(d, w)).as_tuple() \
        if not isinstance(misreg, (tuple, list, np.ndarray)) else tuple(misreg)
    A, b = composite(pair_geom(dm, wfs), p)
    return im(dm.ifs, dm.mask, wfs.grid_m, wfs.n_sub, wfs.pupil_mask, wfs.subap_valid, A, b,
              wfs.pupil_diam_m / wfs.grid_m, wfs.slope_scale, cols, nthreads)


def pair_tangent(workload, d: int, w: int, cols=None, misreg=None, nthreads: int = 0):
    dm, wfs = workload.dms[d], workload.wfss[w]
    p = (misreg if misreg is not None else workload.pair(d, w)).as_tuple() \
        if not isinstance(misreg, (tuple, list, np.ndarray)) else tuple(misreg)
    g = pair_geom(dm, wfs)
    A, b = composite(g, p)
    dA, db = composite_jac(g, p)
    return im_tangent(dm.ifs, dm.mask, wfs.grid_m, wfs.n_sub, wfs.pupil_mask, wfs.subap_valid,
                      A, b, dA, db, wfs.pupil_diam_m / wfs.grid_m, wfs.slope_scale, cols, nthreads)


# ---------------------------------------------------------------------------
# Probe responses of the learned estimator
# ---------------------------------------------------------------------------
def probe_screens(dm, cmd: np.ndarray) -> np.ndarray:
    """Modal screens S_m = sum_a cmd[m, a] IF_a in double precision, [n_modes, N, N]."""
    flat = np.asarray(dm.ifs, np.float64).reshape(dm.n_act, -1)
    return (np.asarray(cmd, np.float64) @ flat).reshape(len(cmd), dm.grid_n, dm.grid_n)


def probe(screens: np.ndarray, dm_mask, wfs, A, b, dA=None, db=None):
    """Responses [n_modes, 2 nv] of the screens at (A, b) and, with dA/db, the
    tangents [4, n_modes, 2 nv] (core set fixed)."""
    screens = np.ascontiguousarray(screens, np.float64)
    n_modes, N = screens.shape[0], screens.shape[1]
    P = _u8(wfs.pupil_mask)
    _, _, nv = valid_subaps(P, wfs.n_sub, wfs.subap_valid)
    out = np.zeros((n_modes, 2 * nv))
    tan = dA is not None
    dout = np.zeros((4, n_modes, 2 * nv)) if tan else None
    dA_ = _f64(dA).ravel() if tan else None
    db_ = _f64(db).ravel() if tan else None
    m, vi = _u8(dm_mask), _u8(wfs.subap_valid)
    A, b = _f64(A), _f64(b)
    lib().synor_probe(_p(screens, ctypes.c_double), n_modes, N, _p(m, ctypes.c_uint8),
                      wfs.grid_m, wfs.n_sub, _p(P, ctypes.c_uint8), _p(vi, ctypes.c_uint8),
                      _p(A, ctypes.c_double), _p(b, ctypes.c_double), _p(dA_, ctypes.c_double),
                      _p(db_, ctypes.c_double), wfs.pupil_diam_m / wfs.grid_m, wfs.slope_scale,
                      _p(out, ctypes.c_double), _p(dout, ctypes.c_double))
    return (out, dout) if tan else out


def to_maps(rows: np.ndarray, wfs) -> np.ndarray:
    """Scatter response rows [n_modes, 2 nv] into slope maps [n_sub, n_sub, 2 n_modes]
    (channel 2 m + 0 = x slope of mode m, 2 m + 1 = y slope; invalid subapertures 0)."""
    rows = np.asarray(rows)
    ros, _, nv = valid_subaps(wfs.pupil_mask, wfs.n_sub, wfs.subap_valid)
    n_modes = rows.shape[0]
    maps = np.zeros((wfs.n_sub, wfs.n_sub, 2 * n_modes))
    si, sj = np.nonzero(ros >= 0)
    r = ros[si, sj]
    maps[si, sj, 0::2] = rows[:, r].T
    maps[si, sj, 1::2] = rows[:, nv + r].T
    return maps


def probe_maps(screens, dm, wfs, p, tangents: bool = False):
    """Slope maps of one sample at misregistration p = (sx, sy, rot_deg, mag)."""
    g = pair_geom(dm, wfs)
    A, b = composite(g, p)
    if not tangents:
        return to_maps(probe(screens, dm.mask, wfs, A, b), wfs)
    dA, db = composite_jac(g, p)
    out, dout = probe(screens, dm.mask, wfs, A, b, dA, db)
    return to_maps(out, wfs), np.stack([to_maps(dout[k], wfs) for k in range(4)])


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    lib().synor_philox4x32_10(c.ctypes.data_as(u32), k.ctypes.data_as(u32), out.ctypes.data_as(u32))
    return out


def gauss(seed: int, sample: int, elems) -> np.ndarray:
    """Standard normal deviates of the given noise elements of one sample."""
    e = np.ascontiguousarray(elems, np.int64)
    z = np.zeros(len(e))
    lib().synor_gauss(ctypes.c_uint64(seed), ctypes.c_uint64(sample),
                      e.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(e),
                      z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return z


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via float32; returned as float32."""
    f = np.ascontiguousarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def noisy_maps(clean: np.ndarray, valid: np.ndarray, seed: int, sample: int,
               noise_rel: float) -> np.ndarray:
    """Probe input of one sample: clean maps [n_sub, n_sub, C] plus Gaussian
    noise of standard deviation noise_rel * (peak |slope| of the sample) on the
    valid subapertures (invalid ones stay 0), rounded to bfloat16."""
    clean = np.asarray(clean, np.float64)
    sigma = noise_rel * np.abs(clean).max()
    z = gauss(seed, sample, np.arange(clean.size)).reshape(clean.shape)
    out = np.where(valid[:, :, None], clean + sigma * z, 0.0)
    return bf16_round(out)


def gn_fit(screens, dm, wfs, y, p0, max_iter: int = 30, tol: float = 1e-4,
           scale=(8.0, 8.0, 2.0, 0.02)):
    """Levenberg-Marquardt fit of a probe measurement y [n_sub, n_sub, C] (FP64).

    Residual r = y - s(p) over all map entries, Jacobian from the probe
    tangents; each step solves (J^T J + mu diag(J^T J)) dp = J^T r (Cholesky);
    mu starts at 0, becomes 1e-3 (or x10) when the cost rises and the step is
    rejected, /10 (0 below 1e-7) after an accepted step; stop when an accepted
    step, divided by `scale`, has norm below tol, or after max_iter steps.
    Returns (p, ||y - s(p)|| / ||y||, steps, converged).
    """
    y = np.asarray(y, np.float64)
    sc = np.asarray(scale, np.float64)

    def evaluate(p):
        s, T = probe_maps(screens, dm, wfs, p, tangents=True)
        r = (y - s).ravel()
        J = T.reshape(4, -1).T
        return r @ r, J.T @ J, J.T @ r

    p = np.asarray(p0, np.float64).copy()
    c, H, g = evaluate(p)
    mu, it, conv = 0.0, 0, False
    while it < max_iter:
        try:
            L = np.linalg.cholesky(H + mu * np.diag(np.diag(H)))
        except np.linalg.LinAlgError:
            mu = 1e-3 if mu == 0.0 else mu * 10.0
            it += 1
            continue
        dp = np.linalg.solve(L.T, np.linalg.solve(L, g))
        it += 1
        pt = p + dp
        ct, Ht, gt = evaluate(pt)
        if ct <= c:
            p, c, H, g = pt, ct, Ht, gt
            mu = 0.0 if mu * 0.1 < 1e-7 else mu * 0.1
            if np.linalg.norm(dp / sc) < tol:
                conv = True
                break
        else:
            mu = 1e-3 if mu == 0.0 else mu * 10.0
            if mu > 1e12:
                break
    return p, float(np.sqrt(c / (y.ravel() @ y.ravel()))), it, conv
