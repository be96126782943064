"""FP64 CPU oracle for synthetic interaction matrices (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2606_07759_b300``) never imports it, and the two share
no code: the C source here re-derives every step from the paper (Sec. 2.1
composite affine and single bilinear resample, Sec. 2.2 aligned numerical
derivative and subaperture mean, Sec. 2.3 edge repair).

``build()`` compiles ``synim_oracle.c`` with gcc (FP64, no FMA contraction,
OpenMP over independent columns).

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
