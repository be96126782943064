"""ctypes declarations of include/synim.h (same names; argument marshalling only).

Loading fails loudly when libsynim.so is missing and cannot be built: there
is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import shutil

from . import build as _build

c_int32, c_int64, c_double, c_float, c_void_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                 ctypes.c_float, ctypes.c_void_p)

SYNIM_OK = 0
STATUS_NAMES = {0: "SYNIM_OK", 1: "SYNIM_ERR_INVALID_ARG", 2: "SYNIM_ERR_SHAPE", 3: "SYNIM_ERR_OOM",
                4: "SYNIM_ERR_CUDA", 5: "SYNIM_ERR_TIMEOUT", 6: "SYNIM_ERR_NOT_CONVERGED",
                7: "SYNIM_ERR_NOT_TRAINED", 8: "SYNIM_ERR_BOUNDS"}


class synim_dm_desc(ctypes.Structure):
    _fields_ = [("n_act", c_int32), ("grid_n", c_int32), ("pixel_pitch_m", c_double),
                ("altitude_m", c_double), ("ifs", c_void_p), ("ifs_on_device", c_int32),
                ("mask", c_void_p), ("support_eps", c_float)]


class synim_wfs_desc(ctypes.Structure):
    _fields_ = [("n_sub", c_int32), ("grid_m", c_int32), ("pupil_diam_m", c_double),
                ("src_height_m", c_double), ("field_rad", c_double * 2), ("rot_deg", c_double),
                ("mag", c_double * 2), ("shift_m", c_double * 2), ("pupil_mask", c_void_p),
                ("subap_valid", c_void_p), ("obstruction", c_double), ("slope_scale", c_double)]


class synim_misreg(ctypes.Structure):
    _fields_ = [("shift_x_px", c_double), ("shift_y_px", c_double), ("rot_deg", c_double),
                ("mag", c_double)]


ENGINE_NUMERICAL = 0     # SYNIM_ENGINE_NUMERICAL
ENGINE_TELESCOPING = 1   # SYNIM_ENGINE_TELESCOPING


class synim_noise_desc(ctypes.Structure):
    _fields_ = [("n_photons", c_double), ("ron_e", c_double), ("pixel_scale_rad", c_double), ("n_pix", c_int32),
                ("lgs", c_int32), ("fwhm_rad", c_double), ("wavelength_m", c_double), ("llt_xy_m", c_double * 2),
                ("na_altitude_m", c_double), ("na_thickness_m", c_double), ("zenith_rad", c_double)]


class synim_opts(ctypes.Structure):
    _fields_ = [("threads_per_cta", c_int32), ("ctas_per_sm", c_int32), ("use_graph", c_int32),
                ("autotune", c_int32), ("profile", c_int32), ("device_mem_cap", ctypes.c_int64),
                ("slope_engine", c_int32)]


class synim_train_opts(ctypes.Structure):
    _fields_ = [("epochs", c_int32), ("batch", c_int32), ("lr", c_float), ("lr_final", c_float),
                ("beta1", c_float), ("beta2", c_float), ("eps", c_float), ("noise_rel", c_float),
                ("seed", ctypes.c_uint64), ("sample0", ctypes.c_uint64)]


# name -> (restype, argtypes); mirrors include/synim.h
SIGNATURES = {
    "synim_im_create": (c_int32, [ctypes.POINTER(synim_dm_desc), c_int32, ctypes.POINTER(synim_wfs_desc),
                                  c_int32, ctypes.POINTER(synim_opts), ctypes.POINTER(c_void_p)]),
    "synim_im_query": (c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(c_int64),
                                 ctypes.POINTER(c_int64)]),
    "synim_pair_affine": (c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(synim_misreg),
                                    ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "synim_im_compute": (c_int32, [c_void_p, ctypes.POINTER(synim_misreg), ctypes.POINTER(c_void_p),
                                   c_void_p]),
    "synim_im_sensitivity": (c_int32, [c_void_p, ctypes.POINTER(synim_misreg), ctypes.POINTER(c_void_p),
                                       ctypes.POINTER(c_void_p), c_void_p]),
    "synim_im_vjp": (c_int32, [c_void_p, ctypes.POINTER(synim_misreg), ctypes.POINTER(c_void_p),
                               ctypes.POINTER(c_double), c_void_p]),
    "synim_im_check": (c_int32, [c_void_p, c_void_p]),
    "synim_wait_selftest": (c_int32, [c_void_p, ctypes.c_int64, c_void_p]),
    "synim_projection_rows": (c_int32, [c_void_p, c_int32, c_int32, c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "synim_projection_matrix": (c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(c_double), c_int32, c_int32,
                                          ctypes.POINTER(c_int32), c_void_p, c_void_p]),
    "synim_projection_opt": (c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(c_double), c_int32, c_int32,
                                       ctypes.POINTER(c_int32), c_int32, ctypes.POINTER(c_int32), c_double, c_void_p,
                                       c_void_p]),
    "synim_dm_window": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_int32)]),
    "synim_linalg_gemm": (c_int32, [c_int32, c_int32, c_int32, c_float, c_void_p, c_int64, c_void_p, c_int64,
                                    c_int32, c_float, c_void_p, c_int64, c_void_p]),
    "synim_linalg_spd_solve": (c_int32, [c_void_p, c_int32, c_int64, c_void_p, c_int32, c_int64, c_void_p]),
    "synim_atm_covariance": (c_int32, [c_void_p, c_int32, c_int32, c_double, c_double, c_void_p, c_void_p]),
    "synim_noise_covariance": (c_int32, [c_void_p, c_int32, ctypes.POINTER(synim_noise_desc), c_void_p, c_void_p]),
    "synim_mmse_reconstructor": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "synim_im_kernel_ms": (c_int32, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int32)]),
    "synim_im_compute_noalloc": (c_int32, [ctypes.POINTER(synim_dm_desc), ctypes.POINTER(synim_wfs_desc),
                                           ctypes.POINTER(synim_misreg), c_void_p, ctypes.POINTER(c_int64),
                                           c_void_p]),
    "synim_probe_attach": (c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(c_double), c_int32]),
    "synim_probe_query": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32), c_void_p]),
    "synim_probe_response": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "synim_probe_generate": (c_int32, [c_void_p, c_void_p, c_int64, ctypes.c_uint64, ctypes.c_uint64, c_float,
                                       c_void_p, c_void_p]),
    "synim_misreg_estimate": (c_int32, [c_void_p, c_void_p, c_int64, c_int32, ctypes.POINTER(synim_misreg),
                                        ctypes.POINTER(c_double), c_void_p]),
    "synim_gn_config": (c_int32, [c_void_p, c_int32, c_double, ctypes.POINTER(c_double)]),
    "synim_misreg_estimate_stats": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    "synim_cnn_n_params": (c_int32, [c_int32, c_int32]),
    "synim_cnn_init": (c_int32, [c_void_p, ctypes.POINTER(c_float), ctypes.POINTER(c_double)]),
    "synim_cnn_get": (c_int32, [c_void_p, ctypes.POINTER(c_float), ctypes.POINTER(c_double)]),
    "synim_debug_bounds": (c_int32, []),
    "synim_cnn_save": (c_int32, [c_void_p, c_void_p, c_int64, ctypes.POINTER(c_int64)]),
    "synim_cnn_load": (c_int32, [c_void_p, c_void_p, c_int64]),
    "synim_cnn_forward": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "synim_cnn_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(c_double),
                                 ctypes.POINTER(c_float), c_void_p]),
    "synim_cnn_train": (c_int32, [c_void_p, c_void_p, c_int64, ctypes.POINTER(synim_train_opts),
                                  ctypes.POINTER(c_double), c_void_p]),
    "synim_im_tuning": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                  ctypes.POINTER(c_double)]),
    "synim_im_destroy": (None, [c_void_p]),
    "synim_status_string": (ctypes.c_char_p, [c_int32]),
    "synim_last_error": (ctypes.c_char_p, [c_void_p]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libsynim.so (building it first if it is missing or stale and nvcc
    exists); with SYNIM_DEBUG_BOUNDS=1 in the environment, the bounds-checked
    build libsynim_bounds.so instead."""
    global _lib
    if _lib is not None:
        return _lib
    bounds = os.environ.get("SYNIM_DEBUG_BOUNDS", "0") == "1"
    lib = _build.lib_path(bounds)
    if _build.stale(bounds):
        if shutil.which(_build.NVCC) or os.path.exists(_build.NVCC):
            _build.build(bounds=bounds)
        elif not os.path.exists(lib):
            raise RuntimeError(os.path.basename(lib) + " is not built and nvcc is unavailable: the CUDA path "
                               "cannot run (there is no CPU fallback)")
    L = ctypes.CDLL(lib)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class SynimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def last_error(ctx=None) -> str:
    """Message of the context's last failure (of the last failed create with ctx = None)."""
    msg = load().synim_last_error(ctx)
    return (msg or b"").decode()


def check(status: int, ctx=None):
    if status != SYNIM_OK:
        L = load()
        msg = L.synim_last_error(ctx)
        raise SynimError(status, (msg or b"").decode())
