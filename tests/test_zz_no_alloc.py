"""The no-allocation entry point (synim_im_compute_noalloc) against the context API.

Some callers may not allocate device memory while they run (a real-time
controller with a fixed memory reservation, or a framework whose pooled
allocator owns the GPU).  synim_im_compute_noalloc serves them from one fixed
device array; this test calls it through the C ABI twice in a row, with
different misregistrations so that the second call starts from the first
call's leftover scratch, and checks each result against synim_im_compute at
the parity tolerance of tests/test_im_parity.py.  It also checks that an
input too large for the fixed array is refused with a clear error.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_07759_b300 import abi
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL, FLOOR = 1e-5, 1e-2  # same criterion as the parity tests


def _descs(dm, wfs, ifs_dev, keep):
    mask = None if dm.mask is None else np.ascontiguousarray(dm.mask, np.uint8)
    pm = None if wfs.pupil_mask is None else np.ascontiguousarray(wfs.pupil_mask, np.uint8)
    keep += [mask, pm]
    d = abi.synim_dm_desc(dm.n_act, dm.grid_n, dm.pixel_pitch_m, dm.altitude_m, ifs_dev.data_ptr(), 1,
                          None if mask is None else mask.ctypes.data, dm.support_eps)
    w = abi.synim_wfs_desc()
    w.n_sub, w.grid_m, w.pupil_diam_m, w.src_height_m = wfs.n_sub, wfs.grid_m, wfs.pupil_diam_m, wfs.src_height_m
    w.field_rad[0], w.field_rad[1] = wfs.field_rad
    w.rot_deg, w.mag[0], w.mag[1] = wfs.rot_deg, wfs.mag[0], wfs.mag[1]
    w.shift_m[0], w.shift_m[1] = wfs.shift_m
    w.pupil_mask, w.subap_valid = (None if pm is None else pm.ctypes.data), None
    w.obstruction, w.slope_scale = wfs.obstruction, wfs.slope_scale
    return d, w


def _noalloc(L, d, w, mis, out=None):
    rows = ctypes.c_int64()
    m = abi.synim_misreg(*mis.as_tuple())
    st = L.synim_im_compute_noalloc(ctypes.byref(d), ctypes.byref(w), ctypes.byref(m),
                                    None if out is None else out.data_ptr(), ctypes.byref(rows),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, rows.value


def _assert_close(got, ref, what):
    floor = FLOOR * float(np.abs(ref).max())
    peak = np.maximum(np.abs(ref).max(axis=1), floor)
    err = np.abs(got.astype(np.float64) - ref).max(axis=1)
    assert np.all(err <= TOL * peak), f"{what}: worst rel {np.max(err / peak):.3e}"


@pytest.mark.parametrize("name", ["scao_small", "scao_default_pupil", "elt_reduced", "mcao_reduced_ngs"])
def test_noalloc_matches_context_path_on_two_calls(name):
    import dataclasses
    from paper_2606_07759_b300.synim import SynIM
    L = abi.load()
    if name == "scao_small":
        wl = W.scao_small()
        d_i, w_i = 0, 0
    elif name == "scao_default_pupil":
        # no pupil mask: both paths build the default annulus themselves
        wl = W.scao_small()
        wl.wfss[0] = dataclasses.replace(wl.wfss[0], pupil_mask=None, obstruction=0.2)
        d_i, w_i = 0, 0
    elif name == "elt_reduced":
        wl = W.elt_single(seed=7, n_side=21, grid_n=120, n_sub=17)
        d_i, w_i = 0, 0
    else:
        wl = W.mcao_batched(seed=8, scale=0.2)
        d_i, w_i = 2, 7  # high-altitude DM seen by a 2x2 NGS sensor
    dm, wfs = wl.dms[d_i], wl.wfss[w_i]
    keep = []
    ifs_dev = torch.from_numpy(dm.ifs).cuda()
    d, w = _descs(dm, wfs, ifs_dev, keep)
    st, n_rows = _noalloc(L, d, w, wl.pair(d_i, w_i))
    assert st == 0, L.synim_last_error(None)
    ctx = SynIM([dm], [wfs])
    assert n_rows == ctx.shapes[(0, 0)][0]
    rng = np.random.default_rng(0)
    for call in range(2):
        mis = wl.pair(d_i, w_i) if call == 0 else W.Misreg(*rng.uniform([-1, -1, -1, 0.99], [1, 1, 1, 1.01]))
        out = torch.full((dm.n_act, n_rows), float("nan"), device="cuda")
        st, _ = _noalloc(L, d, w, mis, out)
        assert st == 0, L.synim_last_error(None)
        ref = ctx.compute([mis])[0]
        ctx.check()
        _assert_close(out.cpu().numpy(), ref.cpu().numpy().astype(np.float64), f"{name} call {call}")
    ctx.close()


def test_noalloc_rejects_inputs_beyond_the_fixed_array():
    L = abi.load()
    wl = W.scao_small()
    dm, wfs = wl.dms[0], wl.wfss[0]
    # 160 dense 480 x 480 planes with no support truncation: ~150 MB of windows
    n_act, N = 160, 480
    big = W.DM(np.zeros((n_act, N, N), np.float32), None, dm.pixel_pitch_m, 0.0,
               np.zeros((n_act, 2)), dm.pitch_px, support_eps=0.0)
    ifs_dev = torch.ones((n_act, N, N), device="cuda")
    keep = []
    d, w = _descs(big, wfs, ifs_dev, keep)
    out = torch.empty((n_act, 152), device="cuda")
    st, _ = _noalloc(L, d, w, W.Misreg(), out)
    assert st == 2  # SYNIM_ERR_SHAPE
    msg = L.synim_last_error(None).decode()
    assert "scratch" in msg and "bytes" in msg, msg
    # a host cube is refused too: it cannot be staged without allocating
    d.ifs_on_device = 0
    st, _ = _noalloc(L, d, w, W.Misreg(), out)
    assert st == 1
