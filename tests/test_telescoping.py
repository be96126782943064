"""Parity of the telescoping-sum engine (Sec. 2.2) on the GPU with its FP64
oracle (oracle/telescoping.py), through the C ABI.

Tolerance, derived from the FP32 arithmetic of one slope
s_r = fac_r * sum_e sign_e * phi(edge_e) over its n_e run ends:
- each bilinear sample is off by at most EPS_S = 5e-6 of the actuator's IF
  peak Phi_a: a few roundings of the interpolation (~3e-7) plus the error
  of the FP32 edge coordinate (|x| < 2^7 window pixels: ~8e-6 px, and the
  dropped low part of A times the offset from the box origin: as much
  again) times the IF's steepest slope (< 0.3 Phi_a per pixel for the
  zonal IFs and the cosine modes used here), plus support_eps times the
  DM's IF peak (the packed support window leaves out the IF values below
  that threshold, which the oracle's dense cube keeps);
- the FP32 running sum adds at most n_e 2^-24 sum_e |phi_e| (the standard
  recursive-summation bound);
so |gpu - oracle| <= fac_r (n_e (EPS_S Phi_a + eps Phi_DM) + n_e 2^-24
sum_e |phi_e|) + 2^-24 |s_r|.  A dropped or extra run end, a wrong sign or a half-pixel
slip moves a slope by fac_r |phi| or fac_r |grad phi| / 2, orders of
magnitude above the bound.  The worst ratio to the numerical engine's
column criterion is reported as well.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import telescoping as TS
from oracle.projection import bilinear
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu

EPS_S = 5e-6


def slope_bound(wl, d, w, cols, mis):
    """The per-slope FP32 error bound of the docstring, [len(cols), 2 nv]."""
    dm, wfs = wl.dms[d], wl.wfss[w]
    A, b = oracle.composite(oracle.pair_geom(dm, wfs), mis.as_tuple())
    ev = TS.edges(wfs.pupil_mask, wfs.n_sub, wfs.subap_valid)
    nv = len(ev)
    dw = wfs.pupil_diam_m / wfs.grid_m
    # every run end of every slope at once: its slope index (axis nv + row)
    ii, jj, slot = [], [], []
    fac = np.zeros(2 * nv)
    for r, (ex, ey, nlit) in enumerate(ev):
        fac[r] = fac[nv + r] = abs(wfs.slope_scale) / (dw * nlit)
        for axis, e in ((0, ex), (1, ey)):
            ii.append(e[:, 0])
            jj.append(e[:, 1])
            slot.append(np.full(e.shape[0], axis * nv + r))
    ii, jj, slot = np.concatenate(ii), np.concatenate(jj), np.concatenate(slot)
    n_e = np.bincount(slot, minlength=2 * nv).astype(np.float64)
    x, y = A[0] * jj + A[1] * ii + b[0], A[2] * jj + A[3] * ii + b[1]
    ifs = np.asarray(dm.ifs, np.float64)
    trunc = getattr(dm, "support_eps", 1e-9) * np.abs(ifs).max()
    out = np.zeros((len(cols), 2 * nv))
    for c, a in enumerate(cols):
        peak = np.abs(ifs[a]).max()
        s_abs = np.bincount(slot, weights=np.abs(bilinear(ifs[a], x, y)), minlength=2 * nv)
        out[c] = fac * (n_e * (EPS_S * peak + trunc) + n_e * 2.0 ** -24 * s_abs)
    return out


def assert_slopes(gpu, ref, bound, what):
    assert gpu.shape == ref.shape, (what, gpu.shape, ref.shape)
    err = np.abs(gpu.astype(np.float64) - ref)
    lim = bound + 2.0 ** -24 * np.abs(ref)
    bad = np.argwhere(err > lim)
    assert bad.size == 0, (f"{what}: {len(bad)} slopes fail, e.g. (col, row) {bad[:3].tolist()}: err "
                           f"{err[tuple(bad[0])]:.3e} > {lim[tuple(bad[0])]:.3e}")
    # the numerical engine's column criterion, for the record
    floor = 1e-2 * max(np.abs(ref).max(), 1e-30)
    return float(np.max(err.max(axis=1) / np.maximum(np.abs(ref).max(axis=1), floor)))


def tele_ims(wl, misregs=None, **kw):
    from paper_2606_07759_b300.synim import SynIM
    s = SynIM(wl.dms, wl.wfss, slope_engine="telescoping", **kw)
    out = s.compute(misregs if misregs is not None else wl.misregs)
    s.check()
    res = [t.cpu().numpy() for t in out]
    s.close()
    return res


def check_tele(wl, cols_per_dm=None, misregs=None, seed=0, sensors=None, **kw):
    ims = tele_ims(wl, misregs, **kw)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for d, dm in enumerate(wl.dms):
        if cols_per_dm is None or cols_per_dm >= dm.n_act:
            cols = np.arange(dm.n_act)
        else:
            cols = np.unique(np.concatenate([[0, dm.n_act - 1, dm.n_act // 2],
                                             rng.choice(dm.n_act, cols_per_dm, replace=False)]))
        for w in (range(len(wl.wfss)) if sensors is None else sensors):
            p = d * len(wl.wfss) + w
            mis = misregs[p] if misregs is not None else wl.misregs[p]
            ref = TS.im(wl, d, w, cols=cols, misreg=mis)
            worst = max(worst, assert_slopes(ims[p][cols], ref, slope_bound(wl, d, w, cols, mis),
                                             f"telescoping {wl.name} dm{d} wfs{w}"))
    print(f"{wl.name}: worst column error / column peak {worst:.2e}")
    return worst


def test_scao_small_all_columns():
    check_tele(W.scao_small())


@pytest.mark.parametrize("seed", [2, 11])
def test_elt_geometry_reduced_all_columns(seed):
    check_tele(W.elt_single(seed=seed, n_side=21, grid_n=120, n_sub=17))


def test_mcao_reduced_all_pairs_all_columns():
    # LGS 14x14 (cone) and NGS 2x2 (k > 32: whole-warp subapertures)
    check_tele(W.mcao_batched(seed=3, scale=0.2))


def test_mcao_full_size_sampled_columns():
    # the batched MCAO workload in the launch configuration the benchmark times
    # (autotuned); sampled columns of every DM on two LGS and one NGS sensor
    check_tele(W.mcao_batched(seed=3), cols_per_dm=4, sensors=(0, 3, 6), autotune=True)


def test_explicit_subap_valid_and_single_actuator():
    wl = W.scao_small()
    dm = wl.dms[0]
    one = W.DM(dm.ifs[40:41].copy(), dm.mask, dm.pixel_pitch_m, 0.0, dm.act_xy_px[40:41], dm.pitch_px)
    valid = np.zeros((10, 10), np.uint8)
    valid[2:8, 3:9] = 1
    valid[4, 5] = 0   # a hole: its neighbours keep their own run ends
    wfs = W.WFS(10, 80, 8.0, 0.0, (0.0, 0.0), wl.wfss[0].pupil_mask, obstruction=0.2, subap_valid=valid,
                slope_scale=2.5)
    check_tele(W.Workload("one", [one], [wfs], [W.Misreg(0.1, 0.2, 1.0, 1.0)]))


def test_dense_modal_cube():
    check_tele(W.modal_scao())


def test_rotation_large_shift_odd_rows_and_k2():
    # 90 deg rotation and a shift that moves some actuators off the sensor;
    # an odd nv (no 16-byte stores); a k = 2 sensor (every lit pixel is a run end).
    wl = W.scao_small()
    M = 20
    P = W.disc_mask(M, M / 2.0, 0.2 * M / 2.0)
    P[0, 8] = 0
    wl.wfss.append(W.WFS(10, M, 8.0, 0.0, (0.0, 0.0), P, obstruction=0.2))
    mis = [W.Misreg(7.5, -3.25, 90.0, 1.0), W.Misreg(0.4, 0.3, -12.0, 1.03)]
    check_tele(wl, misregs=mis)


def test_graph_replay_plain_launch_and_autotune_agree():
    from paper_2606_07759_b300.synim import SynIM
    wl = W.mcao_batched(seed=4, scale=0.15)
    s = SynIM(wl.dms, wl.wfss, slope_engine="telescoping")
    a = [t.clone() for t in s.compute(wl.misregs)]
    b = s.compute(wl.misregs)
    s.check()
    s2 = SynIM(wl.dms, wl.wfss, slope_engine="telescoping", use_graph=False)
    c = s2.compute(wl.misregs)
    s2.check()
    for x, y, z in zip(a, b, c):
        assert torch.equal(x, y) and torch.equal(x, z)   # fixed reduction orders: bit-identical
    # the autotuner may pick other lanes per subaperture (another summation
    # order): the same slopes to FP32 rounding
    s3 = SynIM(wl.dms, wl.wfss, slope_engine="telescoping", autotune=True)
    t = s3.compute(wl.misregs)
    s3.check()
    th, lanes, ms = s3.tuning(0)
    assert th in (128, 256) and 1 <= lanes <= 32 and ms > 0
    for x, z in zip(a, t):
        assert float((x - z).abs().max()) <= 1e-5 * float(x.abs().max())
    for q in (s, s2, s3):
        q.close()


def test_tangents_and_vjp_are_refused():
    from paper_2606_07759_b300 import abi
    from paper_2606_07759_b300.synim import SynIM
    wl = W.scao_small()
    s = SynIM(wl.dms, wl.wfss, slope_engine="telescoping")
    with pytest.raises(abi.SynimError):
        s.sensitivity(wl.misregs)
    s.close()


def test_plane_gives_its_exact_gradient_on_the_gpu():
    # a tilted plane IF: every valid subaperture's slope is the plane's gradient
    # (FP32: relative 1e-5 of it), whatever its lit shape
    N, M, n, D, dd = 96, 48, 6, 3.6, 0.05
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    plane = (0.25 * xx - 0.5 * yy + 3.0)[None].astype(np.float32)
    P = W.disc_mask(M, M / 2.0, 0.2 * M / 2.0)
    dm = W.DM(plane, None, dd, 0.0, np.array([[N / 2, N / 2]]), 1.0)
    dm.support_eps = 0.0
    wl = W.Workload("plane", [dm], [W.WFS(n, M, D, 0.0, (0.0, 0.0), P)], [W.Misreg(0.3, -0.2, 0.0, 1.0)])
    got = tele_ims(wl)[0][0].astype(np.float64)
    ref = TS.im(wl, 0, 0)[0]
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
