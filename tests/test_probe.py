"""Probe responses on the GPU (synim_probe_response / synim_probe_generate)
against the FP64 oracle, at the full geometry of the learned estimator:
40x40 Shack-Hartmann (k = 8, M = 320), 41x41 DM (N = 320), 16 probe modes.

Criteria:
  - clean maps: per (sample, mode, axis) map, max |gpu - ref| <= 1e-5 x the
    map's peak |ref| (floored at 1e-2 of the sample's peak), the IM parity
    criterion applied to the slope vector of one probe mode;
  - tangents: <= 1e-4 x max |T_k| on subapertures that use no pixel sampled
    within 1e-5 px of a bilinear cell line (there the derivative of the
    interpolant jumps and either cell is a correct floor-cell derivative);
  - noisy bfloat16 inputs: at most one bfloat16 unit in the last place apart
    (the clean values differ by rounding, which can move a value across a
    bfloat16 rounding boundary), or the clean tolerance for values near zero,
    and identical bits for almost all entries.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def learned():
    from paper_2606_07759_b300.synim import SynIM
    wl, cmd = W.learned()
    s = SynIM(wl.dms, wl.wfss)
    s.probe_attach(0, 0, cmd)
    screens = oracle.probe_screens(wl.dms[0], cmd)
    yield wl, cmd, s, screens
    s.close()


def _params(seed, n):
    rng = np.random.default_rng(seed)
    p = W.random_misregs(rng, n, 8.0, 2.0, 0.02)
    p[0] = (8.0, -8.0, 2.0, 1.02)   # corner of the training range
    return p


def _assert_maps_close(got, ref, valid, what):
    got = np.asarray(got, np.float64)
    peak_s = np.abs(ref).max()
    C = ref.shape[-1]
    for c in range(C):
        r = ref[..., c][valid]
        g = got[..., c][valid]
        peak = max(np.abs(r).max(), 1e-2 * peak_s)
        err = np.abs(g - r).max()
        assert err <= 1e-5 * peak, f"{what} channel {c}: {err / peak:.3e}"
    assert not got[~valid].any()


def test_probe_maps_match_oracle(learned):
    wl, cmd, s, screens = learned
    dm, wfs = wl.dms[0], wl.wfss[0]
    P = _params(1, 6)
    maps = s.probe_response(P).cpu().numpy()
    s.check()
    assert maps.shape == (6, 40, 40, 32)
    for q in range(len(P)):
        ref = oracle.probe_maps(screens, dm, wfs, P[q])
        _assert_maps_close(maps[q], ref, s.probe_valid, f"sample {q}")


@pytest.mark.parametrize("name", ["scao_small", "elt_reduced"])
def test_probe_maps_with_mask_edges_match_oracle(name):
    # geometries whose DM mask edge (annulus with a central obstruction) lies
    # inside the sensor pupil: the ring repair of the probe kernel at work
    from paper_2606_07759_b300.synim import SynIM
    wl = W.scao_small() if name == "scao_small" else W.elt_single(seed=6, n_side=21, grid_n=120, n_sub=17)
    dm, wfs = wl.dms[0], wl.wfss[0]
    cmd = W.probe_modes(dm, wfs.pupil_diam_m, 12)
    s = SynIM(wl.dms, wl.wfss)
    s.probe_attach(0, 0, cmd)
    screens = oracle.probe_screens(dm, cmd)
    P = np.array([wl.misregs[0].as_tuple(), (0.8, -0.6, 1.5, 1.015), (-1.0, 1.0, -2.0, 0.98)])
    maps, dmaps = s.probe_response(P, tangents=True)
    s.check()
    maps, dmaps = maps.cpu().numpy(), dmaps.cpu().numpy()
    assert maps.shape[-1] == 24
    for q in range(len(P)):
        ref, T = oracle.probe_maps(screens, dm, wfs, P[q], tangents=True)
        _assert_maps_close(maps[q], ref, s.probe_valid, f"{name} sample {q}")
        for k in range(4):
            scale = np.abs(T[k]).max()
            err = np.abs(dmaps[k, q].astype(np.float64) - T[k])
            # kinks flagged as in the tangent test below, on this geometry
            keep = s.probe_valid & ~_kink_subaps(wl, P[q])
            assert err[keep].max() <= 1e-4 * scale, f"{name} sample {q} p{k}"
    s.close()


def test_probe_maps_equal_command_times_gpu_im(learned):
    # linearity across the two GPU paths: probe maps = cmd . IM
    wl, cmd, s, screens = learned
    P = _params(2, 2)
    maps = s.probe_response(P).cpu().numpy()
    ros, _, nv = oracle.valid_subaps(wl.wfss[0].pupil_mask, 40)
    for q in range(2):
        im = s.compute([W.Misreg(*P[q])])[0].cpu().numpy().astype(np.float64)   # [n_act, 2 nv]
        rows = cmd @ im
        ref = oracle.to_maps(rows, wl.wfss[0])
        _assert_maps_close(maps[q], ref, s.probe_valid, f"cmd.IM sample {q}")


def _kink_subaps(wl, p, near=1e-5):
    """Subapertures whose slopes use a pixel sampled within `near` of a cell line."""
    from scipy.ndimage import binary_dilation
    from test_sensitivity import stencil_pixels
    dm, wfs = wl.dms[0], wl.wfss[0]
    M, n = wfs.grid_m, wfs.n_sub
    A, b = oracle.composite(oracle.pair_geom(dm, wfs), p)
    ii, jj = np.mgrid[0:M, 0:M].astype(np.float64)
    bad = np.zeros((M, M), bool)
    for c in (A[0] * jj + A[1] * ii + b[0], A[2] * jj + A[3] * ii + b[1]):
        f = c - np.floor(c)
        bad |= (f < near) | (f > 1 - near)
    bad = binary_dilation(binary_dilation(bad, iterations=2) & stencil_pixels(wfs), iterations=1)
    return bad.reshape(n, M // n, n, M // n).any(axis=(1, 3))


def test_probe_tangents_match_oracle(learned):
    wl, cmd, s, screens = learned
    dm, wfs = wl.dms[0], wl.wfss[0]
    P = _params(3, 3)
    maps, dmaps = s.probe_response(P, tangents=True)
    maps0 = s.probe_response(P)
    s.check()
    maps, dmaps, maps0 = maps.cpu().numpy(), dmaps.cpu().numpy(), maps0.cpu().numpy()
    np.testing.assert_array_equal(maps, maps0)   # the tangent pass writes the same maps
    for q in range(len(P)):
        _, T = oracle.probe_maps(screens, dm, wfs, P[q], tangents=True)
        keep = s.probe_valid & ~_kink_subaps(wl, P[q])
        assert keep.sum() > 0.9 * s.probe_valid.sum()
        for k in range(4):
            scale = np.abs(T[k]).max()
            err = np.abs(dmaps[k, q][keep].astype(np.float64) - T[k][keep]).max()
            assert err <= 1e-4 * scale, f"sample {q} p{k}: {err / scale:.3e}"


def test_probe_generate_matches_oracle(learned):
    wl, cmd, s, screens = learned
    dm, wfs = wl.dms[0], wl.wfss[0]
    P = _params(4, 4)
    seed, sample0 = 0x1234_5678_9ABC, 1_000_003
    out = s.probe_generate(P, seed=seed, sample0=sample0, noise_rel=0.01)
    s.check()
    got = out.float().cpu().numpy()
    same = 0
    for q in range(len(P)):
        clean = oracle.probe_maps(screens, dm, wfs, P[q])
        ref = oracle.noisy_maps(clean, s.probe_valid, seed, sample0 + q, 0.01)
        ulp = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(ref), 1e-30))) - 7)
        # one bfloat16 step, or the clean-map tolerance where the noisy value
        # is so close to zero that its bfloat16 step is finer than that
        tol = np.maximum(ulp, 1e-5 * np.abs(clean).max())
        assert np.all(np.abs(got[q] - ref) <= tol), f"sample {q}"
        same += np.sum(got[q] == ref)
    assert same >= 0.99 * got.size


def test_probe_generate_without_noise_is_rounded_clean(learned):
    wl, cmd, s, screens = learned
    P = _params(5, 3)
    clean = s.probe_response(P)
    out = s.probe_generate(P, seed=1, noise_rel=0.0)
    s.check()
    torch.testing.assert_close(out, clean.to(torch.bfloat16), rtol=0, atol=0)


def test_probe_edge_cases(learned):
    from paper_2606_07759_b300 import abi
    wl, cmd, s, screens = learned
    empty = s.probe_response(np.zeros((0, 4)))
    assert empty.shape[0] == 0
    # a sample far off the DM: no core pixel reaches the sensor, slopes are 0
    far = s.probe_response(np.array([[1000.0, 0.0, 0.0, 1.0]])).cpu().numpy()
    assert not far.any()
    with pytest.raises(abi.SynimError):
        s.probe_generate(np.zeros((1, 4)) + [0, 0, 0, 1], seed=0, noise_rel=-1.0)
