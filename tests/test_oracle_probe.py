"""Pins of the oracle's probe-response, noise and bfloat16 functions.

The probe response of a modal screen S_m = sum_a cmd[m, a] IF_a is pinned to
the already pinned IM oracle through linearity (every step of the method is
linear in the phase for a fixed core set, so response = cmd . IM), its
tangents likewise and by central differences; Philox4x32-10 by its published
known-answer vectors; the Box-Muller deviates by their distribution; the
bfloat16 rounding by PyTorch's CPU conversion (a library routine).
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2606_07759_b300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
MIS = [(0.3, -0.2, 0.5, 1.01), (-0.7, 0.45, -1.3, 0.985)]
P0 = (1e-3, 1e-3, 1e-3, 1.0 + 1e-5)   # fit start: prior centre, off the exact grid alignment


def _scao_with_probes():
    wl = W.scao_small()
    dm, wfs = wl.dms[0], wl.wfss[0]
    cmd = W.probe_modes(dm, wfs.pupil_diam_m, 16)
    return wl, dm, wfs, cmd


def test_philox_known_answers():
    kat = json.load(open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")))
    for c in kat["cases"]:
        ctr = [int(v, 16) for v in c["ctr"]]
        key = [int(v, 16) for v in c["key"]]
        out = [int(v, 16) for v in c["out"]]
        assert list(oracle.philox4x32_10(ctr, key)) == out


def test_gauss_distribution():
    z = oracle.gauss(12345, 7, np.arange(400_000))
    assert abs(z.mean()) < 0.008
    assert abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(np.abs(z) < 1.0) - 0.682689) < 0.004
    assert abs(np.mean(np.abs(z) > 3.0) - 0.0026998) < 0.0005
    # no correlation between the cosine and sine deviates of one pair, nor
    # between neighbouring pairs
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.01
    assert abs(np.corrcoef(z[0::4], z[2::4])[0, 1]) < 0.01
    # another sample index or seed gives other numbers
    assert not np.allclose(z[:16], oracle.gauss(12345, 8, np.arange(16)))
    assert not np.allclose(z[:16], oracle.gauss(12346, 7, np.arange(16)))


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 65504.0]])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(oracle.bf16_round(x), ref)
    assert oracle.bf16_round(np.float32([1.0 + 2.0 ** -8]))[0] == 1.0           # tie to even
    assert oracle.bf16_round(np.float32([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


@pytest.mark.parametrize("mis", MIS)
def test_probe_equals_command_times_im(mis):
    wl, dm, wfs, cmd = _scao_with_probes()
    screens = oracle.probe_screens(dm, cmd)
    g = oracle.pair_geom(dm, wfs)
    A, b = oracle.composite(g, mis)
    got = oracle.probe(screens, dm.mask, wfs, A, b)
    im = oracle.pair_im(wl, 0, 0, misreg=mis)          # [n_act, 2 nv]
    ref = cmd @ im
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_probe_tangents_equal_command_times_im_tangents():
    wl, dm, wfs, cmd = _scao_with_probes()
    screens = oracle.probe_screens(dm, cmd)
    g = oracle.pair_geom(dm, wfs)
    A, b = oracle.composite(g, MIS[1])
    dA, db = oracle.composite_jac(g, MIS[1])
    out, dout = oracle.probe(screens, dm.mask, wfs, A, b, dA, db)
    T = oracle.pair_tangent(wl, 0, 0, misreg=MIS[1])   # [4, n_act, 2 nv]
    for k in range(4):
        ref = cmd @ T[k]
        assert np.abs(dout[k] - ref).max() <= 1e-11 * np.abs(ref).max(), k
    assert np.abs(out - oracle.probe(screens, dm.mask, wfs, A, b)).max() == 0.0


def test_probe_tangents_match_central_differences():
    wl, dm, wfs, cmd = _scao_with_probes()
    screens = oracle.probe_screens(dm, cmd)
    p0 = np.array(MIS[0])
    _, T = oracle.probe_maps(screens, dm, wfs, p0, tangents=True)
    steps = [1e-4, 1e-4, 1e-4, 1e-6]
    for k in range(4):
        e = np.zeros(4)
        e[k] = steps[k]
        fd = (oracle.probe_maps(screens, dm, wfs, p0 + e) - oracle.probe_maps(screens, dm, wfs, p0 - e)) / (2 * steps[k])
        # most entries are smooth at this step; kinks (a sample crossing a
        # bilinear cell line) move only a small fraction
        err = np.abs(fd - T[k])
        scale = np.abs(T[k]).max()
        assert np.median(err) <= 1e-6 * scale
        assert np.mean(err <= 1e-3 * scale) > 0.9, k


def test_maps_layout():
    wl, dm, wfs, _ = _scao_with_probes()
    ros, _, nv = oracle.valid_subaps(wfs.pupil_mask, wfs.n_sub)
    rows = np.arange(3 * 2 * nv, dtype=np.float64).reshape(3, 2 * nv) + 1.0
    maps = oracle.to_maps(rows, wfs)
    assert maps.shape == (wfs.n_sub, wfs.n_sub, 6)
    for si in range(wfs.n_sub):
        for sj in range(wfs.n_sub):
            r = ros[si, sj]
            if r < 0:
                assert not maps[si, sj].any()
                continue
            for m in range(3):
                assert maps[si, sj, 2 * m] == rows[m, r]
                assert maps[si, sj, 2 * m + 1] == rows[m, nv + r]


def test_noisy_maps():
    wl, dm, wfs, cmd = _scao_with_probes()
    screens = oracle.probe_screens(dm, cmd)
    clean = oracle.probe_maps(screens, dm, wfs, MIS[0])
    ros, _, _ = oracle.valid_subaps(wfs.pupil_mask, wfs.n_sub)
    valid = ros >= 0
    np.testing.assert_array_equal(oracle.noisy_maps(clean, valid, 3, 11, 0.0), oracle.bf16_round(clean))
    noisy = oracle.noisy_maps(clean, valid, 3, 11, 0.05)
    assert not noisy[~valid].any()
    sigma = 0.05 * np.abs(clean).max()
    z = (noisy[valid] - clean[valid]) / sigma
    assert abs(z.std() - 1.0) < 0.05 and abs(z.mean()) < 0.05


def test_gn_fit_recovers_noise_free_truth():
    # zero residual at the truth: the fit must land on it (the minimum is exact).
    # The start is the prior centre nudged off the exact grid alignment: at
    # the identity with N = M every sample sits on a bilinear cell line, where
    # the floor-cell Jacobian is one-sided.
    wl, dm, wfs, cmd = _scao_with_probes()
    screens = oracle.probe_screens(dm, cmd)
    truth = np.array([0.6, -0.4, 0.8, 1.012])
    y = oracle.probe_maps(screens, dm, wfs, truth)
    p, res, it, conv = oracle.gn_fit(screens, dm, wfs, y, P0, tol=1e-7)
    assert conv and it <= 20
    assert np.all(np.abs(p - truth) / np.array([8, 8, 2, 0.02]) < 1e-10), p - truth
    assert res < 1e-9


def test_gn_fit_is_a_minimiser_under_noise():
    wl, dm, wfs, cmd = _scao_with_probes()
    screens = oracle.probe_screens(dm, cmd)
    truth = np.array([-0.3, 0.5, -0.6, 0.991])
    clean = oracle.probe_maps(screens, dm, wfs, truth)
    ros, _, _ = oracle.valid_subaps(wfs.pupil_mask, wfs.n_sub)
    y = oracle.noisy_maps(clean, ros >= 0, 9, 0, 0.01).astype(np.float64)
    p, res, it, conv = oracle.gn_fit(screens, dm, wfs, y, P0, max_iter=50)
    assert conv
    r_truth = np.linalg.norm(y - clean) / np.linalg.norm(y)
    assert res <= r_truth * (1 + 1e-12)
    # and the fit sits near the truth (noise of 1% of the peak; a 10x10
    # sensor constrains rotation and magnification only loosely)
    assert np.all(np.abs(p - truth) / np.array([8, 8, 2, 0.02]) < 0.1)
