"""Misregistration estimators on the GPU (synim_misreg_estimate) at the learned
estimator's geometry: the Gauss-Newton / Levenberg-Marquardt fit against the
FP64 oracle's fit (same algorithm, same data), and its exact recovery of the
truth from noise-free responses.
"""
import numpy as np
import pytest

import oracle
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu

SCALE = np.array([8.0, 8.0, 2.0, 0.02])
P0 = (1e-3, 1e-3, 1e-3, 1.0 + 1e-5)


@pytest.fixture(scope="module")
def learned():
    from paper_2606_07759_b300.synim import SynIM
    wl, cmd = W.learned()
    s = SynIM(wl.dms, wl.wfss)
    s.probe_attach(0, 0, cmd)
    screens = oracle.probe_screens(wl.dms[0], cmd)
    yield wl, cmd, s, screens
    s.close()


def _truths(seed, n):
    rng = np.random.default_rng(seed)
    t = W.random_misregs(rng, n, 8.0, 2.0, 0.02)
    t[0] = (-7.5, 7.0, -1.8, 0.982)
    return t


def test_gn_recovers_noise_free_truth(learned):
    wl, cmd, s, screens = learned
    truth = _truths(11, 6)
    y = s.probe_response(truth)
    s.gn_config(max_iter=40, tol=1e-6)
    p, res, it, conv = s.estimate(y, "gn")
    s.gn_config()
    assert conv.all(), it
    err = np.abs(p - truth) / SCALE
    assert err.max() < 1e-4, err
    assert res.max() < 1e-4


def test_gn_matches_oracle_fit(learned):
    wl, cmd, s, screens = learned
    dm, wfs = wl.dms[0], wl.wfss[0]
    truth = _truths(12, 2)
    y = s.probe_generate(truth, seed=77, noise_rel=0.01).float()
    p, res, it, conv = s.estimate(y, "gn", init=np.tile(P0, (2, 1)))
    yh = y.cpu().numpy().astype(np.float64)
    for q in range(2):
        pr, rr, itr, cr = oracle.gn_fit(screens, dm, wfs, yh[q], P0)
        assert cr and conv[q]
        assert np.all(np.abs(p[q] - pr) / SCALE < 2e-3), (p[q] - pr) / SCALE
        # both sit at the noise floor: the estimate is within ~1% of the range
        assert np.all(np.abs(p[q] - truth[q]) / SCALE < 0.02), (p[q] - truth[q]) / SCALE
        # the reported residual is the regenerated-response residual at the estimate
        s_at = oracle.probe_maps(screens, dm, wfs, p[q])
        ref = np.linalg.norm(yh[q] - s_at) / np.linalg.norm(yh[q])
        assert abs(res[q] - ref) <= 1e-4 * ref


def test_estimate_needs_a_network(learned):
    from paper_2606_07759_b300 import abi
    wl, cmd, s, screens = learned
    y = s.probe_response(_truths(13, 1))
    with pytest.raises(abi.SynimError) as e:
        s.estimate(y, "cnn")
    assert e.value.status == 7
