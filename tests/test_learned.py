"""What the trained network gains over the fit alone (learned-estimator
geometry, GPU): a network trained on the GPU on 20k generated samples
estimates the misregistration of held-out noisy measurements far better
than the prior, and as the fit's starting point it reaches the fit's own
answer in fewer steps than the fit from the prior centre."""
import numpy as np
import pytest

from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu

SCALE = np.array([8.0, 8.0, 2.0, 0.02])


def test_network_gain_over_the_fit_alone():
    from paper_2606_07759_b300.synim import SynIM, cnn_init_params
    wl, cmd = W.learned()
    s = SynIM(wl.dms, wl.wfss)
    s.probe_attach(0, 0, cmd)
    s.cnn_init(cnn_init_params(32, seed=0, input_scale=0.2), (0.0, 0.0, 0.0, 1.0), tuple(SCALE))
    ptr = W.random_misregs(np.random.default_rng(5), 20000, 8.0, 2.0, 0.02)
    loss = s.cnn_train(ptr, epochs=10, batch=256, lr=2e-3, lr_final=1e-4, seed=6)
    s.check()
    assert loss[-1] < 0.01 * loss[0] or loss[-1] < 2e-3, loss
    pte = W.random_misregs(np.random.default_rng(99), 256, 8.0, 2.0, 0.02)
    y = s.probe_generate(pte, seed=1234, sample0=10 ** 9, noise_rel=0.01).float()
    p_cnn, r_cnn, _, _ = s.estimate(y, "cnn")
    p_gn, r_gn, it_gn, cv_gn = s.estimate(y, "gn")
    p_h, r_h, it_h, cv_h = s.estimate(y, "cnn+gn")
    prior_rms = 1.0 / np.sqrt(3.0)   # uniform over the range
    rms_cnn = np.sqrt((((p_cnn - pte) / SCALE) ** 2).mean(0))
    assert np.all(rms_cnn < 0.1 * prior_rms), rms_cnn
    # the hybrid lands on the fit's answer ...
    d = np.abs(p_h - p_gn) / SCALE
    assert np.mean(d.max(axis=1) < 2e-3) > 0.95
    assert cv_h.mean() >= cv_gn.mean()
    # ... in fewer steps
    assert it_h.mean() < 0.75 * it_gn.mean(), (it_h.mean(), it_gn.mean())
    # the fit is the more accurate estimator; both beat the network alone
    rms_gn = np.sqrt((((p_gn - pte) / SCALE) ** 2).mean(0))
    assert np.all(rms_gn < rms_cnn)
    assert np.median(r_h) <= np.median(r_cnn)
    s.close()
