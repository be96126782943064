"""What the trained network gains over the fit alone (learned-estimator
geometry, GPU): a network trained on the GPU on 20k generated samples
estimates the misregistration of held-out noisy measurements far better
than the prior, and as the fit's starting point it reaches the fit's own
answer in fewer steps than the fit from the prior centre.  Small batches
run as captured graphs; their results equal the plain launches'."""
import numpy as np
import pytest

from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu

SCALE = np.array([8.0, 8.0, 2.0, 0.02])


@pytest.fixture(scope="module")
def trained():
    from paper_2606_07759_b300.synim import SynIM, cnn_init_params
    wl, cmd = W.learned()
    s = SynIM(wl.dms, wl.wfss)
    s.probe_attach(0, 0, cmd)
    s.cnn_init(cnn_init_params(32, seed=0, input_scale=0.2), (0.0, 0.0, 0.0, 1.0), tuple(SCALE))
    ptr = W.random_misregs(np.random.default_rng(5), 20000, 8.0, 2.0, 0.02)
    loss = s.cnn_train(ptr, epochs=10, batch=256, lr=2e-3, lr_final=1e-4, seed=6)
    s.check()
    yield wl, cmd, s, loss
    s.close()


def test_network_gain_over_the_fit_alone(trained):
    wl, cmd, s, loss = trained
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


def test_small_batch_graphs_equal_plain_launches(trained):
    """The captured small-batch chains (network; network + residual; network
    + 1 or 3 fit passes) give bit-identical results to the same chain run as
    plain launches on a context created with use_graph = 0, replays
    included, and pick up a changed fit setting."""
    from paper_2606_07759_b300.synim import SynIM
    wl, cmd, s, _ = trained
    w, c, r = s.cnn_get()
    s2 = SynIM(wl.dms, wl.wfss, use_graph=False)
    s2.probe_attach(0, 0, cmd)
    s2.cnn_init(w, tuple(c), tuple(r))
    pte = W.random_misregs(np.random.default_rng(41), 5, 8.0, 2.0, 0.02)
    y = s.probe_generate(pte, seed=4321, sample0=7 * 10 ** 8, noise_rel=0.01).float()
    try:
        for max_iter in (1, 3):
            s.gn_config(max_iter=max_iter)
            s2.gn_config(max_iter=max_iter)
            for n in (1, 4):
                for m in ("cnn", "cnn+gn"):
                    ref = s2.estimate(y[:n], m)
                    for _ in range(2):   # capture, then replay
                        got = s.estimate(y[:n], m)
                        for a, b in zip(got, ref):
                            np.testing.assert_array_equal(a, b)
                    if m == "cnn+gn":
                        assert np.all(got[2] <= max_iter)
        # a batch above the graph limit takes the plain launches on both
        ref = s2.estimate(y[:5].repeat(8, 1, 1, 1), "cnn")
        got = s.estimate(y[:5].repeat(8, 1, 1, 1), "cnn")
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)
    finally:
        s.gn_config()
        s2.close()
