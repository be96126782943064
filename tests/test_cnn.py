"""The estimator network on the GPU (BF16 tensor-core convolutions, FP32
accumulation) against the FP64 oracle (oracle/cnn.py) on the same BF16
inputs and the same BF16-rounded convolution weights.

Criteria (relative L2 error per output and per parameter-gradient tensor):
  - forward outputs: <= 1e-2 against the exact FP64 network;
  - gradients: <= 1e-2 against the FP64 backward with the GPU's stored
    activations and activation gradients rounded to BF16 (the precision
    model of the kernels; oracle.cnn.loss_grad_rounded; FP32 sums still move
    a few values across a BF16 rounding boundary), and <= 5e-2 against
    the exact FP64 gradient.  The first layer's weight gradient sits three
    BF16 roundings below the loss and sums tens of thousands of products of
    mixed sign, so its rounding error alone reaches ~3% on random weights.
Batch sizes cover one sample, a ragged GEMM tile (37 samples: 59200 rows,
not a multiple of 128) and the full pass (256).
"""
import numpy as np
import pytest
import torch

import oracle
import oracle.cnn as oc
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu

NORM_C, NORM_R = (0.0, 0.0, 0.0, 1.0), (8.0, 8.0, 2.0, 0.02)
TENSORS = ["W1", "b1", "W2", "b2", "W3", "b3", "Wfc", "bfc"]



@pytest.fixture(scope="module")
def net():
    from paper_2606_07759_b300.synim import SynIM, cnn_init_params
    wl, cmd = W.learned()
    s = SynIM(wl.dms, wl.wfss)
    s.probe_attach(0, 0, cmd)
    P = cnn_init_params(32, seed=0, input_scale=0.2)
    rng = np.random.default_rng(1)
    P = P + rng.normal(0, 0.01, P.shape).astype(np.float32)   # non-zero biases
    s.cnn_init(P, NORM_C, NORM_R)
    yield s, P
    s.close()


def _oracle_params(P):
    """The FP32 masters with the convolution weights rounded to BF16, as the GPU uses them."""
    q = P.astype(np.float64).copy()
    n1, n2 = 64 * 9 * 32, 64 * 9 * 64
    for o, n in ((0, n1), (n1 + 64, n2), (n1 + 64 + n2 + 64, n2)):
        q[o:o + n] = oracle.bf16_round(P[o:o + n])
    return q


def _batch(s, n, seed):
    rng = np.random.default_rng(seed)
    p = W.random_misregs(rng, n, 8.0, 2.0, 0.02)
    x = s.probe_generate(p, seed=seed, noise_rel=0.01)
    t = ((p - np.array(NORM_C)) / np.array(NORM_R)).astype(np.float32)
    return x, t


def _split(v):
    return oc.unpack(v, 32)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("n", [1, 37, 256])
def test_forward_matches_oracle(net, n):
    s, P = net
    x, _ = _batch(s, n, 10 + n)
    got = s.cnn_forward(x).cpu().numpy()
    ref = oc.forward(_oracle_params(P), x.float().cpu().numpy(), 32)
    assert _rel(got, ref) <= 1e-2, _rel(got, ref)


@pytest.mark.parametrize("n", [8, 37])
def test_gradients_match_oracle(net, n):
    s, P = net
    x, t = _batch(s, n, 20 + n)
    loss, g = s.cnn_grad(x, t)
    xh = x.float().cpu().numpy()
    lref, gref = oc.loss_grad(_oracle_params(P), xh, t, 32)
    lrnd, grnd = oc.loss_grad_rounded(_oracle_params(P), xh, t, 32)
    assert abs(loss - lref) <= 1e-2 * lref
    for name, a, b, c in zip(TENSORS, _split(g), _split(gref), _split(grnd)):
        r_exact = _rel(a.numpy(), b.numpy())
        r_model = _rel(a.numpy(), c.numpy())
        assert r_model <= 1e-2, f"{name}: {r_model:.3e} against the BF16 precision model"
        assert r_exact <= 5e-2, f"{name}: {r_exact:.3e} against the exact gradient"


def test_training_reduces_the_loss():
    from paper_2606_07759_b300.synim import SynIM, cnn_init_params
    wl, cmd = W.learned()
    s = SynIM(wl.dms, wl.wfss)
    s.probe_attach(0, 0, cmd)
    s.cnn_init(cnn_init_params(32, seed=4, input_scale=0.2), NORM_C, NORM_R)
    rng = np.random.default_rng(5)
    p = W.random_misregs(rng, 4096, 8.0, 2.0, 0.02)
    losses = s.cnn_train(p, epochs=4, batch=128, lr=2e-3, seed=6)
    s.check()
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], losses
    w, c, r = s.cnn_get()
    assert np.isfinite(w).all()
    s.close()


def test_checkpoint_resume_equals_uninterrupted(tmp_path):
    """A run saved after its first training call and resumed in a fresh
    context (parameters, Adam moments and step count restored) ends with
    the same parameters, bit for bit, as the uninterrupted run; foreign,
    truncated and wrong-shape checkpoints are refused."""
    import struct
    from paper_2606_07759_b300 import abi
    from paper_2606_07759_b300.synim import SynIM, cnn_init_params
    wl, cmd = W.learned()
    P0 = cnn_init_params(32, seed=8, input_scale=0.2)
    rng = np.random.default_rng(9)
    p1 = W.random_misregs(rng, 1024, 8.0, 2.0, 0.02)
    p2 = W.random_misregs(rng, 1024, 8.0, 2.0, 0.02)

    def fresh():
        s = SynIM(wl.dms, wl.wfss)
        s.probe_attach(0, 0, cmd)
        return s

    a = fresh()
    a.cnn_init(P0, NORM_C, NORM_R)
    a.cnn_train(p1, epochs=1, batch=128, lr=2e-3, seed=6)
    ck = a.cnn_save(tmp_path / "net.ckpt")
    a.cnn_train(p2, epochs=1, batch=128, lr=2e-3, seed=7)
    wa, ca, ra = a.cnn_get()
    a.close()

    magic, version, n_sub, ch, step, n_params = struct.unpack_from("<8sIiiiq", ck, 0)
    assert (magic, version, n_sub, ch, step) == (b"SYNIMCNN", 1, 40, 32, 1024 // 128)
    assert n_params == P0.size and len(ck) == 128 + 3 * 4 * P0.size
    np.testing.assert_array_equal(np.frombuffer(ck, np.float64, 8, 32), list(NORM_C) + list(NORM_R))

    b = fresh()
    b.cnn_load(tmp_path / "net.ckpt")
    assert b.cnn_save() == ck                       # the round trip is exact
    b.cnn_train(p2, epochs=1, batch=128, lr=2e-3, seed=7)
    wb, cb, rb = b.cnn_get()
    np.testing.assert_array_equal(wb, wa)
    np.testing.assert_array_equal(cb, ca)
    np.testing.assert_array_equal(rb, ra)
    for bad in (b"XXXXXXXX" + ck[8:], ck[:-4], ck[:100]):
        with pytest.raises(abi.SynimError) as e:
            b.cnn_load(bad)
        assert e.value.status == 1
    b.close()
    c = SynIM(wl.dms, wl.wfss)
    c.probe_attach(0, 0, np.vstack([cmd, cmd]))     # 32 modes: 64 channels
    with pytest.raises(abi.SynimError) as e:
        c.cnn_load(ck)
    assert e.value.status == 2
    c.close()
