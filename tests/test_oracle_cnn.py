"""Pins of the FP64 oracle of the estimator network (oracle/cnn.py): the
convolution layout against the explicit sum that defines it, the output
sizes, and the gradient against central finite differences."""
import numpy as np

import oracle.cnn as oc
from paper_2606_07759_b300.synim import cnn_init_params


def _explicit_conv(x, W, b, stride):
    B, H, _, C = x.shape
    Ho = (H - 1) // stride + 1
    out = np.zeros((B, Ho, Ho, W.shape[0]))
    for n in range(B):
        for y in range(Ho):
            for xx in range(Ho):
                acc = b.copy()
                for ky in range(3):
                    for kx in range(3):
                        iy, ix = y * stride + ky - 1, xx * stride + kx - 1
                        if 0 <= iy < H and 0 <= ix < H:
                            acc += W[:, ky, kx, :] @ x[n, iy, ix, :]
                out[n, y, xx] = np.maximum(acc, 0.0)
    return out


def test_convolution_layout_matches_explicit_sum():
    rng = np.random.default_rng(0)
    p = cnn_init_params(32, seed=1, side=5).astype(np.float64)
    p += rng.normal(0, 0.01, p.shape)        # non-zero biases too
    x = rng.standard_normal((2, 5, 5, 32))
    t = oc.unpack(p, 32, 5)
    import torch
    a1, a2, a3, g, out = [v.numpy() for v in oc.layers(t, torch.as_tensor(x))]
    W1, b1, W2, b2, W3, b3, Wfc, bfc = [v.numpy() for v in t]
    e1 = _explicit_conv(x, W1, b1, 1)
    e2 = _explicit_conv(e1, W2, b2, 2)
    e3 = _explicit_conv(e2, W3, b3, 2)
    np.testing.assert_allclose(a1, e1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a2, e2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a3, e3, rtol=0, atol=1e-12)
    assert a2.shape[1] == 3 and a3.shape[1] == 2
    np.testing.assert_allclose(out, e3.reshape(2, -1) @ Wfc.reshape(4, -1).T + bfc, rtol=0, atol=1e-12)


def test_output_sizes_of_the_learned_geometry():
    import torch
    p = cnn_init_params(32)
    a1, a2, a3, g, out = oc.layers(oc.unpack(p, 32, 40), torch.zeros((1, 40, 40, 32), dtype=torch.float64))
    assert a1.shape == (1, 40, 40, 64) and a2.shape == (1, 20, 20, 64) and a3.shape == (1, 10, 10, 64)
    assert out.shape == (1, 4)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    p = cnn_init_params(32, seed=3, side=6).astype(np.float64)
    p += rng.normal(0, 0.02, p.shape)
    x = rng.standard_normal((2, 6, 6, 32))
    tgt = rng.uniform(-1, 1, (2, 4))
    _, g = oc.loss_grad(p, x, tgt, 32)
    n1 = 64 * 9 * 32
    # entries of every tensor: W1, b1, W2, b2, W3, b3, Wfc, bfc
    idx = [5, 1000, n1 + 3, n1 + 64 + 77, n1 + 64 + 36864 + 10, n1 + 64 + 36864 + 64 + 999,
           n1 + 2 * (64 + 36864) + 5, len(p) - 4 * 2 * 2 * 64 - 4 + 17, len(p) - 2]
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (oc.loss_grad(p + e, x, tgt, 32)[0] - oc.loss_grad(p - e, x, tgt, 32)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3), (i, fd, g[i])


def test_written_out_backward_equals_autograd():
    rng = np.random.default_rng(7)
    p = cnn_init_params(32, seed=8, side=8).astype(np.float64)
    p += rng.normal(0, 0.02, p.shape)
    x = rng.standard_normal((3, 8, 8, 32))
    tgt = rng.uniform(-1, 1, (3, 4))
    l0, g0 = oc.loss_grad(p, x, tgt, 32)
    l1, g1 = oc.loss_grad_rounded(p, x, tgt, 32, rounded=False)
    assert abs(l0 - l1) <= 1e-14 * l0
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-12 * np.abs(g0).max())


def test_bf16_rounding_helper_matches_torch():
    import torch
    from oracle.cnn import _bf16
    v = torch.as_tensor(np.random.default_rng(0).standard_normal(5000) * 1e3)
    np.testing.assert_array_equal(_bf16(v).numpy(), v.to(torch.bfloat16).to(torch.float64).numpy())
