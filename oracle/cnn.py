"""FP64 CPU oracle of the learned estimator's network (test infrastructure).

The network (conv 3x3 stride 1 C->64, conv 3x3 stride 2 64->64, conv 3x3
stride 2 64->64, each with bias and ReLU; dense layer from the flattened
last feature map (H3 x H3 x 64, NHWC order) to 4 outputs; mean squared
error) written with PyTorch CPU operators in float64,
the gradient by PyTorch's automatic differentiation.  Parameters come as the
flat FP32 vector of the library (W[co][ky][kx][ci] per layer, then biases;
Wfc[j][y][x][c]); inputs are NHWC.  Tests pin the convolution layout against an
explicit sum and the gradient against central differences.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def feature_side(h0: int) -> int:
    """Side of the last feature map: two stride-2 convolutions of an h0 map."""
    h = (h0 - 1) // 2 + 1
    return (h - 1) // 2 + 1


def unpack(params, n_channels: int, h0: int = 40):
    p = torch.as_tensor(np.asarray(params, np.float64))
    h3 = feature_side(h0)
    shapes = [(64, 3, 3, n_channels), (64,), (64, 3, 3, 64), (64,), (64, 3, 3, 64), (64,), (4, h3, h3, 64), (4,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    assert o == p.numel(), (o, p.numel())
    return out


def pack(tensors) -> np.ndarray:
    return np.concatenate([t.detach().reshape(-1).numpy() for t in tensors])


def layers(tensors, x):
    """Activations (a1, a2, a3 NHWC, flattened features g, output) of float64 input x [B, H, H, C]."""
    W1, b1, W2, b2, W3, b3, Wfc, bfc = tensors
    h = x.permute(0, 3, 1, 2)
    a1 = F.relu(F.conv2d(h, W1.permute(0, 3, 1, 2), b1, stride=1, padding=1))
    a2 = F.relu(F.conv2d(a1, W2.permute(0, 3, 1, 2), b2, stride=2, padding=1))
    a3 = F.relu(F.conv2d(a2, W3.permute(0, 3, 1, 2), b3, stride=2, padding=1))
    a3h = a3.permute(0, 2, 3, 1)
    g = a3h.reshape(a3h.shape[0], -1)
    out = g @ Wfc.reshape(4, -1).T + bfc
    return a1.permute(0, 2, 3, 1), a2.permute(0, 2, 3, 1), a3h, g, out


def forward(params, x, n_channels: int) -> np.ndarray:
    t = unpack(params, n_channels, np.shape(x)[1])
    with torch.no_grad():
        return layers(t, torch.as_tensor(np.asarray(x, np.float64)))[-1].numpy()


def loss_grad(params, x, target, n_channels: int):
    """(mean squared error over the B x 4 outputs, gradient as a flat float64 vector)."""
    t = [v.clone().requires_grad_(True) for v in unpack(params, n_channels, np.shape(x)[1])]
    out = layers(t, torch.as_tensor(np.asarray(x, np.float64)))[-1]
    loss = ((out - torch.as_tensor(np.asarray(target, np.float64))) ** 2).mean()
    loss.backward()
    return float(loss.detach()), pack([v.grad for v in t])


def _bf16(t):
    """Round a float64 tensor to the nearest bfloat16 (ties to even), via float32."""
    f = t.to(torch.float32).contiguous()
    u = f.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    u = torch.where(u >= 2 ** 31, u - 2 ** 32, u).to(torch.int32)
    return u.view(torch.float32).to(torch.float64)


def loss_grad_rounded(params, x, target, n_channels: int, rounded: bool = True):
    """Loss and gradient with the backward pass written out layer by layer and,
    when `rounded`, every stored activation (a1, a2, a3) and activation
    gradient (dz3, dz2, dz1) rounded to bfloat16: the precision model of a
    BF16 training step, all arithmetic in between in float64.  With
    rounded=False this is the exact gradient (a test checks it against
    loss_grad)."""
    R = _bf16 if rounded else (lambda v: v)
    W1, b1, W2, b2, W3, b3, Wfc, bfc = unpack(params, n_channels, np.shape(x)[1])
    x = torch.as_tensor(np.asarray(x, np.float64))
    t = torch.as_tensor(np.asarray(target, np.float64))
    h = x.permute(0, 3, 1, 2)
    Wc = [w.permute(0, 3, 1, 2) for w in (W1, W2, W3)]
    a1 = R(F.relu(F.conv2d(h, Wc[0], b1, stride=1, padding=1)))
    a2 = R(F.relu(F.conv2d(a1, Wc[1], b2, stride=2, padding=1)))
    a3 = R(F.relu(F.conv2d(a2, Wc[2], b3, stride=2, padding=1)))
    a3h = a3.permute(0, 2, 3, 1)
    g = a3h.reshape(a3h.shape[0], -1)
    Wf = Wfc.reshape(4, -1)
    out = g @ Wf.T + bfc
    B = x.shape[0]
    dout = 2.0 * (out - t) / (4.0 * B)
    dWfc, dbfc = (dout.T @ g).reshape(Wfc.shape), dout.sum(0)
    dz3 = R((dout @ Wf).reshape(a3h.shape).permute(0, 3, 1, 2) * (a3 > 0))
    dW3 = torch.nn.grad.conv2d_weight(a2, Wc[2].shape, dz3, stride=2, padding=1)
    dz2 = R(torch.nn.grad.conv2d_input(a2.shape, Wc[2], dz3, stride=2, padding=1) * (a2 > 0))
    dW2 = torch.nn.grad.conv2d_weight(a1, Wc[1].shape, dz2, stride=2, padding=1)
    dz1 = R(torch.nn.grad.conv2d_input(a1.shape, Wc[1], dz2, stride=2, padding=1) * (a1 > 0))
    dW1 = torch.nn.grad.conv2d_weight(h, Wc[0].shape, dz1, stride=1, padding=1)
    grads = [dW1.permute(0, 2, 3, 1), dz1.sum((0, 2, 3)), dW2.permute(0, 2, 3, 1), dz2.sum((0, 2, 3)),
             dW3.permute(0, 2, 3, 1), dz3.sum((0, 2, 3)), dWfc, dbfc]
    return float(((out - t) ** 2).mean()), pack(grads)
