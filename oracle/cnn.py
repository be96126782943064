"""FP64 CPU oracle of the learned estimator's network (test infrastructure).

The network (conv 3x3 stride 1 C->64, conv 3x3 stride 2 64->64, conv 3x3
stride 2 64->64, each with bias and ReLU; global average pooling; dense
64->4; mean squared error) written with PyTorch CPU operators in float64,
the gradient by PyTorch's automatic differentiation.  Parameters come as the
flat FP32 vector of the library (W[co][ky][kx][ci] per layer, then biases;
Wfc[j][c]); inputs are NHWC.  Tests pin the convolution layout against an
explicit sum and the gradient against central differences.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def unpack(params, n_channels: int):
    p = torch.as_tensor(np.asarray(params, np.float64))
    shapes = [(64, 3, 3, n_channels), (64,), (64, 3, 3, 64), (64,), (64, 3, 3, 64), (64,), (4, 64), (4,)]
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
    """Activations (a1, a2, a3 NHWC, pooled g, output) of float64 input x [B, H, H, C]."""
    W1, b1, W2, b2, W3, b3, Wfc, bfc = tensors
    h = x.permute(0, 3, 1, 2)
    a1 = F.relu(F.conv2d(h, W1.permute(0, 3, 1, 2), b1, stride=1, padding=1))
    a2 = F.relu(F.conv2d(a1, W2.permute(0, 3, 1, 2), b2, stride=2, padding=1))
    a3 = F.relu(F.conv2d(a2, W3.permute(0, 3, 1, 2), b3, stride=2, padding=1))
    g = a3.mean(dim=(2, 3))
    out = g @ Wfc.T + bfc
    return a1.permute(0, 2, 3, 1), a2.permute(0, 2, 3, 1), a3.permute(0, 2, 3, 1), g, out


def forward(params, x, n_channels: int) -> np.ndarray:
    t = unpack(params, n_channels)
    with torch.no_grad():
        return layers(t, torch.as_tensor(np.asarray(x, np.float64)))[-1].numpy()


def loss_grad(params, x, target, n_channels: int):
    """(mean squared error over the B x 4 outputs, gradient as a flat float64 vector)."""
    t = [v.clone().requires_grad_(True) for v in unpack(params, n_channels)]
    out = layers(t, torch.as_tensor(np.asarray(x, np.float64)))[-1]
    loss = ((out - torch.as_tensor(np.asarray(target, np.float64))) ** 2).mean()
    loss.backward()
    return float(loss.detach()), pack([v.grad for v in t])
