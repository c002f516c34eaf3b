"""CPU oracle of the learned-background network -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy statement of the small convolutional network that maps
per-box quantile features to the background / rms mesh: 3x3 convolutions
with zero padding ("same" size), bias, ReLU between layers, a linear output
layer, and the mean-squared-error loss.  Forward and backward passes are
written out directly (no autograd), so the GPU kernels' gradients can be
checked against them; the backward pass itself is pinned by finite
differences in tests/test_cnn_oracle.py.

Layouts: activations NHWC (batch, height, width, channels); weights
W[co, ci, dy, dx] with dy, dx in 0..2 standing for offsets -1..+1; the
output at (y, x) is sum over ci, dy, dx of W[co, ci, dy, dx] x[y+dy-1, x+dx-1, ci].
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, W, b):
    """x: (N, H, W, Ci); W: (Co, Ci, 3, 3); b: (Co,) -> (N, H, W, Co)."""
    N, H, Wd, Ci = x.shape
    xp = np.zeros((N, H + 2, Wd + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    out = np.zeros((N, H, Wd, W.shape[0]))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("nhwc,oc->nhwo", xp[:, dy:dy + H, dx:dx + Wd, :], W[:, :, dy, dx])
    return out + b[None, None, None, :]


def conv3x3_backward(x, W, dout):
    """Gradients of conv3x3 with respect to x, W and b, given dL/dout."""
    N, H, Wd, Ci = x.shape
    xp = np.zeros((N, H + 2, Wd + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            dW[:, :, dy, dx] = np.einsum("nhwo,nhwc->oc", dout, xp[:, dy:dy + H, dx:dx + Wd, :])
            dxp[:, dy:dy + H, dx:dx + Wd, :] += np.einsum("nhwo,oc->nhwc", dout, W[:, :, dy, dx])
    db = dout.sum(axis=(0, 1, 2))
    return dxp[:, 1:-1, 1:-1, :], dW, db


def forward(x, params):
    """params: list of (W, b).  Returns the list of layer outputs (after the
    activation; the last one linear)."""
    acts = [x]
    for i, (W, b) in enumerate(params):
        y = conv3x3(acts[-1], W, b)
        if i + 1 < len(params):
            y = np.maximum(y, 0.0)
        acts.append(y)
    return acts


def mse(pred, target):
    return float(np.mean((pred - target) ** 2))


def backward(acts, params, target):
    """Gradients of the mean-squared error with respect to every (W, b),
    plus dL/d(layer output) of each layer (for per-layer checks)."""
    grads = [None] * len(params)
    dys = [None] * len(params)
    d = 2.0 * (acts[-1] - target) / target.size
    for i in range(len(params) - 1, -1, -1):
        if i + 1 < len(params):
            d = d * (acts[i + 1] > 0)          # ReLU
        dys[i] = d
        dx, dW, db = conv3x3_backward(acts[i], params[i][0], d)
        grads[i] = (dW, db)
        d = dx
    return grads, dys


def bf16_round(a):
    """Round FP32/FP64 values to bfloat16 (nearest, ties to even), as the GPU
    stores weights and activations."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
