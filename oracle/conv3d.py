"""Reference 3-D convolutional network for the learned warm start (ORACLE).

Test infrastructure only: the product path never imports this module.

Plain float64 numpy: 3x3x3 'same' convolutions (zero padding) written as a sum
over the 27 shifted copies of the padded input, ReLU after every layer but
the last, a logistic output, mean-squared-error loss, and the gradient by the
chain rule: the weight gradient correlates the output gradient with the
shifted inputs, the input gradient convolves the output gradient with the
spatially flipped, channel-transposed weights.  Hidden layers use a leaky
ReLU with slope 1/100.  Weights are [Co][Ci][3][3][3]
with taps ordered (dz, dy, dx), each in {-1, 0, 1}.
"""
from __future__ import annotations

import numpy as np

LEAK = 0.01


def _shift(xp, dz, dy, dx, D, H, W):
    return xp[:, :, dz:dz + D, dy:dy + H, dx:dx + W]


def conv3d_same(x, w, b):
    B, Ci, D, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.zeros((B, w.shape[0], D, H, W)) + b[None, :, None, None, None]
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out += np.einsum("oc,bcdhw->bodhw", w[:, :, dz, dy, dx], _shift(xp, dz, dy, dx, D, H, W))
    return out


def forward(params, x):
    """Activations of every layer (the last one is the logistic output)."""
    acts = []
    h = x
    for l, (w, b) in enumerate(params):
        z = conv3d_same(h, w, b)
        h = 1.0 / (1.0 + np.exp(-z)) if l + 1 == len(params) else np.where(z > 0, z, LEAK * z)
        acts.append(h)
    return acts


def loss_and_grad(params, x, t, w=None):
    """Loss of the output against t and its parameter gradient.

    Without w the pressure MSE; with per-cell face-flux weights w (the sum of
    T_R^2 over the cell's Robin faces) the squared flux errors T_R (y - t) of
    those faces are added: mean((1 + w) (y - t)^2).
    """
    acts = forward(params, x)
    y = acts[-1]
    n = y.size
    wt = 1.0 if w is None else 1.0 + w
    loss = float(np.sum(wt * (y - t) ** 2) / n)
    g = 2.0 * wt * (y - t) / n * y * (1.0 - y)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, b = params[l]
        inp = x if l == 0 else acts[l - 1]
        B, Ci, D, H, W = inp.shape
        ip = np.pad(inp, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
        gw = np.zeros_like(w)
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    gw[:, :, dz, dy, dx] = np.einsum("bodhw,bcdhw->oc", g, _shift(ip, dz, dy, dx, D, H, W))
        grads[l] = (gw, g.sum(axis=(0, 2, 3, 4)))
        if l > 0:
            wt = np.transpose(w[:, :, ::-1, ::-1, ::-1], (1, 0, 2, 3, 4))
            g = conv3d_same(g, wt, np.zeros(Ci)) * np.where(inp > 0, 1.0, LEAK)
    return loss, grads


def unflatten(flat, cin, cout):
    """Split a flat parameter vector (per layer: weights then biases) into layers."""
    params, off = [], 0
    for ci, co in zip(cin, cout):
        w = flat[off: off + co * ci * 27].reshape(co, ci, 3, 3, 3)
        off += co * ci * 27
        b = flat[off: off + co]
        off += co
        params.append((np.array(w, dtype=np.float64), np.array(b, dtype=np.float64)))
    return params


def flatten(grads):
    return np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
