"""FP64 reference of the planner's small fully connected network.

TEST INFRASTRUCTURE ONLY (see the package header).  Written from the
definitions: layer l maps x -> act(W_l x + b_l) with W_l of shape
(d_{l+1}, d_l), ReLU on hidden layers and the identity on the last; the loss
is the mean of the squared differences over every output element; gradients
by the chain rule, layer by layer; Adam (Kingma and Ba, 2015) with bias
correction, beta1 = 0.9, beta2 = 0.999, eps = 1e-8.  Parameters are one flat
vector packed per layer as W_l (row-major) followed by b_l, the layout the
C ABI uses.
"""

from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def unpack(dims: Sequence[int], params: np.ndarray) -> List[Tuple[np.ndarray, np.ndarray]]:
    layers, at = [], 0
    for l in range(len(dims) - 1):
        n_w = dims[l + 1] * dims[l]
        W = params[at:at + n_w].reshape(dims[l + 1], dims[l])
        at += n_w
        b = params[at:at + dims[l + 1]]
        at += dims[l + 1]
        layers.append((W, b))
    if at != len(params):
        raise ValueError("parameter vector does not match dims")
    return layers


def param_count(dims: Sequence[int]) -> int:
    return sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))


def forward(dims, params, x):
    """Returns the list of layer outputs a_1..a_L (a_L is the prediction)."""
    layers = unpack(dims, np.asarray(params, dtype=np.float64))
    a = np.asarray(x, dtype=np.float64)
    outs = []
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = np.maximum(z, 0.0) if l + 1 < len(layers) else z
        outs.append(a)
    return outs


def loss(dims, params, x, t) -> float:
    y = forward(dims, params, x)[-1]
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(dims, params, x, t) -> np.ndarray:
    """d loss / d params by the chain rule (reverse order over the layers)."""
    params = np.asarray(params, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    layers = unpack(dims, params)
    outs = forward(dims, params, x)
    y = outs[-1]
    dz = 2.0 * (y - np.asarray(t, dtype=np.float64)) / y.size  # last layer is linear
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        a_in = x if l == 0 else outs[l - 1]
        W, _ = layers[l]
        grads.append((dz.T @ a_in, dz.sum(axis=0)))
        if l > 0:
            da = dz @ W
            dz = da * (outs[l - 1] > 0.0)  # ReLU derivative of the layer below
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return np.concatenate(flat)


def adam_steps(dims, params, x, t, epochs, lr, m=None, v=None):
    """`epochs` full-batch Adam steps; returns (params, m, v, losses)."""
    b1, b2, eps = 0.9, 0.999, 1e-8
    p = np.array(params, dtype=np.float64)
    m = np.zeros_like(p) if m is None else np.array(m, dtype=np.float64)
    v = np.zeros_like(p) if v is None else np.array(v, dtype=np.float64)
    losses = []
    for ep in range(epochs):
        losses.append(loss(dims, p, x, t))
        g = gradient(dims, p, x, t)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        mhat = m / (1 - b1 ** (ep + 1))
        vhat = v / (1 - b2 ** (ep + 1))
        p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v, losses
