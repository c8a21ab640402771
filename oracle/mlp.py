"""FP64 CPU reference of the surrogate network (test infrastructure only,
same import rule as the rest of ``oracle``).

A fully connected network x -> tanh(x W_1 + b_1) -> ... -> tanh(. W_D + b_D)
-> (. W_out + b_out) with a mean-squared-error loss
L = sum((y - t)^2) / (batch * n_out), and one Adam step
(Kingma & Ba: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr m_hat / (sqrt(v_hat) + eps), m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t)).

Parameters are one flat vector in this order, layer by layer: W (n_in x
n_out, row-major: W[i, j] multiplies input i into output j), then b (n_out).
The backward pass is written out by hand (chain rule), not by automatic
differentiation, and is pinned against central finite differences in the
tests.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(n_in, width, depth, n_out):
    dims = [n_in] + [width] * depth + [n_out]
    return [(dims[l], dims[l + 1]) for l in range(len(dims) - 1)]


def num_params(n_in, width, depth, n_out):
    return sum(a * b + b for a, b in layer_shapes(n_in, width, depth, n_out))


def unpack(theta, n_in, width, depth, n_out):
    out, o = [], 0
    for a, b in layer_shapes(n_in, width, depth, n_out):
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bias = theta[o:o + b]
        o += b
        out.append((W, bias))
    return out


def forward(theta, x, n_in, width, depth, n_out):
    """Returns (y, cache) with cache = list of layer inputs and outputs."""
    layers = unpack(theta, n_in, width, depth, n_out)
    h = np.asarray(x, dtype=np.float64)
    acts = [h]
    for l, (W, b) in enumerate(layers):
        z = h @ W + b
        h = np.tanh(z) if l < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grad(theta, x, t, n_in, width, depth, n_out):
    y, acts = forward(theta, x, n_in, width, depth, n_out)
    B = y.shape[0]
    d = y - t
    loss = float((d * d).sum() / (B * n_out))
    dz = 2.0 * d / (B * n_out)            # dL/dy, the output layer is linear
    layers = unpack(theta, n_in, width, depth, n_out)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        h_in = acts[l]
        grads[l] = (h_in.T @ dz, dz.sum(axis=0))
        if l > 0:
            dh = dz @ W.T
            dz = dh * (1.0 - acts[l] ** 2)   # tanh' = 1 - tanh^2
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
