"""Oracle: the per-subdomain MLP of the learned initial guess (FP64).

Not in the paper: the guess is an addition to the method (the paper only
requires some starting value u^0 for Newton, Section 3c).  Network: input x
(per subdomain, traces of the last three time steps, zero-padded), two hidden
layers of 256 with ReLU, linear output; loss = mean over the real (unpadded)
outputs of the squared error, summed over the batch of subdomains:
    L = sum_j sum_o mask_jo (y_jo - t_jo)^2 / sum(mask).
Adam (Kingma & Ba, 2015) with bias correction updates the parameters.

The weights used by the forward pass are bfloat16 values; the oracle takes them
as given (already rounded), so GPU and oracle differ only by FP32 rounding.

Pinned by central finite differences of L in every parameter block (tests).
"""
from __future__ import annotations

import numpy as np


def init_params(n_in, n_hidden, n_out, seed=0):
    """He-uniform weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)

    def lin(n_i, n_o):
        lim = np.sqrt(6.0 / n_i)
        return rng.uniform(-lim, lim, size=(n_o, n_i)), np.zeros(n_o)

    W1, b1 = lin(n_in, n_hidden)
    W2, b2 = lin(n_hidden, n_hidden)
    W3, b3 = lin(n_hidden, n_out)
    W3 *= 0.1
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)


def forward(p, X):
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grads(p, X, T, mask):
    y, (X, z1, h1, z2, h2) = forward(p, X)
    cnt = mask.sum()
    r = (y - T) * mask
    L = float((r * r).sum() / cnt)
    dy = 2.0 * r / cnt
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return L, g


def adam_step(p, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v per parameter and the step count."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[:] = beta1 * m + (1 - beta1) * g[k]
        v[:] = beta2 * v + (1 - beta2) * g[k] * g[k]
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
