"""Oracle: the per-subdomain MLP of the learned initial guess (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Not in the paper: the guess is an addition to the method (the paper only
requires some starting value u^0 for Newton, Section 3c).  Network: input x
(per subdomain, traces of the last three time steps on the subdomain's
interface, zero-padded), two hidden layers of 256 with ReLU, linear output;
loss = mean over the real (unpadded) outputs of the squared error, summed over
the batch of subdomains:
    L = sum_j sum_o mask_jo (y_jo - t_jo)^2 / sum(mask).
Adam (Kingma & Ba, 2015, Algorithm 1) with bias correction updates the
parameters.

Precision of the network as the GPU defines it (bf16=True): every operand of a
matrix product is a bfloat16 value (weights, inputs, hidden activations, and the
output and hidden gradients entering the backward products), accumulation and
everything else is FP32 on the GPU and FP64 here.  The rounding points are:
    Xb = bf16(X); Z1 = Xb W1b^T + b1; H1b = bf16(relu(Z1)); Z2 = H1b W2b^T + b2;
    H2b = bf16(relu(Z2)); Y = H2b W3b^T + b3;
    dY = 2 mask (Y - T) / cnt; dW3 = bf16(dY)^T H2b; dZ2 = (bf16(dY) W3b) * (Z2 > 0);
    dW2 = bf16(dZ2)^T H1b; dZ1 = (bf16(dZ2) W2b) * (Z1 > 0); dW1 = bf16(dZ1)^T Xb;
    db_k = column sums of the unrounded dZ_k (dY for db3).
bf16() is round to nearest, ties to even, of the value's binary expansion.

Pinned by central finite differences of L in every parameter block (bf16=False),
by the rounding against torch's float32 -> bfloat16 conversion, and by Adam
values worked out by hand (tests).
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to the nearest bfloat16 value (ties to even), returned as float64.

    A bfloat16 keeps the sign, the 8 exponent bits and the top 7 fraction bits of a
    float32.  The value is first rounded to float32 (exact for the float32 inputs the
    GPU rounds), then its 32-bit pattern is rounded at bit 16."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    keep = (b >> 16) & 1
    r = ((b + 0x7FFF + keep) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out.reshape(np.shape(a))


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


def _r(a, on):
    return bf16(a) if on else a


def forward(p, X, bf=False):
    W1, W2, W3 = (_r(p[k], bf) for k in ("W1", "W2", "W3"))
    Xb = _r(X, bf)
    z1 = Xb @ W1.T + p["b1"]
    h1 = _r(np.maximum(z1, 0.0), bf)
    z2 = h1 @ W2.T + p["b2"]
    h2 = _r(np.maximum(z2, 0.0), bf)
    y = h2 @ W3.T + p["b3"]
    return y, (Xb, z1, h1, z2, h2)


def loss_and_grads(p, X, T, mask, bf=False):
    y, (X, z1, h1, z2, h2) = forward(p, X, bf)
    W2, W3 = _r(p["W2"], bf), _r(p["W3"], bf)
    cnt = mask.sum()
    r = (y - T) * mask
    L = float((r * r).sum() / cnt)
    dy = 2.0 * r / cnt
    g = {}
    dyb = _r(dy, bf)
    g["W3"] = dyb.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dyb @ W3
    dz2 = dh2 * (z2 > 0)
    dz2b = _r(dz2, bf)
    g["W2"] = dz2b.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2b @ W2
    dz1 = dh1 * (z1 > 0)
    g["W1"] = _r(dz1, bf).T @ X
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
