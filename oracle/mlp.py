"""FP64 reference of the pricing surrogate: a fully connected network with
SiLU activations and a linear scalar output, its mean-squared-error loss, the
exact backward pass and one Adam update.

TEST INFRASTRUCTURE ONLY (see the oracle package docstring).

The paper leans on the computational identity between a DNN layer and a
time step of a multivariate simulation (Sec. III.C) and on back-propagation
for sensitivities (Sec. I.A.3); the surrogate that revalues the risk
portfolio is this network, trained on Monte Carlo prices.

Parameter layout (shared by name with the library, held as a list here):
for layer l: W_l of shape [in_l, out_l] (row-major), b_l of shape [out_l];
h_0 = x, z_l = h_l W_l + b_l, h_{l+1} = silu(z_l) for hidden layers, output
y = z_L (shape [n]).  silu(z) = z / (1 + e^{-z}).
Pinned by central finite differences of the loss (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np


def layer_sizes(n_in: int, width: int, hidden: int):
    return [n_in] + [width] * hidden + [1]


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x):
    """params: list of (W, b); x: [n, n_in].  Returns (y [n], cache)."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        z = h @ W + b
        cache.append((h, z))
        h = silu(z) if l < len(params) - 1 else z
    return h[:, 0], cache


def loss_and_grads(params, x, t):
    """MSE loss (1/n) sum (y - t)^2 and its gradients, by the chain rule."""
    y, cache = forward(params, x)
    n = y.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(r * r))
    dh = (2.0 / n) * r[:, None]
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        h, z = cache[l]
        dz = dh if l == len(params) - 1 else dh * silu_grad(z)
        W, _ = params[l]
        grads[l] = (h.T @ dz, dz.sum(axis=0))
        dh = dz @ W.T
    return loss, grads


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of every tensor; returns new lists."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for p_, g_, m_, v_ in ((W, gW, mW, vW), (b, gb, mb, vb)):
            m2 = beta1 * m_ + (1 - beta1) * g_
            v2 = beta2 * v_ + (1 - beta2) * g_ * g_
            mh = m2 / (1 - beta1 ** step)
            vh = v2 / (1 - beta2 ** step)
            new.append((p_ - lr * mh / (np.sqrt(vh) + eps), m2, v2))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v


def pack(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unpack(flat, sizes):
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = np.asarray(flat[o:o + a * b], dtype=np.float64).reshape(a, b)
        o += a * b
        bb = np.asarray(flat[o:o + b], dtype=np.float64)
        o += b
        out.append((W, bb))
    return out
