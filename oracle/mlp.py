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
Pinned by central finite differences of the loss (tests/test_oracle_mlp.py);
the derivative-label loss (dloss_and_grads) by finite differences of the
network in its inputs and of that loss in the parameters, and by its
reduction to the plain loss when every derivative weight is zero.
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


def silu_grad2(z):
    """Second derivative of silu: s (1 - s) (2 + z (1 - 2 s)), s = 1 / (1 + e^{-z})."""
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s))


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


def input_grads(params, x, dirs):
    """dy/dx_j for every input index j in dirs, shape [n, len(dirs)]: the
    chain rule carried forward layer by layer (one tangent per direction:
    dz_l = dh_l W_l, dh_{l+1} = silu'(z_l) dz_l, starting from the unit
    vector e_j)."""
    h = np.asarray(x, dtype=np.float64)
    n = h.shape[0]
    out = np.empty((n, len(dirs)))
    for k, j in enumerate(dirs):
        hh, dh = h, np.zeros_like(h)
        dh[:, j] = 1.0
        for l, (W, b) in enumerate(params):
            z = hh @ W + b
            dz = dh @ W
            if l < len(params) - 1:
                hh, dh = silu(z), silu_grad(z) * dz
            else:
                hh, dh = z, dz
        out[:, k] = dh[:, 0]
    return out


def dloss_and_grads(params, x, t, g, dirs, lams):
    """Loss with derivative labels (the network fitted to prices and to
    their sensitivities, Sec. I.A.3):
        L = (1/n) sum_i [(y_i - t_i)^2 + sum_k lam_k m_ik (dy_i/dx_{j_k} - g_ik)^2],
    m_ik = 1 where g_ik is finite, else 0 (no label), and its gradient with
    respect to every parameter.  Forward: the primal activations and, per
    direction k, the tangents dz_l^k = dh_l^k W_l, dh_{l+1}^k = silu'(z_l) dz_l^k
    (dh_0^k = e_{j_k}).  Reverse, through both:
        W_l-bar = h_l^T z_l-bar + sum_k dh_l^kT dz_l^k-bar,  b_l-bar = sum_i z_l-bar,
        h_l-bar = z_l-bar W_l^T,  dh_l^k-bar = dz_l^k-bar W_l^T,
        z_{l-1}-bar = h_l-bar silu'(z) + sum_k dh_l^k-bar silu''(z) dz_{l-1}^k,
        dz_{l-1}^k-bar = dh_l^k-bar silu'(z),
    seeded with y-bar = 2 (y - t) / n and dy^k-bar = 2 lam_k m_k (dy^k - g_k) / n.
    Returns (loss, parts [1 + K] = price term then each direction's term, grads)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64).reshape(x.shape[0], len(dirs))
    n, K, L = x.shape[0], len(dirs), len(params)
    hs, zs, dhs, dzs = [x], [], [], []
    dh = np.zeros((K, n, x.shape[1]))
    for k, j in enumerate(dirs):
        dh[k, :, j] = 1.0
    dhs.append(dh)
    h = x
    for l, (W, b) in enumerate(params):
        z = h @ W + b
        dz = dh @ W  # [K, n, out]
        zs.append(z)
        dzs.append(dz)
        if l < L - 1:
            h, dh = silu(z), silu_grad(z)[None] * dz
        else:
            h, dh = z, dz
        hs.append(h)
        dhs.append(dh)
    y, dy = hs[-1][:, 0], dhs[-1][:, :, 0]  # [n], [K, n]
    m = np.isfinite(g).T.astype(np.float64)  # [K, n]
    gz = np.where(np.isfinite(g), g, 0.0).T
    r, rd = y - t, m * (dy - gz)
    parts = [float(np.mean(r * r))] + [float(lams[k] * np.mean(rd[k] * rd[k])) for k in range(K)]
    zbar = (2.0 / n) * r[:, None]
    dzbar = np.stack([(2.0 * lams[k] / n) * rd[k][:, None] for k in range(K)]) if K else np.zeros((0, n, 1))
    grads = [None] * L
    for l in range(L - 1, -1, -1):
        W, _ = params[l]
        gW = hs[l].T @ zbar + sum(dhs[l][k].T @ dzbar[k] for k in range(K))
        grads[l] = (gW, zbar.sum(axis=0))
        if l == 0:
            break
        hbar = zbar @ W.T
        dhbar = dzbar @ W.T
        z = zs[l - 1]
        zbar = hbar * silu_grad(z) + sum(dhbar[k] * silu_grad2(z) * dzs[l - 1][k] for k in range(K))
        dzbar = dhbar * silu_grad(z)[None]
    return float(sum(parts)), parts, grads


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
