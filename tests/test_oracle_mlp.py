"""Pins of the FP64 MLP oracle: gradients against central finite differences
of the loss, SiLU derivative against differences, Adam against its first
step's closed form (|update| = lr for every non-zero gradient)."""
import numpy as np

from oracle import mlp


def _params(sizes, rng):
    return [(rng.standard_normal((a, b)) / np.sqrt(a), 0.1 * rng.standard_normal(b))
            for a, b in zip(sizes[:-1], sizes[1:])]


def test_silu_grad_matches_difference():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    assert np.allclose(mlp.silu_grad(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), rtol=1e-8, atol=1e-10)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    sizes = mlp.layer_sizes(5, 7, 3)
    P = _params(sizes, rng)
    x = rng.standard_normal((11, 5))
    t = rng.standard_normal(11)
    loss, grads = mlp.loss_and_grads(P, x, t)
    flat = mlp.pack(P)
    g = mlp.pack(grads)
    h = 1e-6
    for i in rng.choice(flat.size, 60, replace=False):
        up, dn = flat.copy(), flat.copy()
        up[i] += h
        dn[i] -= h
        fd = (mlp.loss_and_grads(mlp.unpack(up, sizes), x, t)[0] -
              mlp.loss_and_grads(mlp.unpack(dn, sizes), x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_first_step_moves_by_lr():
    rng = np.random.default_rng(4)
    sizes = mlp.layer_sizes(5, 4, 2)
    P = _params(sizes, rng)
    _, G = mlp.loss_and_grads(P, rng.standard_normal((8, 5)), rng.standard_normal(8))
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in P]
    P2, _, _ = mlp.adam_step(P, G, zeros, zeros, 1, 1e-3)
    d = np.abs(mlp.pack(P2) - mlp.pack(P))
    g = np.abs(mlp.pack(G))
    assert np.allclose(d[g > 1e-6], 1e-3, rtol=1e-3)


def test_pack_roundtrip():
    rng = np.random.default_rng(5)
    sizes = mlp.layer_sizes(5, 16, 4)
    P = _params(sizes, rng)
    Q = mlp.unpack(mlp.pack(P), sizes)
    assert all(np.array_equal(a, c) and np.array_equal(b, d) for (a, b), (c, d) in zip(P, Q))
    assert mlp.pack(P).size == 5 * 16 + 16 + 3 * (16 * 16 + 16) + 16 + 1
