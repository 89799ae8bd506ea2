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


def test_silu_second_derivative_matches_difference():
    z = np.linspace(-8, 8, 101)
    h = 1e-5
    assert np.allclose(mlp.silu_grad2(z), (mlp.silu_grad(z + h) - mlp.silu_grad(z - h)) / (2 * h), rtol=1e-7,
                       atol=1e-9)


def test_input_grads_match_finite_differences():
    rng = np.random.default_rng(6)
    sizes = mlp.layer_sizes(5, 9, 3)
    P = _params(sizes, rng)
    x = rng.standard_normal((13, 5))
    dirs = [0, 1, 4]
    got = mlp.input_grads(P, x, dirs)
    h = 1e-6
    for k, j in enumerate(dirs):
        up, dn = x.copy(), x.copy()
        up[:, j] += h
        dn[:, j] -= h
        fd = (mlp.forward(P, up)[0] - mlp.forward(P, dn)[0]) / (2 * h)
        assert np.allclose(got[:, k], fd, rtol=1e-7, atol=1e-9)


def test_derivative_loss_gradient_matches_finite_differences():
    """Every part of the derivative-label loss: masked labels (NaN) included,
    unequal weights, directions not in input order."""
    rng = np.random.default_rng(7)
    sizes = mlp.layer_sizes(5, 7, 3)
    P = _params(sizes, rng)
    x = rng.standard_normal((12, 5))
    t = rng.standard_normal(12)
    dirs, lams = [1, 0], [0.7, 2.5]
    g = rng.standard_normal((12, 2))
    g[3, 0] = g[7, 1] = g[9, :] = np.nan
    loss, parts, grads = mlp.dloss_and_grads(P, x, t, g, dirs, lams)
    dy = mlp.input_grads(P, x, dirs)
    y = mlp.forward(P, x)[0]
    ok = np.isfinite(g)
    want = [np.mean((y - t) ** 2)] + [lams[k] * np.mean(np.where(ok[:, k], dy[:, k] - np.nan_to_num(g[:, k]), 0) ** 2)
                                      for k in range(2)]
    assert np.allclose(parts, want, rtol=1e-12) and abs(loss - sum(want)) <= 1e-12 * abs(loss)
    flat, gf = mlp.pack(P), mlp.pack(grads)
    h = 1e-6
    for i in rng.choice(flat.size, 80, replace=False):
        up, dn = flat.copy(), flat.copy()
        up[i] += h
        dn[i] -= h
        fd = (mlp.dloss_and_grads(mlp.unpack(up, sizes), x, t, g, dirs, lams)[0] -
              mlp.dloss_and_grads(mlp.unpack(dn, sizes), x, t, g, dirs, lams)[0]) / (2 * h)
        assert abs(fd - gf[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, gf[i])


def test_derivative_loss_without_weights_is_the_plain_loss():
    rng = np.random.default_rng(8)
    sizes = mlp.layer_sizes(5, 6, 2)
    P = _params(sizes, rng)
    x, t = rng.standard_normal((9, 5)), rng.standard_normal(9)
    a, _, ga = mlp.dloss_and_grads(P, x, t, rng.standard_normal((9, 2)), [0, 1], [0.0, 0.0])
    b, gb = mlp.loss_and_grads(P, x, t)
    assert abs(a - b) <= 1e-14 * b
    assert np.allclose(mlp.pack(ga), mlp.pack(gb), rtol=1e-12, atol=1e-15)
