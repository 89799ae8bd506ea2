"""GPU parity of the surrogate network's kernels with the FP64 oracle
(oracle/mlp.py): forward, MSE loss, back-propagated gradient, one Adam step,
and that native training reduces the loss."""
import numpy as np
import pytest

import workloads
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

SIZES = omlp.layer_sizes(5, 256, 4)


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def _data(n, seed=1):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(n, 5)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2] - 0.5 * x[:, 3] ** 2 + 0.1 * x[:, 4]).astype(np.float32)
    return x, t


def test_forward_fp32_matches_oracle(gb):
    import torch
    init = workloads.mlp_init()
    net = gb.Mlp(5, 256, 4, init)
    x, _ = _data(1000)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = omlp.forward(omlp.unpack(init.astype(np.float64), SIZES), x.astype(np.float64))
    assert np.max(np.abs(y - want)) <= 1e-5 * np.max(np.abs(want)) + 1e-6
    net.close()


def test_loss_and_gradient_match_oracle(gb):
    import torch
    init = workloads.mlp_init(seed=7)
    net = gb.Mlp(5, 256, 4, init)
    x, t = _data(777, seed=2)
    loss, g = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    P = omlp.unpack(init.astype(np.float64), SIZES)
    l_ref, G = omlp.loss_and_grads(P, x.astype(np.float64), t.astype(np.float64))
    g_ref = omlp.pack(G)
    assert abs(loss - l_ref) <= 1e-5 * l_ref
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * scale, np.max(np.abs(g - g_ref)) / scale
    net.close()


def test_one_adam_step_matches_oracle(gb):
    import torch
    init = workloads.mlp_init(seed=8)
    net = gb.Mlp(5, 256, 4, init)
    x, t = _data(512, seed=3)
    net.train(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), epochs=1, batch=512, lr=1e-3)
    P = omlp.unpack(init.astype(np.float64), SIZES)
    _, G = omlp.loss_and_grads(P, x.astype(np.float64), t.astype(np.float64))
    Z = [(np.zeros_like(W), np.zeros_like(b)) for W, b in P]
    P1, _, _ = omlp.adam_step(P, G, Z, Z, 1, 1e-3)
    got, want, g = net.params(), omlp.pack(P1), np.abs(omlp.pack(G))
    big = g > 1e-4 * g.max()  # Adam's first step is lr * sign(g): compare where the sign is resolved
    assert np.max(np.abs(got[big] - want[big])) <= 1e-6 + 1e-6 * np.max(np.abs(want))
    net.close()


def test_training_reduces_loss(gb):
    import torch
    net = gb.Mlp(5, 256, 4, workloads.mlp_init(seed=9))
    x, t = _data(1 << 15, seed=4)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0, _ = net.loss_grad(xd, td)
    l1 = net.train(xd, td, epochs=20, batch=1024, lr=1e-3)
    assert l1 < 0.05 * l0, (l0, l1)
    net.close()
