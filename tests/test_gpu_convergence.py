"""Two of the paper's claims as measured properties of the GPU path: the
time-discretisation bias dominates the precision bias and shrinks as 1/H
(Sec. V, the vanilla-call experiment of Sec. VI.A.1), and the Monte Carlo
error falls as N^-1/2 (Sec. VI.D)."""
import math

import numpy as np
import pytest

from closed_forms import bs_call

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def euler_second_moment(S0, r, sig, T, H):
    """E[S_H^2] of the arithmetic Euler scheme: each step multiplies the
    conditional second moment by (1 + r dt)^2 + sigma^2 dt."""
    dt = T / H
    return S0 ** 2 * ((1 + r * dt) ** 2 + sig ** 2 * dt) ** H


@pytest.mark.parametrize("H", [25, 50, 100])
def test_discretisation_bias_dominates_precision(gb, orc, H):
    """The vanilla market of the paper (S0 100, r 0.05, sigma 0.2, T 1) on
    the observable S_T^2, whose value is known both for the SDE,
    S0^2 e^{(2r + sigma^2) T}, and for the Euler scheme (above).  Euler and
    log-Euler (exact in law) run on the same normals, so the mean of the
    per-path difference estimates the discretisation bias with a small
    standard error: it matches the closed form within 4 SE and is resolved
    at many SE.  The precision bias, the mean FP32 (GPU) minus FP64 (oracle)
    difference on the same paths, is below 2 % of it."""
    S0, sig, r, T, N = 100.0, 0.2, 0.05, 1.0, 1 << 22
    exact = S0 ** 2 * math.exp((2 * r + sig ** 2) * T)
    bias = euler_second_moment(S0, r, sig, T, H) - exact
    model = dict(kind="gbm", s0=[S0], sigma=[sig], r=r)
    sims = {}
    for scheme in ("euler", "log_euler"):
        cfg = dict(steps=H, T=T, paths=N, seed=42, scheme=scheme)
        sims[scheme] = gb.simulate(model, cfg, save_every=H)[-1, 0].double().cpu().numpy()
    D = sims["euler"] ** 2 - sims["log_euler"] ** 2
    m, se = D.mean(), D.std(ddof=1) / math.sqrt(N)
    assert abs(m - bias) <= 4 * se, (H, m, bias, se)
    assert abs(bias) >= 10 * se, (H, bias, se)
    n = 1 << 16
    P = orc.gbm_paths([S0], [sig], r, T, H, n, scheme="euler", save_every=H)[-1, 0]
    prec = np.mean(sims["euler"][:n] ** 2 - P ** 2)
    print(f"H={H}: discretisation bias {bias:.4f} (measured {m:.4f} +- {se:.4f}), "
          f"FP32 - FP64 on {n} paths {prec:.2e}")
    assert abs(prec) <= 0.02 * abs(bias)


def test_discretisation_bias_is_first_order():
    """The Euler bias of S_T^2 times H tends to a constant (weak order 1):
    H * bias at H = 25, 50, 100 within 5 % of its limit
    -S0^2 e^{(2r + sigma^2) T} T^2 ((2r + sigma^2)^2 / 2 - r^2)."""
    S0, sig, r, T = 100.0, 0.2, 0.05, 1.0
    a = 2 * r + sig ** 2
    exact = S0 ** 2 * math.exp(a * T)
    limit = -exact * T ** 2 * (a * a / 2 - r * r)
    for H in (25, 50, 100):
        hb = H * (euler_second_moment(S0, r, sig, T, H) - exact)
        assert abs(hb - limit) <= 0.05 * abs(limit), (H, hb, limit)


def test_error_falls_as_inverse_square_root(gb):
    """Log-Euler GBM call (exact in law): the standard error times sqrt(N)
    is constant over N = 2^12 .. 2^20, within the sampling noise of the SE
    itself, and every price is within 3 SE of Black-Scholes."""
    S0, K, r, sig, T = 100.0, 100.0, 0.05, 0.2, 1.0
    want = bs_call(S0, K, r, sig, T)
    scaled = []
    for e in (12, 14, 16, 18, 20):
        N = 1 << e
        (p, se), = gb.price(dict(kind="gbm", s0=[S0], sigma=[sig], r=r), dict(steps=8, T=T, paths=N, seed=7),
                            [dict(kind="call", strike=K)])
        assert abs(p - want) <= 3 * se, (N, p, want, se)
        scaled.append(se * math.sqrt(N))
    scaled = np.array(scaled)
    print("SE * sqrt(N):", scaled)
    assert scaled.max() / scaled.min() <= 1.08
