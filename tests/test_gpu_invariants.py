"""Invariants of the GPU path that need no oracle: the discounted price is a
martingale at every step (log-Euler GBM and the full-truncation Heston
scheme are exact martingales in law: each log step has conditional mean
exp(r dt)), and put-call parity holds path by path on the headline BF16
basket launch (Sec. I.A.2, Eq. 3)."""
import math

import numpy as np
import pytest

import workloads
from gpu_util import cfg_of, gbm_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


@pytest.mark.parametrize("kind", ["gbm1d", "basket64", "heston"])
def test_discounted_price_is_a_martingale(gb, kind):
    """e^{-r t_i} E[S_a(t_i)] = S0_a for every asset a and every saved step
    t_i, within 4.5 standard errors (up to 64 x 8 comparisons)."""
    T = 1.0
    if kind == "heston":
        m = dict(workloads.HESTON_PARAMS)
        model, s0, r, steps, N = dict(kind="heston", **m), np.array([m["s0"]]), m["r"], 64, 1 << 20
    elif kind == "gbm1d":
        w = workloads.gbm_1d(paths=1, steps=64)
        model, s0, r, steps, N = gbm_model(w), np.asarray(w["s0"], float).ravel(), w["r"], 64, 1 << 20
    else:
        w = workloads.basket_d64(paths=1)
        model, s0, r, steps, N = gbm_model(w), np.asarray(w["s0"], float), w["r"], 64, 1 << 16
    S = gb.simulate(model, dict(steps=steps, T=T, paths=N, seed=11), save_every=steps // 8)
    S = S[:, :len(s0)].double().cpu().numpy()                      # [9, d, N]
    t = np.arange(S.shape[0]) * T / 8
    disc = np.exp(-r * t)[:, None]
    mean = S.mean(axis=2) * disc
    se = S.std(axis=2, ddof=1) / math.sqrt(N) * disc
    z = np.abs(mean[1:] - s0[None, :]) / se[1:]
    print(f"{kind}: max |discounted mean - S0| / SE over {z.size} (step, asset) pairs: {z.max():.2f}")
    assert np.allclose(mean[0], s0, rtol=1e-6)
    assert z.max() <= 4.5


def test_put_call_parity_on_the_headline_launch(gb):
    """The d = 64 basket, 2^18 paths x 252 steps, BF16 contraction (the
    benchmark's launch): on the same paths call(K) - put(K) =
    e^{-rT} (E[U_T] - K), with e^{-rT} E[U_T] the zero-strike call, to the
    FP32 rounding of the payoffs; and the zero-strike call is the basket's
    initial value within 3 SE (the martingale)."""
    w = workloads.basket_d64()
    u0 = float(np.asarray(w["weights"]) @ np.asarray(w["s0"]))
    K = u0
    # the benchmark's payoffs first (the up-and-out call keeps the monitored
    # kernel variant), then the put and the zero-strike call
    pays = list(w["payoffs"]) + [dict(kind="put", strike=K), dict(kind="call", strike=0.0)]
    assert pays[0] == dict(kind="call", strike=K)
    (c, _), _, (p, _), (f, sf) = gb.price(gbm_model(w), cfg_of(w, precision="bf16"), pays)
    disc = math.exp(-w["r"] * w["T"])
    print(f"C - P = {c - p:.6f}, forward - disc K = {f - disc * K:.6f}; forward {f:.4f} vs U0 {u0:.4f} (SE {sf:.4f})")
    assert abs((c - p) - (f - disc * K)) <= 2e-6 * u0
    assert abs(f - u0) <= 3 * sf
