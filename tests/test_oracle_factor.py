"""Pins of the oracle's factor-model GBM (rho = B B^T + diag(e^2), increments
from k common and d idiosyncratic normals per step):
  * with no factors the stream layout is that of independent assets, so the
    scheme must equal the Cholesky scheme with the identity correlation path
    by path;
  * the loadings of the seeded market reproduce its correlation matrix;
  * the exact-lognormal geometric basket call (closed form with that
    correlation) within 3 SE, and the empirical correlation of one-step log
    returns;
  * one asset with a partial loading is Black-Scholes."""
import numpy as np

import workloads
from closed_forms import bs_call, geometric_basket_call

PAYS = [dict(kind="call", strike=95.0), dict(kind="put", strike=105.0), dict(kind="asian_call", strike=100.0),
        dict(kind="uo_call", strike=95.0, barrier=125.0), dict(kind="di_put", strike=105.0, barrier=85.0)]


def test_no_factors_equals_independent_cholesky_paths(orc):
    d = 5
    s0 = np.linspace(90, 110, d)
    sg = np.linspace(0.15, 0.35, d)
    for scheme in ("log_euler", "euler"):
        f = orc.gbm_factor_payoffs(s0, sg, np.zeros((d, 0)), 0.04, 1.0, 8, 3000, PAYS, scheme=scheme)
        g = orc.gbm_payoffs(s0, sg, 0.04, 1.0, 8, 3000, PAYS, scheme=scheme)
        assert np.max(np.abs(f - g)) <= 1e-12 * np.max(np.abs(g))


def test_market_loadings_reproduce_its_correlation():
    for d, k in [(16, 4), (64, 4), (512, 16)]:
        _, _, corr = workloads.basket_market(d, k)
        _, _, B = workloads.basket_market_factors(d, k)
        e2 = 1.0 - (B * B).sum(axis=1)
        assert np.all(e2 > 0)
        assert np.max(np.abs(B @ B.T + np.diag(e2) - corr)) < 1e-12


def test_geometric_basket_and_return_correlation(orc):
    d, k, T, r = 12, 3, 1.0, 0.05
    s0, sg, B = workloads.basket_market_factors(d, k, seed=9)
    corr = B @ B.T + np.diag(1.0 - (B * B).sum(axis=1))
    w = np.full(d, 1.0 / d)
    _, ST = orc.gbm_factor_payoffs(s0, sg, B, r, T, 1, 1 << 16, [dict(kind="call", strike=0.0)], weights=w,
                                   terminal=True)
    G = np.exp(w @ np.log(ST))
    K = float(np.exp(w @ np.log(s0)))
    f = np.exp(-r * T) * np.maximum(G - K, 0.0)
    want = geometric_basket_call(s0, sg, corr, w, K, r, T)
    assert abs(f.mean() - want) <= 3 * f.std(ddof=1) / np.sqrt(f.size)
    R = np.log(ST / s0[:, None])
    emp = np.corrcoef(R)
    assert np.max(np.abs(emp - corr)) < 5.0 / np.sqrt(R.shape[1])


def test_one_asset_partial_loading_is_black_scholes(orc):
    f = orc.gbm_factor_payoffs(100.0, 0.3, np.array([[0.6]]), 0.05, 1.0, 4, 1 << 17, [dict(kind="call", strike=100.0)])[0]
    assert abs(f.mean() - bs_call(100.0, 100.0, 0.05, 0.3, 1.0)) <= 3 * f.std(ddof=1) / np.sqrt(f.size)
