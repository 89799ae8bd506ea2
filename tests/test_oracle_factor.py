"""Pins of the oracle's factor-model GBM (rho = B B^T + diag(e^2), increments
from k common and d idiosyncratic normals per step):
  * with no factors the stream layout is that of independent assets, so the
    scheme must equal the Cholesky scheme with the identity correlation path
    by path;
  * the loadings of the seeded market reproduce its correlation matrix;
  * the exact-lognormal geometric basket call (closed form with that
    correlation) within 3 SE, and the empirical correlation of one-step log
    returns;
  * one asset with a partial loading is Black-Scholes;
  * the pathwise Greeks of a basket call / put: common-random-number central
    differences in S0_a, sigma_a and r, and the one-asset Black-Scholes
    delta, vega and rho within 3 SE."""
import numpy as np

import workloads
import pytest

from closed_forms import bs_call, bs_call_greeks, geometric_basket_call

PAYS = [dict(kind="call", strike=95.0), dict(kind="put", strike=105.0), dict(kind="asian_call", strike=100.0),
        dict(kind="uo_call", strike=95.0, barrier=125.0), dict(kind="di_put", strike=105.0, barrier=85.0)]


def test_no_factors_equals_independent_cholesky_paths(orc):
    d = 5
    s0 = np.linspace(90, 110, d)
    sg = np.linspace(0.15, 0.35, d)
    for scheme in ("log_euler", "euler"):
        f, ST = orc.gbm_factor_payoffs(s0, sg, np.zeros((d, 0)), 0.04, 1.0, 8, 3000, PAYS, scheme=scheme,
                                       terminal=True)
        g = orc.gbm_payoffs(s0, sg, 0.04, 1.0, 8, 3000, PAYS, scheme=scheme)
        assert np.max(np.abs(f - g)) <= 1e-12 * np.max(np.abs(g))
        # the terminal prices it reports are the prices, under either scheme
        P = orc.gbm_paths(s0, sg, 0.04, 1.0, 8, 3000, scheme=scheme, save_every=8)[-1]
        assert np.allclose(ST, P, rtol=1e-12)


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


@pytest.mark.parametrize("kind,T", [("call", 1.0), ("put", 1.0), ("call", 0.6)])
def test_factor_greeks_against_crn_differences(orc, kind, T):
    """Pathwise d/dS0_a, d/dsigma_a, d/dr against central differences of the
    per-path payoffs simulated with the bumped parameter on the same stream
    (the loadings held fixed): per path they differ only where the basket
    crosses the strike within the bump, so the mean difference lies within
    3 SE of the per-path difference, and far below the Greek itself."""
    d, k, M, N = 6, 2, 8, 1 << 13
    s0, sg, B = workloads.basket_market_factors(d, k, seed=5)
    w = np.linspace(1.0, 2.0, d)
    w /= w.sum()
    r = 0.04
    K = float(w @ s0) * (1.0 if kind == "call" else 1.02)
    pay = dict(kind=kind, strike=K)
    g = orc.gbm_factor_greeks(s0, sg, B, r, T, M, N, pay, weights=w)
    assert np.all(np.isfinite(g))
    checks = []
    for a in (0, 3, d - 1):
        e = np.zeros(d)
        e[a] = 1.0
        h = 1e-4 * s0[a]
        up = orc.gbm_factor_payoffs(s0 + h * e, sg, B, r, T, M, N, [pay], weights=w)[0]
        dn = orc.gbm_factor_payoffs(s0 - h * e, sg, B, r, T, M, N, [pay], weights=w)[0]
        checks.append((f"delta{a}", (up - dn) / (2 * h), g[a]))
        h = 1e-5
        up = orc.gbm_factor_payoffs(s0, sg + h * e, B, r, T, M, N, [pay], weights=w)[0]
        dn = orc.gbm_factor_payoffs(s0, sg - h * e, B, r, T, M, N, [pay], weights=w)[0]
        checks.append((f"vega{a}", (up - dn) / (2 * h), g[d + a]))
    h = 1e-6
    up = orc.gbm_factor_payoffs(s0, sg, B, r + h, T, M, N, [pay], weights=w)[0]
    dn = orc.gbm_factor_payoffs(s0, sg, B, r - h, T, M, N, [pay], weights=w)[0]
    checks.append(("rho", (up - dn) / (2 * h), g[2 * d]))
    for name, f_d, pw in checks:
        diff = f_d - pw
        m, se = orc.mean_se(diff)
        assert abs(m) <= 3 * se + 1e-9, (kind, name, m, se)
        assert abs(np.mean(pw)) > 10 * abs(m), (kind, name, np.mean(pw), m)


def test_factor_greeks_one_asset_black_scholes(orc):
    """One asset with a partial loading is Black-Scholes: the pathwise delta,
    vega and rho within 3 SE of the closed-form Greeks."""
    S, K, r, sg, T = 100.0, 95.0, 0.05, 0.3, 1.0
    g = orc.gbm_factor_greeks(S, sg, np.array([[0.6]]), r, T, 4, 1 << 17, dict(kind="call", strike=K))
    for row, want in zip(g, bs_call_greeks(S, K, r, sg, T)):
        m, se = orc.mean_se(row)
        assert abs(m - want) <= 3 * se, (m, se, want)
