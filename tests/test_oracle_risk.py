"""Pins of the risk oracle (oracle/risk.py and the risk functions of
oracle.c): VaR / CVaR against their definitions and the normal closed forms,
scenario moments, nested values and labels against Black-Scholes."""
import math

import numpy as np
import pytest

import closed_forms as cf
import workloads
from oracle import risk


def test_var_cvar_definition_brute_force():
    rng = np.random.default_rng(0)
    for n in (1, 2, 10, 101, 1000):
        pnl = rng.standard_normal(n)
        for alpha in (0.5, 0.9, 0.99):
            var, cvar, nt = risk.var_cvar(pnl, alpha)
            losses = sorted(-pnl, reverse=True)
            k = max(1, math.ceil((1 - alpha) * n - 1e-9))
            assert var == losses[k - 1]
            above = [l for l in losses if l > var]
            assert nt == len(above)
            assert cvar == (np.mean(above) if above else var)
            assert cvar >= var


def test_var_is_the_upper_quantile_of_the_sample():
    """VaR_alpha read as the upper alpha-quantile of the empirical loss law,
    inf{x : F_n(x) > alpha} (F_n(x) = #(losses <= x) / n, exact rational
    comparison), found by scanning the candidate losses; CVaR_alpha as the
    conditional mean of the losses above it, E_n[L | L > VaR] (VaR itself
    when no loss is above).  Ties included."""
    from fractions import Fraction
    rng = np.random.default_rng(4)
    for n in (1, 2, 3, 10, 99, 100, 101, 1000, 1001):
        for alpha in (0.5, 0.9, 0.95, 0.99, 0.999):
            for ties in (False, True):
                pnl = rng.standard_normal(n)
                if ties:
                    pnl = np.round(pnl, 1)
                losses = -pnl
                a = Fraction(str(alpha))
                cand = sorted(set(losses.tolist()))
                want = next(x for x in cand if Fraction(int(np.sum(losses <= x)), n) > a) \
                    if any(Fraction(int(np.sum(losses <= x)), n) > a for x in cand) else max(cand)
                above = losses[losses > want]
                var, cvar, nt = risk.var_cvar(pnl, alpha)
                assert var == want, (n, alpha, ties, var, want)
                assert nt == above.size
                assert cvar == pytest.approx(above.mean() if above.size else want, rel=1e-12, abs=1e-12)


def test_var_cvar_normal_closed_form():
    rng = np.random.default_rng(1)
    n, alpha = 1 << 20, 0.99
    pnl = 2.0 + 3.0 * rng.standard_normal(n)
    var, cvar, _ = risk.var_cvar(pnl, alpha)
    from scipy.stats import norm
    z = norm.ppf(alpha)
    assert abs(var - (-2.0 + 3.0 * z)) < 0.03
    assert abs(cvar - (-2.0 + 3.0 * norm.pdf(z) / (1 - alpha))) < 0.03


def test_scenario_moments(orc):
    s0, sg, corr = workloads.basket_market(6, 2, seed=5)
    h, mu, n = 1 / 252, 0.05, 1 << 17
    S = risk.scenarios(s0, sg, corr, mu, h, n)
    X = np.log(S / s0)
    Sigma = np.diag(sg) @ corr @ np.diag(sg) * h
    se = np.sqrt((np.outer(np.diag(Sigma), np.diag(Sigma)) + Sigma ** 2) / n)
    assert np.all(np.abs(np.cov(X.T) - Sigma) < 5 * se)
    assert np.all(np.abs(X.mean(axis=0) - (mu - 0.5 * sg ** 2) * h) < 5 * np.sqrt(np.diag(Sigma) / n))


def test_nested_value_is_black_scholes(orc):
    # European call and put from the same state within 3 SE of Black-Scholes
    V = risk.option_values([100.0], [0.25], 0.05, 1 / 252, 1, 0, [0, 0], [0, 1], [105.0, 95.0], [np.inf, np.inf],
                           [251, 251], 1 << 16)
    tau = 251 / 252
    for v, want in zip(V, [cf.bs_call(100, 105, 0.05, 0.25, tau), cf.bs_put(100, 95, 0.05, 0.25, tau)]):
        assert abs(v - want) < 3 * 0.06  # SE of the 2^16-path estimate is below 0.06 here
    # up-and-out <= vanilla, and 0 at or above the barrier
    U = risk.option_values([100.0], [0.25], 0.05, 1 / 252, 1, 0, [0, 0], [4, 4], [100.0, 100.0], [130.0, 99.0],
                           [60, 60], 4096)
    van = risk.option_values([100.0], [0.25], 0.05, 1 / 252, 1, 0, [0], [0], [100.0], [np.inf], [60], 4096)
    assert 0 < U[0] < van[0] and U[1] == 0.0
    # at or above the barrier on the revaluation date the option is already
    # knocked out, even where later prices would fall back and finish in
    # the money (a low strike)
    Z = risk.option_values([100.0], [0.25], 0.05, 1 / 252, 1, 0, [0, 0], [4, 0], [50.0, 50.0], [100.0, np.inf],
                           [60, 60], 4096)
    assert Z[0] == 0.0 and Z[1] > 40.0


def test_base_values_run_the_full_maturity(orc):
    """Base-date values (scen < 0) price from s0 over the horizon plus the
    remaining steps: Black-Scholes at (rem + hsteps) dt within 3 SE."""
    rem, hsteps, inner = 230, 20, 1 << 16
    V = risk.option_values([100.0], [0.25], 0.05, 1 / 252, hsteps, -1, [0, 0], [0, 1], [105.0, 95.0],
                           [np.inf, np.inf], [rem, rem], inner)
    tau = (rem + hsteps) / 252
    for v, want in zip(V, [cf.bs_call(100, 105, 0.05, 0.25, tau), cf.bs_put(100, 95, 0.05, 0.25, tau)]):
        assert abs(v - want) < 3 * 0.06, (v, want)  # SE of the 2^16-path estimate is below 0.06 here


def test_nested_up_and_out_monitors_every_step(orc):
    """The nested revaluation's up-and-out call is knocked out when any of
    its monitored prices reaches the barrier: its value equals the discretely
    monitored up-and-out call of the GBM pricer (the same estimand, pinned by
    the path-maximum test, on other streams) within 3 combined SE, while the
    call knocked out on the terminal price alone lies far above both."""
    S, sg, r, dt, steps, K, H = 100.0, 0.25, 0.05, 1 / 252, 60, 100.0, 112.0
    inner, T = 1 << 16, steps / 252
    V = risk.option_values([S], [sg], r, dt, 0, 0, [0], [4], [K], [H], [steps], inner)[0]
    f = orc.gbm_payoffs(S, sg, r, T, steps, 1 << 17, [dict(kind="uo_call", strike=K, barrier=H)])[0]
    m, se = orc.mean_se(f)
    se_v = f.std(ddof=1) / math.sqrt(inner)  # the nested estimate's payoff law is the same
    assert abs(V - m) <= 3 * math.hypot(se, se_v), (V, m, se, se_v)
    # knocked out only at maturity: C(K) - C(H) - (H - K) * digital(H)
    d2 = (math.log(S / H) + (r - 0.5 * sg * sg) * T) / (sg * math.sqrt(T))
    terminal_only = cf.bs_call(S, K, r, sg, T) - cf.bs_call(S, H, r, sg, T) - (H - K) * math.exp(-r * T) * cf.ncdf(d2)
    assert terminal_only - V > 20 * math.hypot(se, se_v), (terminal_only, V)


def test_labels_european_are_black_scholes(orc):
    pts = np.array([[1.0, 0.2, 1.0, 0.05, 0.0], [1.2, 0.3, 0.5, 0.02, 0.0], [0.8, 0.15, 2.0, 0.07, 0.0]])
    lab = risk.labels(pts, 1 << 15)
    for p, l in zip(pts, lab):
        want = cf.bs_call(p[0], 1.0, p[3], p[1], p[2])
        assert abs(l - want) < 4 * p[0] * p[1] * math.sqrt(p[2]) / math.sqrt(1 << 15) + 1e-4
    b = risk.labels(np.array([[1.0, 0.2, 1.0, 0.05, 0.8], [1.3, 0.2, 1.0, 0.05, 0.8]]), 4096)
    assert 0 < b[0] < lab[0] and b[1] == 0.0


def test_european_portfolio_nested_matches_exact_revaluation(orc):
    """European-only portfolio: nested Monte Carlo PnL (oracle, 2^12 inner
    paths) against the exact Black-Scholes revaluation on the same scenarios:
    agreement within the inner-noise standard error."""
    pf = workloads.risk_portfolio(n_under=4, per_under=8, barriers=False)
    S = risk.scenarios(pf["s0"], pf["sigma"], pf["corr"], pf["mu"], pf["horizon"], 8)
    steps = np.rint(pf["maturity"] * 252).astype(int)
    rem = steps - 1
    kind = pf["kind"]
    def exact(state, taus):
        return np.array([(cf.bs_call if k == 0 else cf.bs_put)(state[u], K, pf["r"], pf["sigma"][u], t)
                         for u, k, K, t in zip(pf["under"], kind, pf["strike"], taus)])
    base_x = exact(pf["s0"], steps / 252)
    for s in range(8):
        V = risk.option_values(S[s], pf["sigma"], pf["r"], 1 / 252, 1, s, pf["under"], kind, pf["strike"],
                               pf["barrier"], rem, 1 << 12)
        Vx = exact(S[s], rem / 252)
        # inner SE of each value <= 0.6 here; positions +-1, 32 options
        assert abs(pf["position"] @ (V - Vx)) < 3 * 0.6 * math.sqrt(32)


def test_label_greeks_pins():
    """The oracle's pathwise label Greeks (orc_surrogate_label_greeks): the
    price column is the label oracle's own value on the same paths; delta
    (d/d S/K) and vega (d/d sigma) of the European points match the
    Black-Scholes closed forms within 4 standard errors (log-Euler is exact in
    law) and the central common-random-number differences of the oracle's own
    labels; barrier points carry NaN."""
    pts = np.array([[1.0, 0.2, 1.0, 0.05, 0.0], [0.8, 0.35, 0.5, 0.02, 0.0], [1.3, 0.15, 63 / 252, 0.07, 0.0],
                    [1.1, 0.25, 2.0, 0.0, 0.0], [1.0, 0.3, 1.0, 0.04, 0.8]])
    paths = 1 << 14
    out = risk.label_greeks(pts, paths)
    lab = risk.labels(pts, paths)
    assert np.all(np.isnan(out[4])) and np.all(np.isfinite(out[:4]))
    for p in range(4):
        sk, sig, tau, r, _ = pts[p]
        assert abs(out[p, 0] - lab[p]) <= 1e-12 * abs(lab[p])
        M = max(1, round(tau * 252))
        T = M * (tau / M)
        d1 = (math.log(sk) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
        delta, vega = cf.ncdf(d1), sk * cf.npdf(d1) * math.sqrt(T)
        assert abs(out[p, 2] - delta) <= 4 * out[p, 3], (p, out[p, 2], delta, out[p, 3])
        assert abs(out[p, 4] - vega) <= 4 * out[p, 5], (p, out[p, 4], vega, out[p, 5])
        # central differences of the same-stream label (h relative 1e-5)
        for col, k in ((2, 0), (4, 1)):
            h = 1e-5 * pts[p, k]
            up, dn = pts.copy(), pts.copy()  # point p keeps its own stream (tag 4, p << 16 | path)
            up[p, k] += h
            dn[p, k] -= h
            fd = (risk.labels(up, paths)[p] - risk.labels(dn, paths)[p]) / (2 * h)
            assert abs(fd - out[p, col]) <= 2e-4 * abs(out[p, col]) + 1e-6, (p, col, fd, out[p, col])
