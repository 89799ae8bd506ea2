"""Pins of the oracle's GBM pricer (Sec. II.A.1 scalar, II.A.2 multivariate
Euler-Maruyama; Eq. 3 estimator) against closed forms, invariants and the
values the paper prints."""
import json
import os

import numpy as np
import pytest

import closed_forms as cf

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def within(est, se, exact, k=3.0):
    return abs(est - exact) <= k * se


def test_black_scholes_atm_call(orc):
    """1-D GBM ATM call, log-Euler (exact in law at the grid), within 3 SE."""
    f = orc.gbm_payoffs(100.0, 0.2, 0.05, 1.0, 64, 1 << 17, [dict(kind="call", strike=100.0)])
    m, se = orc.mean_se(f[0])
    assert within(m, se, cf.bs_call(100, 100, 0.05, 0.2, 1.0)), (m, se)


def test_paper_vanilla_call_value(orc):
    """The paper's vanilla call (Sec. VI.A.1) against its printed value."""
    g = GOLD["vanilla_call"]
    assert abs(cf.bs_call(g["s0"], g["strike"], g["r"], g["sigma"], g["T"]) - g["price"]) < 1e-10
    f = orc.gbm_payoffs(g["s0"], g["sigma"], g["r"], g["T"], 25, 1 << 18,
                        [dict(kind="call", strike=g["strike"])])
    m, se = orc.mean_se(f[0])
    assert within(m, se, g["price"]), (m, se)


def test_put_call_parity_per_path(orc):
    f = orc.gbm_payoffs(100.0, 0.3, 0.05, 2.0, 16, 4096,
                        [dict(kind="call", strike=95.0), dict(kind="put", strike=95.0)])
    S = orc.gbm_paths(100.0, 0.3, 0.05, 2.0, 16, 4096, save_every=16)[-1, 0]
    disc = np.exp(-0.05 * 2.0)
    assert np.allclose(f[0] - f[1], disc * (S - 95.0), rtol=0, atol=1e-11)


def test_martingale_every_step(orc):
    """e^{-r t_i} E[S(t_i)] = S0 at every step, within 3 SE."""
    M, N, r, T = 8, 1 << 16, 0.05, 1.0
    P = orc.gbm_paths(100.0, 0.4, r, T, M, N, save_every=1)
    for i in range(M + 1):
        x = np.exp(-r * i * T / M) * P[i, 0]
        assert abs(x.mean() - 100.0) <= 3 * x.std(ddof=1) / np.sqrt(N) + 1e-12


def test_saved_paths_start_at_s0(orc):
    """Slot 0 of the materialised paths is t_0: every asset's own S0."""
    s0, sg = np.array([90.0, 100.0, 120.0]), np.array([0.2, 0.3, 0.25])
    corr = np.array([[1.0, 0.3, 0.1], [0.3, 1.0, 0.2], [0.1, 0.2, 1.0]])
    for scheme in ("log_euler", "euler"):
        P = orc.gbm_paths(s0, sg, 0.05, 1.0, 4, 64, corr=corr, scheme=scheme, save_every=2)
        assert np.array_equal(P[0], np.repeat(s0[:, None], 64, axis=1))


def test_euler_scheme_moments(orc):
    """Arithmetic Euler (the formula of Sec. II.A.1 with mu = r S, sigma = s S):
    the factors (1 + r D + s sqrt(D) z) are independent, so
    E[S_M] = S0 (1 + r D)^M and E[S_M^2] = S0^2 ((1 + r D)^2 + s^2 D)^M."""
    M, N, r, s, T = 10, 1 << 17, 0.05, 0.3, 1.0
    D = T / M
    S = orc.gbm_paths(100.0, s, r, T, M, N, scheme="euler", save_every=M)[-1, 0]
    m1 = 100.0 * (1 + r * D) ** M
    m2 = 100.0 ** 2 * ((1 + r * D) ** 2 + s * s * D) ** M
    assert abs(S.mean() - m1) <= 3 * S.std(ddof=1) / np.sqrt(N)
    S2 = S * S
    assert abs(S2.mean() - m2) <= 3 * S2.std(ddof=1) / np.sqrt(N)
    # Euler differs from log-Euler on the same stream by O(D) per path
    L = orc.gbm_paths(100.0, s, r, T, M, N, save_every=M)[-1, 0]
    assert np.median(np.abs(S - L) / L) < 0.05


def test_geometric_asian_closed_form_and_am_gm(orc):
    """Discrete geometric-average call (same paths) within 3 SE of the
    Kemna-Vorst closed form; arithmetic >= geometric payoff on every path."""
    M, N, r, s, T, K = 12, 1 << 16, 0.05, 0.25, 1.0, 100.0
    P = orc.gbm_paths(100.0, s, r, T, M, N, save_every=1)
    G = np.exp(np.mean(np.log(P[1:, 0]), axis=0))
    geo = np.exp(-r * T) * np.maximum(G - K, 0.0)
    m, se = orc.mean_se(geo)
    assert within(m, se, cf.geometric_asian_call(100.0, K, r, s, T, M)), (m, se)
    arith = orc.gbm_payoffs(100.0, s, r, T, M, N, [dict(kind="asian_call", strike=K)])[0]
    assert np.all(arith >= geo - 1e-12)
    # and the arithmetic average is exactly the mean of the monitored prices
    A = np.mean(P[1:, 0], axis=0)
    assert np.allclose(arith, np.exp(-r * T) * np.maximum(A - K, 0.0), rtol=1e-13, atol=1e-12)


def test_one_step_barrier_closed_form(orc):
    """An up-and-out call monitored once (M = 1) against its closed form."""
    S, K, H, r, s, T = 100.0, 95.0, 130.0, 0.05, 0.3, 1.0
    f = orc.gbm_payoffs(S, s, r, T, 1, 1 << 18, [dict(kind="uo_call", strike=K, barrier=H)])
    m, se = orc.mean_se(f[0])
    assert within(m, se, cf.one_step_up_and_out_call(S, K, H, r, s, T)), (m, se)


def test_barrier_in_plus_out_is_vanilla(orc):
    pays = [dict(kind="call", strike=100.0), dict(kind="uo_call", strike=100.0, barrier=120.0),
            dict(kind="ui_call", strike=100.0, barrier=120.0), dict(kind="put", strike=100.0),
            dict(kind="do_put", strike=100.0, barrier=85.0), dict(kind="di_put", strike=100.0, barrier=85.0),
            dict(kind="uo_put", strike=100.0, barrier=120.0), dict(kind="ui_put", strike=100.0, barrier=120.0),
            dict(kind="do_call", strike=100.0, barrier=85.0), dict(kind="di_call", strike=100.0, barrier=85.0)]
    f = orc.gbm_payoffs(100.0, 0.3, 0.05, 1.0, 50, 8192, pays)
    assert np.array_equal(f[1] + f[2], f[0])
    assert np.array_equal(f[4] + f[5], f[3])
    assert np.array_equal(f[6] + f[7], f[3])
    assert np.array_equal(f[8] + f[9], f[0])
    # a barrier knocks out some paths but never adds value
    assert np.all(f[1] <= f[0]) and 0 < np.count_nonzero(f[2]) < 8192
    # monitored maximum >= H exactly where the up-and-in is alive (on paths in the money)
    P = orc.gbm_paths(100.0, 0.3, 0.05, 1.0, 50, 8192, save_every=1)
    hit = P[1:, 0].max(axis=0) >= 120.0
    itm = P[-1, 0] > 100.0
    assert np.array_equal((f[2] > 0), hit & itm)


def test_cholesky_against_lapack(orc):
    import workloads
    _, _, corr = workloads.basket_market(64, 4)
    L = orc.cholesky(corr)
    assert np.allclose(L, np.linalg.cholesky(corr), rtol=0, atol=1e-12)
    assert np.max(np.abs(L @ L.T - corr)) < 1e-13
    assert np.all(np.triu(L, 1) == 0)
    bad = corr.copy()
    bad[0, 1] = bad[1, 0] = 1.5
    with pytest.raises(Exception):
        orc.cholesky(bad)


def test_cholesky_rejects_what_lapack_rejects(orc):
    """An indefinite symmetric matrix with unit diagonal (every entry a valid
    correlation) has no Cholesky factor: LAPACK refuses it, and so must the
    oracle, directly and through the pricer."""
    import pytest
    for c in (0.9, 0.6, 0.51):  # last pivot -15.2, -0.8, -0.06
        A = np.array([[1.0, c, c], [c, 1.0, -c], [c, -c, 1.0]])
        with pytest.raises(np.linalg.LinAlgError):
            np.linalg.cholesky(A)
        with pytest.raises(Exception):
            orc.cholesky(A)
        with pytest.raises(Exception):
            orc.gbm_payoffs(np.full(3, 100.0), np.full(3, 0.2), 0.05, 1.0, 4, 16, [dict(kind="call", strike=100.0)],
                            corr=A)


def test_basket_log_return_covariance(orc):
    """Empirical covariance of one-step log returns equals diag(s) rho diag(s) T
    (a transposed factor, L^T z, would give L^T L instead)."""
    import workloads
    d, N, T = 6, 1 << 17, 1.0
    s0, sig, corr = workloads.basket_market(d, 2, seed=3)
    P = orc.gbm_paths(s0, sig, 0.05, T, 1, N, corr=corr, save_every=1)
    X = np.log(P[1] / P[0])
    C = np.cov(X)
    Sigma = np.diag(sig) @ corr @ np.diag(sig) * T
    # standard error of a sample covariance: sqrt((S_ii S_jj + S_ij^2) / N)
    se = np.sqrt((np.outer(np.diag(Sigma), np.diag(Sigma)) + Sigma ** 2) / N)
    assert np.all(np.abs(C - Sigma) < 5 * se)
    mu = np.log(s0) + (0.05 - 0.5 * sig ** 2) * T
    assert np.all(np.abs(np.log(P[1]).mean(axis=1) - mu) < 5 * np.sqrt(np.diag(Sigma) / N))


def test_geometric_basket_closed_form(orc):
    import workloads
    d, N, r, T, M = 8, 1 << 16, 0.05, 1.0, 4
    s0, sig, corr = workloads.basket_market(d, 3, seed=5)
    w = np.full(d, 1.0 / d)
    K = float(np.exp(np.sum(w * np.log(s0))))
    P = orc.gbm_paths(s0, sig, r, T, M, N, corr=corr, save_every=M)[-1]
    G = np.exp(w @ np.log(P))
    geo = np.exp(-r * T) * np.maximum(G - K, 0)
    m, se = orc.mean_se(geo)
    assert within(m, se, cf.geometric_basket_call(s0, sig, corr, w, K, r, T)), (m, se)
    arith = orc.gbm_payoffs(s0, sig, r, T, M, N, [dict(kind="call", strike=K)], corr=corr, weights=w)[0]
    assert np.all(arith >= geo - 1e-12)


def test_identity_correlation_is_independent_assets(orc):
    """With rho = I (given, or left out), asset a of a d-asset basket uses
    normals a, a+d, a+2d ... of its path's stream: reconstruct its path from
    the raw normals."""
    d, M, N, r, T = 3, 5, 64, 0.05, 1.0
    s0, sig = np.array([90.0, 100.0, 110.0]), np.array([0.1, 0.2, 0.3])
    D = T / M
    for corr in (np.eye(d), None):
        P = orc.gbm_paths(s0, sig, r, T, M, N, corr=corr, save_every=1, path_offset=1000)
        for n in range(N):
            z = orc.normals(42, 1000 + n, 0, M * d).reshape(M, d)
            x = np.log(s0) + np.cumsum((r - 0.5 * sig ** 2) * D + sig * np.sqrt(D) * z, axis=0)
            assert np.allclose(P[1:, :, n], np.exp(x), rtol=1e-13)


def test_path_offset_selects_streams(orc):
    a = orc.gbm_payoffs(100.0, 0.2, 0.05, 1.0, 8, 100, [dict(kind="call", strike=100.0)])
    b = orc.gbm_payoffs(100.0, 0.2, 0.05, 1.0, 8, 40, [dict(kind="call", strike=100.0)], path_offset=60)
    assert np.array_equal(a[0, 60:], b[0])


def test_mean_se_definition(orc):
    """Eq. 3's estimator and its standard error against their textbook
    forms: mean = sum f / N, se = sample standard deviation / sqrt(N)
    (np.std with ddof = 1), on small exact cases and on random vectors,
    including one with a large common offset (the compensated sums keep the
    mean to rounding)."""
    import math
    m, se = orc.mean_se([1.0, 2.0, 3.0, 4.0])
    assert m == 2.5 and abs(se - math.sqrt(5.0 / 3.0) / 2.0) <= 1e-15
    m, se = orc.mean_se([7.0])
    assert m == 7.0 and se == 0.0
    m, se = orc.mean_se([3.0, 5.0])
    assert m == 4.0 and se == 1.0
    m, se = orc.mean_se(np.full(1000, 0.1))
    assert abs(m - 0.1) <= 1e-16 and se <= 1e-9
    rng = np.random.default_rng(9)
    for n, off in ((10, 0.0), (1000, 0.0), (100_000, 0.0), (4096, 1e6)):
        f = off + rng.standard_normal(n) * 3.0
        m, se = orc.mean_se(f)
        want_m = math.fsum(f) / n
        want_se = np.std(f, ddof=1) / math.sqrt(n)
        assert abs(m - want_m) <= 1e-15 * max(1.0, abs(want_m))
        assert abs(se - want_se) <= (1e-9 if off == 0.0 else 1e-3) * want_se, (n, off, se, want_se)
