"""Pins of the oracle's forward-mode correlation sensitivities (Sec. I.A.3:
sensitivities to model parameters; Sec. VI.A.2 differentiates the basket
simulation): the Cholesky tangent against LAPACK finite differences and its
defining identity, per-path terminal tangents against bumped simulations on
the same stream, the geometric-basket closed form within 3 SE, and common-
random-number central differences of the arithmetic-basket price; the
Asian (time-averaged) basket against the same differences and, with one
step, against the terminal basket."""
import numpy as np
import pytest

import closed_forms as cf

S0 = np.array([90.0, 100.0, 110.0, 105.0])
SIG = np.array([0.2, 0.3, 0.25, 0.35])
CORR = np.array([[1.0, 0.5, 0.2, -0.1],
                 [0.5, 1.0, 0.3, 0.15],
                 [0.2, 0.3, 1.0, 0.4],
                 [-0.1, 0.15, 0.4, 1.0]])
R, T = 0.05, 1.0


def _unit(d, a, b):
    E = np.zeros((d, d))
    E[a, b] = E[b, a] = 1.0
    return E


def test_cholesky_tangent_against_lapack(orc):
    """L Phi(L^-1 E L^-T) against central differences of numpy's (LAPACK's)
    Cholesky, for unit pair directions and a random symmetric one; and the
    identity dL L^T + L dL^T = E with dL lower triangular."""
    rng = np.random.default_rng(3)
    d = CORR.shape[0]
    L = np.linalg.cholesky(CORR)
    Es = [_unit(d, 2, 0), _unit(d, 3, 1), _unit(d, 1, 0)]
    Q = rng.standard_normal((d, d))
    Es.append(Q + Q.T)
    h = 1e-6
    for E in Es:
        t = orc.cholesky_tangent(L, E)
        fd = (np.linalg.cholesky(CORR + h * E) - np.linalg.cholesky(CORR - h * E)) / (2 * h)
        assert np.max(np.abs(t - fd)) < 1e-8, np.max(np.abs(t - fd))
        assert np.allclose(t @ L.T + L @ t.T, E, atol=1e-12)
        assert np.all(np.triu(t, 1) == 0.0)


def test_terminal_tangents_against_bumped_paths(orc):
    """d x_c(T) / d corr[a][b] assembled from the per-step factor tangents and
    the Cholesky tangent, against central differences of the terminal log-
    prices simulated with corr +- h E_ab on the same stream (smooth in corr:
    agreement to O(h^2) and FP64 cancellation)."""
    d, M, N = 4, 12, 64
    xT, tL = orc.gbm_corr_tangents(S0, SIG, CORR, R, T, M, N)
    L = orc.cholesky(CORR)
    h = 1e-6
    for a, b in [(1, 0), (3, 2), (3, 0)]:
        E = _unit(d, a, b)
        J = orc.cholesky_tangent(L, E)
        up, _ = orc.gbm_corr_tangents(S0, SIG, CORR + h * E, R, T, M, N)
        dn, _ = orc.gbm_corr_tangents(S0, SIG, CORR - h * E, R, T, M, N)
        fd = (up - dn) / (2 * h)
        for c in range(d):
            tang = sum(tL[c * (c + 1) // 2 + e] * J[c, e] for e in range(c + 1))
            assert np.max(np.abs(tang - fd[c])) < 1e-7, (a, b, c, np.max(np.abs(tang - fd[c])))
    # the terminal log-prices themselves are the ones of the plain simulation
    ST = orc.gbm_paths(S0, SIG, R, T, M, N, corr=CORR, save_every=M)[-1]
    assert np.allclose(np.exp(xT), ST, rtol=1e-13)


def test_geometric_basket_corr_sensitivity_closed_form(orc):
    """Pathwise d/d corr[a][b] of a call on prod S_a^{w_a} (its log is exactly
    normal under log-Euler) within 3 SE of the derivative of the closed form,
    taken by a central difference of the closed form itself."""
    d, M, N = 4, 4, 1 << 18
    w = np.array([0.1, 0.4, 0.3, 0.2])
    K = 100.0
    xT, tL = orc.gbm_corr_tangents(S0, SIG, CORR, R, T, M, N)
    G = np.exp(w @ xT)
    g = np.exp(-R * T) * (G > K)[None, :] * w[:, None] * G[None, :]
    dl = np.zeros((d, d, N))
    for a in range(d):
        for b in range(a + 1):
            dl[a, b] = g[a] * tL[a * (a + 1) // 2 + b]
    drho = orc.corr_chain(CORR, dl)
    h = 1e-5
    for a, b in [(1, 0), (2, 1), (3, 0), (3, 2)]:
        E = _unit(d, a, b)
        want = (cf.geometric_basket_call(S0, SIG, CORR + h * E, w, K, R, T)
                - cf.geometric_basket_call(S0, SIG, CORR - h * E, w, K, R, T)) / (2 * h)
        m, se = orc.mean_se(drho[a, b])
        assert abs(m - want) <= 3 * se, (a, b, m, se, want)
        assert se < 0.05 * abs(want)


@pytest.mark.parametrize("kind", ["call", "put"])
def test_arithmetic_basket_against_crn_differences(orc, kind):
    """Pathwise d/d corr[a][b] of an arithmetic basket call / put against
    central differences of the per-path payoffs on the same stream
    (corr +- h E_ab): per path they differ only where the basket crosses the
    strike within the bump, so the mean difference lies within 3 SE of the
    per-path difference."""
    d, M, N = 4, 8, 1 << 13
    pay = dict(kind=kind, strike=100.0)
    res = orc.gbm_corr_greeks(S0, SIG, CORR, R, T, M, N, pay)
    assert np.allclose(res["drho"], np.transpose(res["drho"], (1, 0, 2)))
    assert np.all(res["drho"][np.arange(d), np.arange(d)] == 0.0)
    h = 1e-6
    for a, b in [(1, 0), (2, 0), (3, 1), (3, 2)]:
        E = _unit(d, a, b)
        up = orc.gbm_payoffs(S0, SIG, R, T, M, N, [pay], corr=CORR + h * E)[0]
        dn = orc.gbm_payoffs(S0, SIG, R, T, M, N, [pay], corr=CORR - h * E)[0]
        diff = (up - dn) / (2 * h) - res["drho"][a, b]
        m, se = orc.mean_se(diff)
        assert abs(m) <= 3 * se + 1e-9, (a, b, m, se)
        assert abs(np.mean(res["drho"][a, b])) > 10 * abs(m)
    base = orc.gbm_payoffs(S0, SIG, R, T, M, N, [pay], corr=CORR)[0]
    assert np.allclose(res["f"], base, rtol=1e-13)


def test_factor_tangents_tie_to_delta_and_vega(orc):
    """Per path, sum_b Lrho[a][b] d/dLrho[a][b] is the diffusion part of the
    sigma_a tangent: sigma_a vega_a + sigma_a^2 T S0_a delta_a, with delta and
    vega from the oracle's separate forward-mode Greeks of the same paths."""
    d, M, N = 4, 10, 2000
    w = np.array([0.1, 0.4, 0.3, 0.2])
    pay = dict(kind="call", strike=100.0)
    res = orc.gbm_corr_greeks(S0, SIG, CORR, R, T, M, N, pay, weights=w)
    g = orc.gbm_greeks(S0, SIG, R, T, M, N, [pay], corr=CORR, weights=w)[0]
    L = np.linalg.cholesky(CORR)
    lhs = np.einsum("ab,abn->an", L, res["dl"])
    rhs = SIG[:, None] * g[d:2 * d] + (SIG ** 2 * T * S0)[:, None] * g[:d]
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.abs(rhs).max()


@pytest.mark.parametrize("kind", ["asian_call", "asian_put"])
def test_asian_basket_against_crn_differences(orc, kind):
    """Pathwise d/d corr[a][b] of a call / put on the basket's average over
    the steps against central differences of the per-path payoffs on the same
    stream (corr +- h E_ab): within 3 SE of the per-path difference, and far
    below the sensitivity itself."""
    d, M, N = 4, 8, 1 << 13
    pay = dict(kind=kind, strike=100.0 if kind == "asian_call" else 103.0)
    res = orc.gbm_corr_greeks(S0, SIG, CORR, R, T, M, N, pay)
    assert np.allclose(res["drho"], np.transpose(res["drho"], (1, 0, 2)))
    h = 1e-6
    for a, b in [(1, 0), (2, 0), (3, 1), (3, 2)]:
        E = _unit(d, a, b)
        up = orc.gbm_payoffs(S0, SIG, R, T, M, N, [pay], corr=CORR + h * E)[0]
        dn = orc.gbm_payoffs(S0, SIG, R, T, M, N, [pay], corr=CORR - h * E)[0]
        diff = (up - dn) / (2 * h) - res["drho"][a, b]
        m, se = orc.mean_se(diff)
        assert abs(m) <= 3 * se + 1e-9, (a, b, m, se)
        assert abs(np.mean(res["drho"][a, b])) > 10 * abs(m)
    base = orc.gbm_payoffs(S0, SIG, R, T, M, N, [pay], corr=CORR)[0]
    assert np.allclose(res["f"], base, rtol=1e-13)


def test_asian_with_one_step_is_the_terminal_basket(orc):
    """With one step the average is the terminal basket: the Asian call's
    sensitivities equal the European call's path by path."""
    pay_a, pay_e = dict(kind="asian_call", strike=100.0), dict(kind="call", strike=100.0)
    ra = orc.gbm_corr_greeks(S0, SIG, CORR, R, T, 1, 2000, pay_a)
    re = orc.gbm_corr_greeks(S0, SIG, CORR, R, T, 1, 2000, pay_e)
    scale = np.max(np.abs(re["dl"]))
    assert np.max(np.abs(ra["dl"] - re["dl"])) <= 1e-12 * scale
    assert np.max(np.abs(ra["f"] - re["f"])) <= 1e-12 * np.max(re["f"])
