"""Pins of the oracle's forward-mode pathwise Greeks (Sec. I.A.3; the paper's
basket delta of Sec. VI.A.2): Black-Scholes closed forms within 3 SE, and
common-random-number central finite differences on the same stream."""
import numpy as np
import pytest

import closed_forms as cf

BASE = dict(s0=100.0, v0=0.04, r=0.05, kappa=2.0, theta=0.04, xi=0.5, rho=-0.7)


def test_gbm_greeks_vs_black_scholes(orc):
    N = 1 << 17
    g = orc.gbm_greeks(100.0, 0.2, 0.05, 1.0, 16, N, [dict(kind="call", strike=105.0)])[0]
    want = cf.bs_call_greeks(100.0, 105.0, 0.05, 0.2, 1.0)
    for k in range(3):
        m, se = orc.mean_se(g[k])
        assert abs(m - want[k]) <= 3 * se, (k, m, se, want[k])


def _fd(price_fn, theta, h=1e-6):
    """Central CRN difference on the same stream.  On a fixed path set it tends
    to the pathwise derivative as h -> 0 (kinks are crossed by O(h) paths);
    h = 1e-6 keeps FP64 cancellation near 1e-10."""
    return (price_fn(theta * (1 + h)) - price_fn(theta * (1 - h))) / (2 * h * theta)


@pytest.mark.parametrize("scheme", ["log_euler", "euler"])
@pytest.mark.parametrize("kind", ["call", "put", "asian_call"])
def test_gbm_pathwise_equals_crn_finite_difference(orc, scheme, kind):
    N, M = 1 << 13, 12
    pay = [dict(kind=kind, strike=100.0)]
    base = dict(s0=100.0, sigma=0.25, r=0.05)

    def price(**kw):
        p = dict(base, **kw)
        return orc.gbm_payoffs(p["s0"], p["sigma"], p["r"], 1.0, M, N, pay, scheme=scheme)[0].mean()

    g = orc.gbm_greeks(base["s0"], base["sigma"], base["r"], 1.0, M, N, pay, scheme=scheme)[0].mean(axis=1)
    fd = [_fd(lambda t: price(s0=t), 100.0), _fd(lambda t: price(sigma=t), 0.25), _fd(lambda t: price(r=t), 0.05)]
    for k in range(3):
        assert abs(g[k] - fd[k]) <= 2e-4 * max(1.0, abs(fd[k])), (k, g[k], fd[k])


def test_basket_delta_and_vega_vs_crn_fd(orc):
    import workloads
    d, N, M = 5, 1 << 12, 6
    s0, sig, corr = workloads.basket_market(d, 2, seed=11)
    K = float(np.mean(s0))
    pay = [dict(kind="call", strike=K)]
    g = orc.gbm_greeks(s0, sig, 0.05, 1.0, M, N, pay, corr=corr)[0].mean(axis=1)
    for a in [0, 3]:
        def p_s0(t, a=a):
            s = s0.copy(); s[a] = t
            return orc.gbm_payoffs(s, sig, 0.05, 1.0, M, N, pay, corr=corr)[0].mean()

        def p_sig(t, a=a):
            s = sig.copy(); s[a] = t
            return orc.gbm_payoffs(s0, s, 0.05, 1.0, M, N, pay, corr=corr)[0].mean()
        assert abs(g[a] - _fd(p_s0, s0[a])) <= 2e-4 * max(1, abs(g[a]))
        assert abs(g[d + a] - _fd(p_sig, sig[a])) <= 2e-4 * max(1, abs(g[d + a]))
    # d/dr
    fr = _fd(lambda t: orc.gbm_payoffs(s0, sig, t, 1.0, M, N, pay, corr=corr)[0].mean(), 0.05)
    assert abs(g[2 * d] - fr) <= 2e-4 * max(1, abs(fr))


def test_greeks_reject_barriers(orc):
    with pytest.raises(Exception):
        orc.gbm_greeks(100.0, 0.2, 0.05, 1.0, 4, 16, [dict(kind="uo_call", strike=100.0, barrier=120.0)])


@pytest.mark.parametrize("T", [1.0, 0.75])
@pytest.mark.parametrize("kind", ["call", "asian_call"])
def test_heston_pathwise_equals_crn_finite_difference(orc, kind, T):
    """Feller condition met (2 kappa theta = 0.16 > xi^2 = 0.04): the path map
    is smooth on the sample and every Greek matches the CRN difference (at a
    maturity other than 1 as well, where d/dr's -T P term shows its T)."""
    N, M = 1 << 12, 32
    base = dict(BASE, xi=0.2)
    pay = [dict(kind=kind, strike=100.0)]
    g = orc.heston_greeks(base, T, M, N, pay)[0].mean(axis=1)
    for k, name in enumerate(orc.HESTON_PARAM_ORDER):
        def price(t, name=name):
            return orc.heston_payoffs(dict(base, **{name: t}), T, M, N, pay)[0].mean()
        fd = _fd(price, base[name])
        assert abs(g[k] - fd) <= 1e-5 * max(1.0, abs(fd)), (name, g[k], fd)


@pytest.mark.parametrize("kind", ["call", "asian_call"])
def test_heston_pathwise_vs_fd_feller_violated(orc, kind):
    """Config parameters (2 kappa theta = 0.16 < xi^2 = 0.25): v+ hits 0 and
    sqrt(v+) is not Lipschitz there, so the CRN difference converges to the
    pathwise value only as O(sqrt(h)) for v0, kappa, theta and most slowly for
    xi.  S0, r and rho do not touch the kink and stay tight."""
    N, M, T = 1 << 12, 32, 1.0
    pay = [dict(kind=kind, strike=100.0)]
    g = orc.heston_greeks(BASE, T, M, N, pay)[0].mean(axis=1)
    tol = dict(s0=1e-7, r=1e-7, rho=1e-7, v0=1e-4, kappa=1e-4, theta=1e-4, xi=5e-3)
    for k, name in enumerate(orc.HESTON_PARAM_ORDER):
        def price(t, name=name):
            return orc.heston_payoffs(dict(BASE, **{name: t}), T, M, N, pay)[0].mean()
        fd = _fd(price, BASE[name])
        assert abs(g[k] - fd) <= tol[name] * max(1.0, abs(fd)), (name, g[k], fd)


def test_heston_xi_zero_greeks_are_black_scholes(orc):
    """xi = 0, v0 = theta = sigma^2: delta and rho are Black-Scholes; the
    flat-vol vega is 2 sigma (dP/dv0 + dP/dtheta)."""
    h = dict(BASE, xi=0.0)
    N = 1 << 17
    g = orc.heston_greeks(h, 1.0, 16, N, [dict(kind="call", strike=100.0)])[0]
    delta, vega, rho = cf.bs_call_greeks(100.0, 100.0, 0.05, 0.2, 1.0)
    m, se = orc.mean_se(g[0]); assert abs(m - delta) <= 3 * se
    m, se = orc.mean_se(g[2]); assert abs(m - rho) <= 3 * se
    flat = 2 * 0.2 * (g[1] + g[4])
    m, se = orc.mean_se(flat); assert abs(m - vega) <= 3 * se, (m, se, vega)
