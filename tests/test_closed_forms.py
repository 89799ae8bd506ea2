"""Pins of the textbook closed forms that pin the oracle (tests/closed_forms.py),
each against something other than itself: numerical integration of the
payoff against the lognormal density, finite differences, put-call parity,
and the limits in which a formula reduces to another (one monitoring date,
one asset, a barrier at the spot or out of reach, zero volatility of
variance)."""
import math

import numpy as np
import pytest

import closed_forms as cf


def _lognormal_expectation(payoff, S, r, sigma, T):
    """E[payoff(S_T)] for S_T = S exp((r - sigma^2/2) T + sigma sqrt(T) Z),
    by adaptive quadrature over Z."""
    from scipy.integrate import quad
    m, s = (r - 0.5 * sigma * sigma) * T, sigma * math.sqrt(T)
    val, _ = quad(lambda z: payoff(S * math.exp(m + s * z)) * cf.npdf(z), -12.0, 12.0, limit=400, points=[0.0])
    return val


@pytest.mark.parametrize("S,K,r,sigma,T", [(100, 120, 0.05, 0.2, 1.0), (90, 80, 0.02, 0.45, 2.5),
                                           (100, 100, 0.0, 0.3, 0.25)])
def test_black_scholes_by_quadrature_and_parity(S, K, r, sigma, T):
    disc = math.exp(-r * T)
    call = disc * _lognormal_expectation(lambda x: max(x - K, 0.0), S, r, sigma, T)
    put = disc * _lognormal_expectation(lambda x: max(K - x, 0.0), S, r, sigma, T)
    assert cf.bs_call(S, K, r, sigma, T) == pytest.approx(call, rel=1e-8, abs=1e-10)
    assert cf.bs_put(S, K, r, sigma, T) == pytest.approx(put, rel=1e-8, abs=1e-10)
    assert cf.bs_call(S, K, r, sigma, T) - cf.bs_put(S, K, r, sigma, T) == pytest.approx(S - K * disc, abs=1e-10)


def test_black_scholes_greeks_by_differences():
    S, K, r, sigma, T = 100.0, 95.0, 0.04, 0.3, 1.5
    delta, vega, rho = cf.bs_call_greeks(S, K, r, sigma, T)
    h = 1e-5
    assert delta == pytest.approx((cf.bs_call(S + h, K, r, sigma, T) - cf.bs_call(S - h, K, r, sigma, T)) / (2 * h),
                                  rel=1e-7)
    assert vega == pytest.approx((cf.bs_call(S, K, r, sigma + h, T) - cf.bs_call(S, K, r, sigma - h, T)) / (2 * h),
                                 rel=1e-7)
    assert rho == pytest.approx((cf.bs_call(S, K, r + h, sigma, T) - cf.bs_call(S, K, r - h, sigma, T)) / (2 * h),
                                rel=1e-7)


def test_lognormal_call_by_quadrature():
    from scipy.integrate import quad
    for mu, s2, K in [(4.6, 0.04, 100.0), (0.1, 0.5, 0.8), (2.0, 0.01, 9.0)]:
        s = math.sqrt(s2)
        zk = (math.log(K) - mu) / s  # the payoff's kink
        val, _ = quad(lambda z: max(math.exp(mu + s * z) - K, 0.0) * cf.npdf(z), zk, 12, limit=400)
        assert cf.lognormal_call(mu, s2, K) == pytest.approx(val, rel=1e-8)


def test_geometric_forms_reduce_to_black_scholes():
    """One monitoring date: the geometric Asian is the vanilla call; one
    asset (or perfectly correlated equal assets): so is the geometric basket."""
    S, K, r, sigma, T = 100.0, 105.0, 0.05, 0.25, 1.3
    bs = cf.bs_call(S, K, r, sigma, T)
    assert cf.geometric_asian_call(S, K, r, sigma, T, 1) == pytest.approx(bs, rel=1e-12)
    assert cf.geometric_basket_call([S], [sigma], [[1.0]], [1.0], K, r, T) == pytest.approx(bs, rel=1e-12)
    assert cf.geometric_basket_call([S, S], [sigma, sigma], np.ones((2, 2)), [0.3, 0.7], K, r, T) == \
        pytest.approx(bs, rel=1e-12)
    # more monitoring dates average the path: the geometric Asian is cheaper
    assert cf.geometric_asian_call(S, K, r, sigma, T, 12) < bs


def test_geometric_asian_variance_against_the_sum():
    """log G = (1/M) sum_i log S(t_i): its variance sigma^2 dt / M^2
    sum_{i,j} min(i, j), its mean log S + (r - sigma^2/2) dt (M + 1) / 2,
    computed term by term, give the same price."""
    S, K, r, sigma, T, M = 100.0, 98.0, 0.03, 0.35, 2.0, 7
    dt = T / M
    var = sigma * sigma * dt / M ** 2 * sum(min(i, j) for i in range(1, M + 1) for j in range(1, M + 1))
    mean = math.log(S) + (r - 0.5 * sigma * sigma) * dt * sum(range(1, M + 1)) / M
    want = math.exp(-r * T) * cf.lognormal_call(mean, var, K)
    assert cf.geometric_asian_call(S, K, r, sigma, T, M) == pytest.approx(want, rel=1e-12)


def test_one_step_barrier_by_quadrature():
    S, K, H, r, sigma, T = 100.0, 95.0, 130.0, 0.05, 0.3, 1.0
    want = math.exp(-r * T) * _lognormal_expectation(lambda x: (x - K) if K < x < H else 0.0, S, r, sigma, T)
    assert cf.one_step_up_and_out_call(S, K, H, r, sigma, T) == pytest.approx(want, rel=1e-7)
    assert cf.one_step_up_and_out_call(S, K, 1e9, r, sigma, T) == pytest.approx(cf.bs_call(S, K, r, sigma, T),
                                                                                rel=1e-12)


def test_continuous_barriers_at_their_limits():
    """A knock-in barrier at the spot has already been touched: the vanilla
    option; one far away is never touched: nothing."""
    S, r, sigma, T = 100.0, 0.03, 0.4, 1.5
    assert cf.up_and_in_put_continuous(S, 110.0, S * (1 + 1e-12), r, sigma, T) == \
        pytest.approx(cf.bs_put(S, 110.0, r, sigma, T), rel=1e-8)
    assert cf.up_and_in_put_continuous(S, 110.0, 1e4, r, sigma, T) < 1e-10
    assert cf.down_and_in_call_continuous(S, 90.0, S * (1 - 1e-12), r, sigma, T) == \
        pytest.approx(cf.bs_call(S, 90.0, r, sigma, T), rel=1e-8)
    assert cf.down_and_in_call_continuous(S, 90.0, 1e-3, r, sigma, T) < 1e-10


def test_continuous_barrier_by_the_reflection_density():
    """The down-and-in call with H <= K against quadrature of the payoff over
    the reflected density: for a drifted Brownian motion X started at 0 with
    drift nu and volatility sigma, the density of X_T on paths whose minimum
    reached b < 0 is, for x > b, exp(2 nu b / sigma^2) phi_T(x - 2 b)."""
    from scipy.integrate import quad
    S, K, H, r, sigma, T = 100.0, 100.0, 85.0, 0.05, 0.3, 1.0
    nu, b, s = r - 0.5 * sigma * sigma, math.log(H / S), sigma * math.sqrt(T)

    def dens(x):  # x = log(S_T / S)
        return math.exp(2 * nu * b / sigma ** 2) * cf.npdf((x - 2 * b - nu * T) / s) / s

    val, _ = quad(lambda x: max(S * math.exp(x) - K, 0.0) * dens(x), math.log(K / S), 12 * s, limit=400)
    assert cf.down_and_in_call_continuous(S, K, H, r, sigma, T) == pytest.approx(math.exp(-r * T) * val, rel=1e-8)


def test_heston_reduces_to_black_scholes():
    """xi -> 0 with v0 = theta: deterministic variance theta, the
    Black-Scholes call at sigma = sqrt(theta) (the gap falls linearly in xi)."""
    bs = cf.bs_call(100.0, 95.0, 0.05, 0.2, 1.0)
    gaps = [cf.heston_call(100.0, 95.0, 0.05, 1.0, 0.04, 2.0, 0.04, xi, -0.7) - bs for xi in (1e-3, 1e-4)]
    assert abs(gaps[1]) < 1e-3 and 5.0 < gaps[0] / gaps[1] < 20.0
