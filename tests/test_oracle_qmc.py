"""Pins of the oracle's Sobol sequence and randomised quasi-Monte Carlo
(Sec. IV's QRNGs, the Sobol basket experiment of Sec. VI.D), each against a
fact that does not come from the oracle's code:
  * every dimension's first 2^m points fall one per dyadic interval of
    width 2^-m (the defining stratification of a Sobol dimension);
  * dimensions 1 and 2 form a (0, m, 2)-net: every elementary box of area
    2^-m holds exactly one of the first 2^m points;
  * the degree of each dimension's polynomial (read off its direction
    numbers: m_k = 1 up to k = s, then m_{s+1} > 1) follows the count of
    primitive polynomials of degree s over GF(2), phi(2^s - 1) / s;
  * the randomised estimator is unbiased (Black-Scholes within 3 SE) and its
    error falls faster than plain Monte Carlo's N^-1/2;
  * the random digital shift makes every point uniform on the unit cube: the
    first Sobol point is the origin, so across replications its shifted
    coordinates are the shift itself, and the Box-Muller normals they yield
    must be independent standard normals.
"""
import math

import numpy as np
import pytest

from closed_forms import bs_call


def _phi(n):
    r, m, p = n, n, 2
    while p * p <= m:
        if m % p == 0:
            while m % p == 0:
                m //= p
            r -= r // p
        p += 1
    if m > 1:
        r -= r // m
    return r


def test_one_dimensional_stratification(orc):
    for m in (4, 8, 11):
        P = orc.sobol_points(64, 1 << m)
        for j in range(64):
            assert sorted((P[:, j] >> np.uint32(32 - m)).tolist()) == list(range(1 << m)), (m, j)


def test_first_two_dimensions_form_a_0m2_net(orc):
    m = 10
    P = orc.sobol_points(2, 1 << m).astype(np.uint64)
    for i in range(m + 1):
        a = P[:, 0] >> np.uint64(32 - i) if i else np.zeros(1 << m, dtype=np.uint64)
        b = P[:, 1] >> np.uint64(32 - (m - i)) if m - i else np.zeros(1 << m, dtype=np.uint64)
        cells = a * np.uint64(1 << (m - i)) + b
        assert np.unique(cells).size == 1 << m, i


def test_polynomial_degrees_follow_the_primitive_count(orc):
    V = orc.sobol_directions(64)
    degrees = []
    for j in range(1, 64):
        mk = [int(V[j, k]) >> (31 - k) for k in range(32)]
        assert all(v % 2 == 1 and v < (1 << (k + 1)) for k, v in enumerate(mk))  # odd, m_k < 2^k
        s = next(k for k, v in enumerate(mk) if v != 1)  # m_1..m_s = 1, m_{s+1} > 1
        degrees.append(s)
    assert degrees == sorted(degrees)
    counts = {s: degrees.count(s) for s in set(degrees)}
    for s, c in counts.items():
        full = _phi((1 << s) - 1) // s
        assert c == full or (s == max(counts) and c < full), (s, c, full)


def test_rqmc_call_is_unbiased_and_beats_monte_carlo(orc):
    S, K, r, sg, T = 100.0, 105.0, 0.05, 0.25, 1.0
    want = bs_call(S, K, r, sg, T)
    pays = [dict(kind="call", strike=K)]
    spread = {}
    for m in (10, 14):
        means = np.array([orc.qmc_gbm_payoffs(S, sg, r, T, 1, 1 << m, pays, rep=rep)[0].mean() for rep in range(16)])
        se = means.std(ddof=1) / 4.0
        assert abs(means.mean() - want) <= 3 * se + 1e-12, (m, means.mean(), want, se)
        spread[m] = means.std(ddof=1)
    # plain Monte Carlo: spread falls by 4 from 2^10 to 2^14 points; QMC by far more
    assert spread[10] / spread[14] > 12.0, spread
    mc = orc.gbm_payoffs(np.array([S]), np.array([sg]), r, T, 1, 1 << 14, pays)[0]
    assert spread[14] < 0.1 * mc.std(ddof=1) / 128.0


def test_rqmc_basket_matches_monte_carlo(orc):
    import workloads
    s0, sg, corr = workloads.basket_market(16, 4)
    w = np.full(16, 1 / 16)
    K = float(w @ s0)
    pays = [dict(kind="call", strike=K)]
    q = np.array([orc.qmc_gbm_payoffs(s0, sg, 0.05, 1.0, 1, 1 << 12, pays, rep=rep, corr=corr, weights=w)[0].mean()
                  for rep in range(8)])
    mc = orc.gbm_payoffs(s0, sg, 0.05, 1.0, 1, 1 << 17, pays, corr=corr, weights=w)[0]
    se = math.sqrt(q.var(ddof=1) / 8 + mc.var(ddof=1) / mc.size)
    assert abs(q.mean() - mc.mean()) <= 3 * se


def test_digital_shift_makes_the_origin_uniform(orc):
    """At the first Sobol point (all words zero) replication rep's uniforms
    are its shift words; with independent uniform shifts the normals of the
    two Box-Muller pairs (dimensions 0-1 and 2-3) are i.i.d. N(0, 1) across
    replications.  They are read back exactly from a one-asset, two-step
    path: the strike-0 call gives S_2, the strike-0 Asian call (S_1 + S_2)/2."""
    from scipy import stats
    S, r, sg, T, R = 100.0, 0.05, 0.3, 1.0, 4096
    dt = T / 2
    pays = [dict(kind="call", strike=0.0), dict(kind="asian_call", strike=0.0)]
    disc = math.exp(-r * T)
    z = np.empty((2, R))
    for rep in range(R):
        f = orc.qmc_gbm_payoffs(S, sg, r, T, 2, 1, pays, rep=rep)[:, 0] / disc
        s2, s1 = f[0], 2.0 * f[1] - f[0]
        x1, x2 = math.log(s1 / S), math.log(s2 / s1)
        z[:, rep] = [(x - (r - 0.5 * sg * sg) * dt) / (sg * math.sqrt(dt)) for x in (x1, x2)]
    for k in range(2):
        p = stats.kstest(z[k], "norm").pvalue
        assert p > 1e-3, (k, p)
    assert abs(np.corrcoef(z)[0, 1]) < 4.0 / math.sqrt(R)


@pytest.mark.parametrize("scheme", ["log_euler", "euler"])
def test_rqmc_forward_at_another_maturity(orc, scheme):
    """The zero-strike call of the randomised-QMC pricer at T = 2.5 over 4
    steps is the discounted mean terminal price: S0 under log-Euler (exact in
    law) and S0 (1 + r T/M)^M e^{-rT} under Euler (each step's factor has
    mean 1 + r dt), within 3 SE of the replication means."""
    S, r, sg, T, M = 100.0, 0.04, 0.3, 2.5, 4
    pays = [dict(kind="call", strike=0.0)]
    means = np.array([orc.qmc_gbm_payoffs(S, sg, r, T, M, 1 << 10, pays, rep=rep, scheme=scheme)[0].mean()
                      for rep in range(16)])
    want = S if scheme == "log_euler" else S * (1 + r * T / M) ** M * math.exp(-r * T)
    se = means.std(ddof=1) / 4.0
    assert abs(means.mean() - want) <= 3 * se + 1e-9, (scheme, means.mean(), want, se)
    assert abs(want - S * math.exp(-r * T)) > 50 * se  # the discount's T is resolved


def test_point_offset_selects_points(orc):
    """Points [n0, n0 + m) of a replication are the tail of a run over
    [0, n0 + m): each point depends only on its own index."""
    import workloads
    s0, sg, corr = workloads.basket_market(4, 2)
    pays = [dict(kind="call", strike=100.0), dict(kind="asian_put", strike=105.0)]
    a = orc.qmc_gbm_payoffs(s0, sg, 0.05, 1.0, 3, 300, pays, rep=5, corr=corr)
    b = orc.qmc_gbm_payoffs(s0, sg, 0.05, 1.0, 3, 77, pays, rep=5, corr=corr, point_offset=223)
    assert np.array_equal(a[:, 223:], b)
