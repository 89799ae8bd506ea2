"""Pins of the oracle's continuous barrier monitoring through the Brownian
bridge (Sec. VI.A.1): for GBM the bridge extremes are exact in law given the
grid values, so the estimator is unbiased at any step count.  Pinned by the
paper's own value for the "In and Out Put" (23.1371783926, S0 = 100, K = 120,
H = 140, r = 0.03, sigma = 0.8, read with T = 2) and by the continuous
down-and-in call closed form, at one step and at many; plus in + out =
vanilla per path and the gap to discrete monitoring."""
import numpy as np
import pytest

from closed_forms import bs_call, bs_put, down_and_in_call_continuous, up_and_in_put_continuous

PAPER_IN_OUT_PUT = 23.1371783926


def _mean_se(v):
    return v.mean(), v.std(ddof=1) / np.sqrt(v.size)


@pytest.mark.parametrize("steps", [1, 25])
def test_up_and_in_put_matches_paper_value(orc, steps):
    assert abs(up_and_in_put_continuous(100.0, 120.0, 140.0, 0.03, 0.8, 2.0) - PAPER_IN_OUT_PUT) < 1e-9
    pays = [dict(kind="ui_put", strike=120.0, barrier=140.0)]
    f = orc.gbm1d_bridge_payoffs(100.0, 0.8, 0.03, 2.0, steps, 1 << 17, pays)[0]
    m, se = _mean_se(f)
    assert abs(m - PAPER_IN_OUT_PUT) <= 3 * se, (steps, m, se)


@pytest.mark.parametrize("steps", [1, 16])
def test_down_and_in_call_matches_closed_form(orc, steps):
    S, K, H, r, sg, T = 100.0, 100.0, 85.0, 0.05, 0.3, 1.0
    want = down_and_in_call_continuous(S, K, H, r, sg, T)
    assert 0.5 < want < bs_call(S, K, r, sg, T)
    pays = [dict(kind="di_call", strike=K, barrier=H)]
    f = orc.gbm1d_bridge_payoffs(S, sg, r, T, steps, 1 << 17, pays)[0]
    m, se = _mean_se(f)
    assert abs(m - want) <= 3 * se, (steps, m, se, want)


def test_in_plus_out_is_vanilla_per_path(orc):
    pays = [dict(kind="put", strike=120.0), dict(kind="ui_put", strike=120.0, barrier=140.0),
            dict(kind="uo_put", strike=120.0, barrier=140.0), dict(kind="call", strike=90.0),
            dict(kind="di_call", strike=90.0, barrier=80.0), dict(kind="do_call", strike=90.0, barrier=80.0)]
    f = orc.gbm1d_bridge_payoffs(100.0, 0.5, 0.03, 1.0, 12, 4096, pays)
    assert np.array_equal(f[1] + f[2], f[0])
    assert np.array_equal(f[4] + f[5], f[3])


def test_bridge_knocks_more_often_than_the_grid(orc):
    """The bridge maximum is at least the larger grid value of its step, so a
    continuously monitored in-option is worth at least the discrete one, path
    by path on the same normals; with 25 steps the discrete price misses a
    large part of the continuous value."""
    pays = [dict(kind="ui_put", strike=120.0, barrier=140.0)]
    cont = orc.gbm1d_bridge_payoffs(100.0, 0.8, 0.03, 2.0, 25, 1 << 14, pays)[0]
    disc = orc.gbm_payoffs(np.array([100.0]), np.array([0.8]), 0.03, 2.0, 25, 1 << 14, pays)[0]
    assert np.all(cont >= disc)
    assert disc.mean() < cont.mean() - 1.0
    # the vanilla put is unaffected by the monitoring
    van = orc.gbm1d_bridge_payoffs(100.0, 0.8, 0.03, 2.0, 25, 1 << 14, [dict(kind="put", strike=120.0)])[0]
    m, se = _mean_se(van)
    assert abs(m - bs_put(100.0, 120.0, 0.03, 0.8, 2.0)) <= 3 * se


def test_unmonitored_payoffs_are_the_grid_pricers(orc):
    """European and Asian payoffs do not look at the bridge extremes: on the
    same normals they equal the grid pricer's path by path, for a monitored
    underlying U = w S with w != 1 as well."""
    pays = [dict(kind="call", strike=95.0), dict(kind="put", strike=110.0), dict(kind="asian_call", strike=100.0),
            dict(kind="asian_put", strike=104.0)]
    for w in (1.0, 1.7):
        pw = [dict(p, strike=w * p["strike"]) for p in pays]
        b = orc.gbm1d_bridge_payoffs(100.0, 0.4, 0.03, 1.5, 12, 4096, pw, weight=w)
        g = orc.gbm_payoffs(np.array([100.0]), np.array([0.4]), 0.03, 1.5, 12, 4096, pw, weights=np.array([w]))
        assert np.allclose(b, g, rtol=1e-12, atol=1e-10), w  # U ~ 200: rounding of U near the strike


def test_weighted_barriers_scale(orc):
    """With a monitored underlying U = w S the bridge payoffs (barrier ones
    included) at strike w K and barrier w H are w times those of w = 1 at K
    and H, path by path: the weight reaches the terminal value, the average
    and both monitored extremes."""
    pays = [dict(kind="ui_put", strike=120.0, barrier=140.0), dict(kind="uo_call", strike=95.0, barrier=130.0),
            dict(kind="di_call", strike=90.0, barrier=80.0), dict(kind="do_put", strike=105.0, barrier=85.0)]
    w = 0.6
    scaled = [dict(p, strike=p["strike"] * w, barrier=p["barrier"] * w) for p in pays]
    a = orc.gbm1d_bridge_payoffs(100.0, 0.5, 0.03, 1.0, 16, 4096, scaled, weight=w)
    b = orc.gbm1d_bridge_payoffs(100.0, 0.5, 0.03, 1.0, 16, 4096, pays, weight=1.0)
    assert np.allclose(a, w * b, rtol=1e-12, atol=1e-10)
    assert all(0 < np.count_nonzero(row) < row.size for row in a)
