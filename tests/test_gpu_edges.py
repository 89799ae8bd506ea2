"""Edge cases of the pricing kernels against the oracle: the maximum number of
payoffs in one launch (MC_MAX_PAYOFFS = 32), zero volatility (every path is
the deterministic forward: closed form, zero standard error), and tensor-core
launches smaller than one 128-path tile."""
import math

import numpy as np
import pytest

import workloads
from gpu_util import REL, assert_price_close, cfg_of, gbm_model, oracle_gbm
from test_gpu_price import barrier_band_mass
from test_gpu_tc import emulate, flip_bound, payoffs_from_U

pytestmark = pytest.mark.gpu

MAX_PAYOFFS = 32


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def _many_payoffs(s0):
    kinds = ["call", "put", "asian_call", "asian_put", "uo_call", "ui_call", "uo_put", "ui_put",
             "do_call", "di_call", "do_put", "di_put"]
    pays = []
    for i in range(MAX_PAYOFFS):
        k = kinds[i % len(kinds)]
        K = s0 * (0.8 + 0.4 * i / (MAX_PAYOFFS - 1))
        p = dict(kind=k, strike=K)
        if k.startswith("u"):
            p["barrier"] = s0 * 1.35
        elif k.startswith("d"):
            p["barrier"] = s0 * 0.7
        pays.append(p)
    return pays


def test_maximum_payoff_count_1d(gb, orc):
    """32 payoffs of every kind on one 1-D launch, each against the oracle
    (the barrier ones up to the paths whose extreme is within the FP32 band
    of the barrier)."""
    w = workloads.gbm_1d(paths=5000, steps=32)
    pays = _many_payoffs(100.0)
    got = gb.price(gbm_model(w), cfg_of(w), pays)
    ref = oracle_gbm(orc, w, w["paths"], pays)
    U = orc.gbm_paths(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], w["paths"])[:, 0]
    assert_price_close(got, ref, pays, barrier_band_mass(orc, U, ref, pays), "32 payoffs")
    with pytest.raises(Exception):
        gb.price(gbm_model(w), cfg_of(w), pays + [dict(kind="call", strike=100.0)])


def test_zero_volatility_is_the_forward(gb):
    """sigma = 0: every path follows the forward S0 e^{r t}; the call is
    e^{-rT} (sum w S0 e^{rT} - K)^+ with zero standard error, for the 1-D,
    FP32 basket and BF16 tensor-core kernels."""
    r, T, K = 0.05, 1.0, 95.0
    want = math.exp(-r * T) * max(100.0 * math.exp(r * T) - K, 0.0)
    pay = [dict(kind="call", strike=K), dict(kind="asian_call", strike=K)]
    fwd_avg = 100.0 * np.mean(np.exp(r * T * np.arange(1, 17) / 16))
    want_avg = math.exp(-r * T) * max(fwd_avg - K, 0.0)
    for d, prec in [(1, "fp32"), (8, "fp32"), (64, "bf16")]:
        model = dict(kind="gbm", s0=np.full(d, 100.0), sigma=np.zeros(d), r=r,
                     corr=None if d == 1 else np.eye(d))
        got = gb.price(model, dict(steps=16, T=T, paths=1000, precision=prec), pay)
        assert abs(got[0][0] - want) <= 2e-5 * want, (d, prec, got[0][0], want)
        assert abs(got[1][0] - want_avg) <= 2e-5 * want_avg, (d, prec, got[1][0], want_avg)
        assert got[0][1] <= 1e-3 * want, (d, prec, got[0][1])  # FP32 moment sums: ~1e-4, vs ~0.45 at sigma 0.2


@pytest.mark.parametrize("paths", [1, 5, 127])
def test_tensor_core_launch_below_one_tile(gb, orc, paths):
    """Fewer paths than one 128-row tile on the BF16 tensor-core path: the
    rows past the path count are simulated as zeros and left out."""
    w = workloads.basket_d64(paths=paths, steps=6)
    pays = [dict(kind="call", strike=float(w["weights"] @ w["s0"]))]
    got = gb.price(gbm_model(w), cfg_of(w, precision="bf16"), pays)
    U, aux = emulate(orc, w, "bf16", paths, w["steps"], detail=True)
    m = payoffs_from_U(U, pays, w["r"], w["T"])[0].mean()
    fb = flip_bound(aux, U, pays, w["r"], w["T"])[0]
    assert abs(got[0][0] - m) <= REL * max(abs(m), 1e-6) + fb + 1e-9, (paths, got[0][0], m)


@pytest.mark.parametrize("d", [2, 16, 64, 100])
def test_indefinite_correlation_is_reported(gb, d):
    """A correlation matrix with entries in [-1, 1] that is not positive
    definite (d = 2: correlation 1, a zero second pivot; otherwise three
    assets at 0.9, 0.9, -0.9, determinant -2.89) makes the device's FP64
    Cholesky report MC_ENOTPSD (the small-matrix kernel for d <= 64, the
    general one above), on the FP32 and BF16 paths; the library stays usable,
    and the same market with a valid correlation prices."""
    from paper_1906_02818_gb300 import native
    corr = np.eye(d)
    if d == 2:
        corr[0, 1] = corr[1, 0] = 1.0
    else:
        corr[0, 1] = corr[1, 0] = corr[0, 2] = corr[2, 0] = 0.9
        corr[1, 2] = corr[2, 1] = -0.9
    assert np.linalg.eigvalsh(corr).min() <= 1e-12
    model = dict(kind="gbm", s0=np.full(d, 100.0), sigma=np.full(d, 0.2), r=0.05, corr=corr)
    pays = [dict(kind="call", strike=100.0)]
    for prec in ("fp32", "bf16"):
        with pytest.raises(native.MCError) as e:
            gb.price(model, dict(steps=4, T=1.0, paths=256, precision=prec), pays)
        assert e.value.status == native.MC_ENOTPSD
    valid = np.where(np.eye(d) > 0, 1.0, np.where(corr != 0, 0.5, 0.0))
    got = gb.price(dict(model, corr=valid), dict(steps=4, T=1.0, paths=256), pays)
    assert got[0][0] > 0 and np.isfinite(got[0][1])


@pytest.mark.parametrize("d", [2, 16, 100])
def test_rank_deficient_correlation_threshold(gb, d):
    """Semi-definite (rank-deficient) correlations are rejected by the pivot
    threshold of the device Cholesky (a pivot at or below 4 d 2^-52 of its
    diagonal entry), not by how one rounding falls: d = 2 with correlation 1
    and 1 - 2^-53 (pivots 0 and ~2e-16, far below the threshold), and a
    rank-4 factor correlation for d = 16 and 100 (pivots from the fifth on
    are rounding noise).  Nearly singular but positive definite matrices
    (d = 2 at 1 - 1e-12, pivot 2e-12; the rank-4 correlation plus 1e-9 I)
    are accepted and priced."""
    from paper_1906_02818_gb300 import native
    pays = [dict(kind="call", strike=100.0)]
    model = dict(kind="gbm", s0=np.full(d, 100.0), sigma=np.full(d, 0.2), r=0.05)
    if d == 2:
        bad = [np.array([[1.0, c], [c, 1.0]]) for c in (1.0, 1.0 - 2.0 ** -53)]
        good = [np.array([[1.0, 1.0 - 1e-12], [1.0 - 1e-12, 1.0]])]
    else:
        F = np.random.default_rng(d).standard_normal((d, 4))
        C = F @ F.T
        C = C / np.sqrt(np.outer(np.diag(C), np.diag(C)))
        np.fill_diagonal(C, 1.0)
        C = 0.5 * (C + C.T)
        bad = [C]
        G = C + 1e-9 * np.eye(d)
        G = G / np.sqrt(np.outer(np.diag(G), np.diag(G)))
        np.fill_diagonal(G, 1.0)
        good = [0.5 * (G + G.T)]
    for corr in bad:
        for prec in ("fp32", "bf16"):
            with pytest.raises(native.MCError) as e:
                gb.price(dict(model, corr=corr), dict(steps=4, T=1.0, paths=256, precision=prec), pays)
            assert e.value.status == native.MC_ENOTPSD
    for corr in good:
        got = gb.price(dict(model, corr=corr), dict(steps=4, T=1.0, paths=256), pays)
        assert got[0][0] > 0 and np.isfinite(got[0][1])
