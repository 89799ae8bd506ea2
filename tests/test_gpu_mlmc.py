"""GPU parity of the two-level precision estimator (mc_price_mlmc, Sec. V):
the correction level's per-path FP32 and reduced-precision payoffs against
the FP64 oracle and the oracle's normals rounded as the tensor cores round
them, on the same paths; the combined estimate against the plain FP32 price;
and the variance of the correction against a plain estimate."""
import numpy as np
import pytest

import workloads
from gpu_util import BAND, REL, cfg_of, gbm_model, oracle_gbm
from test_gpu_tc import emulate, flip_bound, payoffs_from_U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


PAYS = [dict(kind="call", strike=0.0), dict(kind="asian_call", strike=0.0), dict(kind="uo_call", strike=0.0, barrier=0.0)]


def _case(d, paths, steps, seed=3):
    s0, sg, corr = workloads.basket_market(d, 3, seed=seed)
    w = np.full(d, 1.0 / d)
    b0 = float(w @ s0)
    pays = [dict(kind="call", strike=b0), dict(kind="asian_call", strike=0.98 * b0),
            dict(kind="uo_call", strike=b0, barrier=1.15 * b0)]
    return dict(s0=s0, sigma=sg, corr=corr, weights=w, r=0.05, T=1.0, steps=steps, paths=paths, seed=42), pays


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp8"])
@pytest.mark.parametrize("d", [8, 64])
def test_correction_level_matches_oracle(gb, orc, prec, d):
    N0, N1, steps = 1000, 700, 12
    w, pays = _case(d, N0, steps)
    res = gb.price_mlmc(gbm_model(w), cfg_of(w, precision=prec), pays, N1)
    exact = oracle_gbm(orc, w, N1, pays, path_offset=N0)                # FP32 level, FP64 arithmetic
    U, aux = emulate(orc, w, prec, N1, steps, path_offset=N0, detail=True)   # reduced-precision level
    quant = payoffs_from_U(U, pays, w["r"], w["T"])
    fb = flip_bound(aux, U, pays, w["r"], w["T"])
    for i, p in enumerate(pays):
        scale = max(abs(exact[i].mean()), 1e-3)
        flip = fb[i]
        if p["kind"] == "uo_call":  # paths whose monitored max is within the FP32 band of H on either side
            near = np.abs(U[1:].max(axis=0) - p["barrier"]) <= 4 * BAND * p["barrier"]
            flip += 2.02 * float(np.maximum(U[-1][near] - p["strike"], 0).sum()) / N1
        for key, want in [("ref_level", exact[i]), ("coarse_level", quant[i]), ("correction", exact[i] - quant[i])]:
            got = res[i][key][0]
            assert abs(got - want.mean()) <= 2 * REL * scale + flip, (prec, d, p["kind"], key, got, want.mean())
        assert abs(res[i]["price"] - (res[i]["coarse"][0] + res[i]["correction"][0])) <= 1e-12 * scale


def test_two_level_estimate_recovers_fp32_price(gb):
    """The d = 64 workload with E4M3 coarse paths (relative bias ~2e-3, many
    standard errors of the correction): the estimate agrees with the FP32
    price on the same first 2^18 paths to within the correction's noise, and
    the correction's standard error is far below a plain estimate's."""
    w = workloads.basket_d64()
    N0, N1 = w["paths"], 1 << 14
    model = gbm_model(w)
    res = gb.price_mlmc(model, cfg_of(w, precision="fp8"), w["payoffs"], N1)
    fp32 = gb.price(model, cfg_of(w), w["payoffs"])
    q = gb.price(model, cfg_of(w, precision="fp8"), w["payoffs"])
    for i in range(len(w["payoffs"])):
        r = res[i]
        bias = q[i][0] - fp32[i][0]
        se_c = r["correction"][1]
        print(f"payoff {i}: fp8 bias {bias:+.5f}, correction {r['correction'][0]:+.5f} +- {se_c:.5f}, "
              f"two-level {r['price']:.5f} vs fp32 {fp32[i][0]:.5f}; plain se at N1 {r['ref_level'][1]:.5f}")
        assert abs(bias) > 5 * se_c  # the reduced precision is visibly biased ...
        assert abs(r["price"] - fp32[i][0]) <= 4 * se_c * np.sqrt(1 + N1 / N0)  # ... and corrected
        assert se_c < 0.2 * r["ref_level"][1]
