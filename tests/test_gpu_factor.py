"""GPU parity of the factor-model basket (loadings B, rho = B B^T + diag(e^2))
with the FP64 oracle on identical streams: aligned and unaligned stream
layouts, one and two warps per path group, no factors, both schemes, barrier
payoffs; and the d = 512 workload against the Cholesky scheme (same law,
other normals)."""
import numpy as np
import pytest

import workloads
from gpu_util import BAND, REL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def _pays(b0):
    return [dict(kind="call", strike=b0), dict(kind="put", strike=1.03 * b0), dict(kind="asian_call", strike=0.98 * b0),
            dict(kind="uo_call", strike=b0, barrier=1.2 * b0), dict(kind="di_put", strike=b0, barrier=0.85 * b0)]


def _band_mass(orc, s0, sg, B, w, steps, paths, pays, scheme):
    out = []
    for p in pays:
        if p["kind"][:2] not in ("uo", "ui", "do", "di"):
            out.append(None)
            continue
        up = p["kind"][0] == "u"
        probe = [dict(kind="ui_call" if up else "di_call", strike=0.0, barrier=p["barrier"] * (1 - BAND)),
                 dict(kind="ui_call" if up else "di_call", strike=0.0, barrier=p["barrier"] * (1 + BAND)),
                 dict(kind="call" if "call" in p["kind"] else "put", strike=p["strike"])]
        f = orc.gbm_factor_payoffs(s0, sg, B, 0.05, 1.0, steps, paths, probe, weights=w, scheme=scheme)
        near = (f[0] > 0) != (f[1] > 0)
        out.append(float(f[2][near].sum()) / paths * 1.01 + 1e-12)
    return out


@pytest.mark.parametrize("d,k,scheme", [(8, 4, "log_euler"), (6, 2, "log_euler"), (100, 3, "euler"),
                                        (300, 16, "log_euler"), (512, 16, "euler"), (5, 0, "log_euler"),
                                        (64, 8, "euler")])
def test_factor_basket_matches_oracle(gb, orc, d, k, scheme):
    from gpu_util import assert_price_close
    s0, sg, B = workloads.basket_market_factors(d, max(k, 1), seed=d + k)
    B = B[:, :k]
    w = np.full(d, 1.0 / d)
    pays = _pays(float(w @ s0))
    steps, paths = 6, 777
    model = dict(kind="gbm", s0=s0, sigma=sg, loadings=B, weights=w, r=0.05)
    got = gb.price(model, dict(steps=steps, T=1.0, paths=paths, seed=42, scheme=scheme), pays)
    ref = orc.gbm_factor_payoffs(s0, sg, B, 0.05, 1.0, steps, paths, pays, weights=w, scheme=scheme)
    assert_price_close(got, ref, pays, _band_mass(orc, s0, sg, B, w, steps, paths, pays, scheme), f"{d}/{k}/{scheme}")


def test_d512_factor_model_matches_cholesky_scheme(gb):
    """The d = 512 market simulated both ways: the same law, other normals."""
    wf = workloads.basket_d512_factor(paths=1 << 18)
    wc = workloads.basket_d512(paths=1 << 18)
    cfg = dict(steps=wf["steps"], T=wf["T"], paths=wf["paths"], seed=42)
    f, = gb.price(dict(kind="gbm", s0=wf["s0"], sigma=wf["sigma"], loadings=wf["loadings"], weights=wf["weights"],
                       r=wf["r"]), cfg, wf["payoffs"])
    c, = gb.price(dict(kind="gbm", s0=wc["s0"], sigma=wc["sigma"], corr=wc["corr"], weights=wc["weights"], r=wc["r"]),
                  dict(cfg, precision="bf16"), wc["payoffs"])
    print(f"d=512 factor {f[0]:.5f} +- {f[1]:.5f}, cholesky (bf16) {c[0]:.5f} +- {c[1]:.5f}")
    assert abs(f[0] - c[0]) <= 3.5 * np.hypot(f[1], c[1])


def test_factor_model_unsupported_calls(gb):
    from paper_1906_02818_gb300 import native
    s0, sg, B = workloads.basket_market_factors(8, 2)
    model = dict(kind="gbm", s0=s0, sigma=sg, loadings=B, r=0.05)
    cfg = dict(steps=4, T=1.0, paths=64)
    pays = [dict(kind="call", strike=100.0)]
    for call in (lambda: gb.greeks(model, cfg, [dict(kind="asian_call", strike=100.0)]),
                 lambda: gb.greeks(model, dict(cfg, scheme="euler"), pays),
                 lambda: gb.price_qmc(model, cfg, pays),
                 lambda: gb.price_mlmc(model, dict(cfg, precision="bf16"), pays, 64),
                 lambda: gb.price(model, dict(cfg, precision="bf16"), pays)):
        with pytest.raises(native.MCError) as e:
            call()
        assert e.value.status == native.MC_EUNSUPPORTED


@pytest.mark.parametrize("d,k,paths,steps,kind", [(12, 4, 3000, 8, "call"), (37, 3, 2000, 6, "put"),
                                                  (300, 16, 1500, 4, "call")])
def test_factor_greeks_match_oracle(gb, orc, d, k, paths, steps, kind):
    """Pathwise delta_a, vega_a and rho of the factor-model kernel against the
    oracle's per-path terms on the same stream: d = 12 (aligned Philox
    blocks), d = 37 with k = 3 (unaligned, blocks straddle), d = 300 with
    k = 16 (two warps per path group); each Greek within 2e-5 of the
    largest |delta| (or its own size) plus the terms of the paths whose basket
    lies within the FP32 band of the strike."""
    s0, sg, B = workloads.basket_market_factors(d, k, seed=d)
    w = np.full(d, 1.0 / d)
    K = float(w @ s0) * (1.0 if kind == "call" else 1.02)
    pay = dict(kind=kind, strike=K)
    model = dict(kind="gbm", s0=s0, sigma=sg, loadings=B, weights=w, r=0.04)
    pr, g = gb.greeks(model, dict(steps=steps, T=1.0, paths=paths, seed=42), [pay])
    ref = orc.gbm_factor_greeks(s0, sg, B, 0.04, 1.0, steps, paths, pay, weights=w)
    f, ST = orc.gbm_factor_payoffs(s0, sg, B, 0.04, 1.0, steps, paths, [pay], weights=w, terminal=True)
    m, se = orc.mean_se(f[0])
    assert abs(pr[0][0] - m) <= REL * abs(m) and abs(pr[0][1] - se) <= 1e-3 * se
    U = w @ ST
    band = np.abs(U - K) <= BAND * K
    scale = np.max(np.abs(ref[:d].mean(axis=1)))
    for j in range(2 * d + 1):
        want, sej = orc.mean_se(ref[j])
        tol = 2e-5 * max(abs(want), scale) + np.abs(ref[j][band]).sum() / paths + 1e-12
        assert abs(g[0, j, 0] - want) <= tol, (d, j, g[0, j, 0], want, tol, int(band.sum()))
        assert abs(g[0, j, 1] - sej) <= 1e-3 * sej + 1e-9 + np.abs(ref[j][band]).sum() / paths, (d, j)
