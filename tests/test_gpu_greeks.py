"""GPU parity of the pathwise Greeks (adjoint kernels) with the oracle's
independent forward-mode Greeks on identical streams, the Black-Scholes
closed forms, common-random-number finite differences (h = 1e-4 relative,
as the Heston workload specifies) and the autograd wrapper."""
import numpy as np
import pytest

import workloads
from closed_forms import bs_call_greeks

pytestmark = pytest.mark.gpu

HES = dict(workloads.HESTON_PARAMS)
ORDER = ("s0", "v0", "r", "kappa", "theta", "xi", "rho")


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def _check(got, ref, orc, names, tol, label, se_frac=0.0):
    """got: [n_pay, G, 2]; ref: oracle per-path [n_pay, G, N].  Passes when
    |gpu - oracle| <= max(tol * |oracle| (floor 1e-2), se_frac * SE)."""
    for p in range(ref.shape[0]):
        for k in range(ref.shape[1]):
            m, se = orc.mean_se(ref[p, k])
            t = tol[names[k]] if isinstance(tol, dict) else tol
            print(f"{label} payoff {p} {names[k]}: gpu {got[p, k, 0]:.6g} oracle {m:.6g} "
                  f"rel {abs(got[p, k, 0] - m) / max(abs(m), 1e-2):.2e} (se {se:.2e})")
            bound = max(t * max(abs(m), 1e-2), se_frac * se)
            assert abs(got[p, k, 0] - m) <= bound, (label, p, names[k], got[p, k, 0], m, bound)


def test_gbm1d_greeks_vs_oracle_and_bs(gb, orc):
    pays = [dict(kind="call", strike=105.0), dict(kind="put", strike=95.0), dict(kind="asian_call", strike=100.0)]
    model = dict(kind="gbm", s0=[100.0], sigma=[0.2], r=0.05)
    cfg = dict(steps=64, T=1.0, paths=1 << 17)
    prices, g = gb.greeks(model, cfg, pays)
    ref = orc.gbm_greeks(100.0, 0.2, 0.05, 1.0, 64, 1 << 17, pays)
    _check(g, ref, orc, ("delta", "vega", "rho"), 2e-5, "gbm")
    want = bs_call_greeks(100.0, 105.0, 0.05, 0.2, 1.0)
    for k in range(3):
        assert abs(g[0, k, 0] - want[k]) <= 3 * g[0, k, 1]
    ref_p = orc.gbm_payoffs(100.0, 0.2, 0.05, 1.0, 64, 1 << 17, pays)
    for i in range(3):
        assert abs(prices[i][0] - ref_p[i].mean()) <= 1e-5 * abs(ref_p[i].mean())


@pytest.mark.parametrize("ckpt", [32, 7, 64])
def test_heston_adjoint_vs_oracle_feller(gb, orc, ckpt):
    """Feller condition met (xi = 0.2): the path map is smooth and the FP32
    adjoint matches the FP64 forward-mode tangents to 1e-5 relative."""
    h = dict(HES, xi=0.2)
    pays = [dict(kind="call", strike=K) for K in (90.0, 100.0, 110.0)] + [dict(kind="asian_call", strike=100.0)]
    cfg = dict(steps=96, T=1.0, paths=1 << 14, ckpt_every=ckpt)
    _, g = gb.greeks(dict(kind="heston", **h), cfg, pays)
    ref = orc.heston_greeks(h, 1.0, 96, 1 << 14, pays)
    _check(g, ref, orc, ORDER, 2e-5, f"heston feller ckpt={ckpt}")


def test_heston_config_adjoint_vs_oracle(gb, orc):
    """The Heston workload (xi = 0.5, Feller violated, 256 steps, checkpoints
    every 32) on an oracle-sized prefix, all 18 payoffs.  d/dS0 and d/dr do
    not pass through the truncated square root: 2e-5.  d/dv0, kappa, theta,
    xi, rho do: a path whose variance lands within FP32 rounding of 0
    contributes dt / (2 sqrt(v+ dt)), unbounded as v -> 0, so FP32 and FP64
    legitimately differ there; they are held to 1e-3 relative or 5 % of the
    Monte Carlo standard error, whichever is larger (measured: <= 2 % of the
    value and <= 1.5 % of the standard error)."""
    w = workloads.heston(paths=1 << 13)
    _, g = gb.greeks(dict(kind="heston", **w["model"]), dict(steps=256, T=1.0, paths=w["paths"], ckpt_every=32),
                     w["payoffs"])
    ref = orc.heston_greeks(w["model"], 1.0, 256, w["paths"], w["payoffs"])
    tol = dict(s0=2e-5, r=2e-5, rho=1e-3, v0=1e-3, kappa=1e-3, theta=1e-3, xi=1e-3)
    _check(g, ref, orc, ORDER, tol, "heston C3", se_frac=0.05)


def test_heston_adjoint_vs_crn_fd(gb, orc):
    """Against central CRN finite differences of the GPU's own prices
    (h = 1e-4 relative): within 3 SE of the FD-pathwise difference budget,
    with the O(sqrt h) kink term of the truncated square root allowed for."""
    w = workloads.heston(paths=1 << 16)
    pays = [dict(kind="call", strike=100.0), dict(kind="asian_call", strike=100.0)]
    cfg = dict(steps=64, T=1.0, paths=w["paths"])
    _, g = gb.greeks(dict(kind="heston", **w["model"]), cfg, pays)
    h = 1e-4
    for k, name in enumerate(ORDER):
        up = gb.price(dict(kind="heston", **dict(w["model"], **{name: w["model"][name] * (1 + h)})), cfg, pays)
        dn = gb.price(dict(kind="heston", **dict(w["model"], **{name: w["model"][name] * (1 - h)})), cfg, pays)
        for p in range(2):
            fd = (up[p][0] - dn[p][0]) / (2 * h * w["model"][name])
            assert abs(g[p, k, 0] - fd) <= 3 * g[p, k, 1] + 0.02 * abs(fd) + 1e-3, (name, p, g[p, k, 0], fd)


def test_heston_xi_zero_is_black_scholes(gb):
    h = dict(HES, xi=0.0)
    _, g = gb.greeks(dict(kind="heston", **h), dict(steps=32, T=1.0, paths=1 << 18),
                     [dict(kind="call", strike=100.0)])
    delta, vega, rho = bs_call_greeks(100.0, 100.0, 0.05, 0.2, 1.0)
    assert abs(g[0, 0, 0] - delta) <= 3 * g[0, 0, 1]
    assert abs(g[0, 2, 0] - rho) <= 3 * g[0, 2, 1]
    flat = 2 * 0.2 * (g[0, 1, 0] + g[0, 4, 0])
    assert abs(flat - vega) <= 3 * (g[0, 1, 1] + g[0, 4, 1]) * 0.4 + 0.05


def test_autograd_backward_calls_adjoint(gb):
    import torch
    params = torch.tensor([HES[k] for k in ORDER], dtype=torch.float64, requires_grad=True)
    cfg = dict(steps=64, T=1.0, paths=1 << 14)
    pays = [dict(kind="call", strike=100.0), dict(kind="asian_call", strike=95.0)]
    prices = gb.HestonPricer.apply(params, cfg, pays)
    (prices[0] + 2 * prices[1]).backward()
    _, g = gb.greeks(dict(kind="heston", **HES), cfg, pays)
    assert np.allclose(params.grad.numpy(), g[0, :, 0] + 2 * g[1, :, 0], rtol=1e-12, atol=1e-12)
    p2 = torch.tensor([100.0, 0.2, 0.05], dtype=torch.float64, requires_grad=True)
    gb.GbmPricer.apply(p2, cfg, [dict(kind="call", strike=100.0)]).sum().backward()
    delta, vega, rho = bs_call_greeks(100.0, 100.0, 0.05, 0.2, 1.0)
    assert np.allclose(p2.grad.numpy(), [delta, vega, rho], rtol=0.05)


def test_greeks_reject_barrier_and_euler(gb):
    from paper_1906_02818_gb300 import native
    with pytest.raises(native.MCError) as e:
        gb.greeks(dict(kind="heston", **HES), dict(steps=8, T=1.0, paths=64),
                  [dict(kind="uo_call", strike=100.0, barrier=120.0)])
    assert e.value.status == native.MC_EUNSUPPORTED
    with pytest.raises(native.MCError):
        gb.greeks(dict(kind="gbm", s0=[100.0], sigma=[0.2], r=0.05),
                  dict(steps=8, T=1.0, paths=64, scheme="euler"), [dict(kind="call", strike=100.0)])
