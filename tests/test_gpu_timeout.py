"""The failure path of the bounded device waits (every mbarrier wait of the
tensor-core kernels gives up after a cap of polls).  With GBMC_TEST_STALL=1
each tensor-core kernel starts with a wait on a barrier phase that nothing
completes, before it has issued any asynchronous copy or MMA, so the wait
runs out deterministically: the kernel records the failure, frees its TMEM
and still finishes its reduction.  The calls must report MC_ETIMEOUT (host
outputs untouched; the network's device rows NaN), and the same calls made
afterwards with the default cap must reproduce the results of a run made
before (bit for bit where the kernel's reduction order is fixed, to rounding
where shared-memory atomics order it): the library and the context stay
usable."""
import contextlib
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


@contextlib.contextmanager
def stalled(cap="2000"):
    """Requests the stall in every tensor-core kernel launched inside; a
    small cap keeps each expiring wait short.  The variables are read by the
    library on every call."""
    os.environ["GBMC_TEST_STALL"] = "1"
    os.environ["GBMC_WAIT_CAP"] = cap
    try:
        yield
    finally:
        del os.environ["GBMC_TEST_STALL"]
        del os.environ["GBMC_WAIT_CAP"]


def _price_expect_timeout(gb, model, cfg, pays):
    from paper_1906_02818_gb300 import api, native
    import ctypes
    L = native.lib()
    mm = api._Marshalled(model, cfg, pays)
    out = (native.McResult * mm.n_payoff)()
    for r in out:
        r.price, r.se = 12345.0, -1.0
    rc = L.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out, None)
    assert rc == native.MC_ETIMEOUT, (rc, L.mc_last_error())
    assert b"bounded wait" in L.mc_last_error()
    assert all(r.price == 12345.0 and r.se == -1.0 for r in out)  # untouched


@pytest.mark.parametrize("case", ["d64_bf16_monitored", "d64_fp8", "d512_bf16", "d512_greeks"])
def test_basket_kernels_time_out_and_recover(gb, orc, case):
    import torch
    if case.startswith("d64"):
        w = workloads.basket_d64(paths=3000, steps=12)
        prec = "bf16" if case == "d64_bf16_monitored" else "fp8"
        pays = w["payoffs"] if prec == "bf16" else [w["payoffs"][0]]
    else:
        w = workloads.basket_d512(paths=2000, steps=4)
        prec = "bf16"
        pays = w["payoffs"]
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
    cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"], precision=prec)
    if case == "d512_greeks":
        before = gb.greeks(model, cfg, pays)
        with stalled():
            with pytest.raises(gb.MCError) as ei:
                gb.greeks(model, cfg, pays)
            assert ei.value.status == -5
        after = gb.greeks(model, cfg, pays)
        for a, b in zip(before, after):  # the large-basket kernel adds its CTA sums in any order
            assert np.allclose(np.asarray(a), np.asarray(b), rtol=1e-6, atol=1e-9)
        return
    before = gb.price(model, cfg, pays)
    with stalled():
        _price_expect_timeout(gb, model, cfg, pays)
        _price_expect_timeout(gb, model, cfg, pays)  # twice in a row
    after = gb.price(model, cfg, pays)
    if case.startswith("d64"):
        assert after == before, (before, after)
    else:  # the large-basket kernel adds its CTA sums in any order
        assert np.allclose(np.asarray(after), np.asarray(before), rtol=1e-6, atol=0), (before, after)
    # and the recovered result is the method's: within 3 SE of the FP64 oracle
    ref = orc.gbm_payoffs(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], w["paths"], pays, corr=w["corr"],
                          weights=w["weights"], seed=w["seed"])
    for (p, se), row in zip(after, ref):
        m, _ = orc.mean_se(row)
        assert abs(p - m) <= 3 * se + 1e-9, (p, m, se)
    torch.cuda.synchronize()


def test_network_kernels_time_out_and_recover(gb):
    import torch
    net = gb.Mlp(5, 256, 4, workloads.mlp_init())
    x = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, (3000, 5)).astype(np.float32)).cuda()
    t = torch.from_numpy(np.random.default_rng(4).uniform(0, 0.3, 3000).astype(np.float32)).cuda()
    y0 = net.forward(x, "bf16").cpu().numpy()
    pf = workloads.risk_portfolio(n_under=4, per_under=8, seed=7, barriers=False)
    r0 = gb.risk(pf, n_scen=2048, method="surrogate", surrogate=net, surrogate_precision="bf16")
    net.set_train_mode("tf32x3")
    l0, g0 = net.loss_grad(x[:2048], t[:2048])
    gd = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, (3000, 2)).astype(np.float32)).cuda()
    d0, gr0 = net.loss_grad_d(x[:2048], t[:2048], gd[:2048], [0, 1], [1.0, 1.0], [0.5, 0.5])
    with stalled():
        # inference: asynchronous, the failure shows as NaN rows ...
        y = net.forward(x, "bf16").cpu().numpy()
        assert np.isnan(y).all()
        # ... and is reported by the next synchronising call on the network
        with pytest.raises(gb.MCError) as ei:
            gb.risk(pf, n_scen=2048, method="surrogate", surrogate=net, surrogate_precision="bf16")
        assert ei.value.status == -5
        # training products on the tensor cores (three-pass TF32), plain and
        # with derivative labels
        with pytest.raises(gb.MCError) as ei:
            net.loss_grad(x[:2048], t[:2048])
        assert ei.value.status == -5
        with pytest.raises(gb.MCError) as ei:
            net.loss_grad_d(x[:2048], t[:2048], gd[:2048], [0, 1], [1.0, 1.0], [0.5, 0.5])
        assert ei.value.status == -5
    assert np.array_equal(net.forward(x, "bf16").cpu().numpy(), y0)
    r1 = gb.risk(pf, n_scen=2048, method="surrogate", surrogate=net, surrogate_precision="bf16")
    assert r1["var"] == pytest.approx(r0["var"], rel=1e-6) and r1["cvar"] == pytest.approx(r0["cvar"], rel=1e-6)
    l1, g1 = net.loss_grad(x[:2048], t[:2048])
    assert l1 == pytest.approx(l0, rel=1e-6)
    assert np.max(np.abs(g1 - g0)) <= 1e-5 * np.max(np.abs(g0))
    d1, gr1 = net.loss_grad_d(x[:2048], t[:2048], gd[:2048], [0, 1], [1.0, 1.0], [0.5, 0.5])
    assert np.allclose(d1, d0, rtol=1e-6, atol=0)
    assert np.max(np.abs(gr1 - gr0)) <= 1e-5 * np.max(np.abs(gr0))
    net.close()
