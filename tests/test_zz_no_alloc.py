"""The allocation-free single-asset pricer (mc_price_gbm1d_noalloc), for
callers that cannot call cudaMalloc: through the C ABI it must reproduce the
regular entry point (mc_price) within the pricing tolerance, on two calls in
a row (the second call reuses the library's fixed scratch array left behind
by the first), and the second call, small enough for the FP64 oracle, must
also match the oracle on the same random stream.  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-5


def test_noalloc_matches_mc_price_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_02818_gb300 import api, native
    L = native.lib()
    pays = [dict(kind="call", strike=100.0), dict(kind="asian_call", strike=100.0),
            dict(kind="uo_call", strike=100.0, barrier=140.0), dict(kind="put", strike=95.0)]
    model = dict(kind="gbm", s0=[100.0], sigma=[0.25], r=0.05)
    for run, cfg in enumerate([dict(steps=64, T=1.0, paths=(1 << 20) + 333, seed=42),
                               dict(steps=37, T=0.5, paths=5000, seed=7, path_offset=123)]):
        want = api.price(model, cfg, pays)
        mm = api._Marshalled(model, cfg, pays)
        out = torch.full((len(pays), 2), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        rc = L.mc_price_gbm1d_noalloc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.mc_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i in range(len(pays)):
            assert abs(got[i, 0] - want[i][0]) <= REL * abs(want[i][0]), (run, pays[i], got[i], want[i])
            assert abs(got[i, 1] - want[i][1]) <= 1e-3 * want[i][1]
        if cfg["paths"] <= 8192:
            # independent of both launch paths: the FP64 oracle on the same
            # path range (path_offset 123); the barrier payoff may differ by
            # the paths whose monitored maximum lies within 2e-5 of H
            import oracle
            ref = oracle.gbm_payoffs(100.0, 0.25, 0.05, cfg["T"], cfg["steps"], cfg["paths"], pays,
                                     seed=cfg["seed"], path_offset=cfg["path_offset"])
            for i, pay in enumerate(pays):
                m, se = oracle.mean_se(ref[i])
                tol = REL * abs(m)
                if pay["kind"] == "uo_call":
                    near = oracle.gbm_payoffs(100.0, 0.25, 0.05, cfg["T"], cfg["steps"], cfg["paths"],
                                              [dict(pay, barrier=pay["barrier"] * (1 - 2e-5)),
                                               dict(pay, barrier=pay["barrier"] * (1 + 2e-5))],
                                              seed=cfg["seed"], path_offset=cfg["path_offset"])
                    tol += float(np.abs(near[1] - near[0]).sum()) / cfg["paths"]
                assert abs(got[i, 0] - m) <= tol, (pay, got[i, 0], m)
                assert abs(got[i, 1] - se) <= 1e-3 * se


def test_noalloc_rejects_out_of_range():
    from paper_1906_02818_gb300 import api, native
    L = native.lib()
    pays = [dict(kind="call", strike=100.0)] * 33
    mm = api._Marshalled(dict(kind="gbm", s0=[100.0], sigma=[0.2], r=0.05), dict(steps=4, T=1.0, paths=10), pays)
    rc = L.mc_price_gbm1d_noalloc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, 33,
                                  ctypes.c_void_p(16), None)
    assert rc == native.MC_EINVAL
    assert b"n_payoff" in L.mc_last_error()
