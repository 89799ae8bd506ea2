"""The allocation-free single-asset pricer (mc_price_gbm1d_noalloc), for
callers that cannot call cudaMalloc: through the C ABI it must reproduce the
regular entry point (mc_price) within the pricing tolerance, on two calls in
a row (the second call reuses the library's fixed scratch array left behind
by the first).  This file is collected last on purpose."""
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


def test_noalloc_rejects_out_of_range():
    from paper_1906_02818_gb300 import api, native
    L = native.lib()
    pays = [dict(kind="call", strike=100.0)] * 33
    mm = api._Marshalled(dict(kind="gbm", s0=[100.0], sigma=[0.2], r=0.05), dict(steps=4, T=1.0, paths=10), pays)
    rc = L.mc_price_gbm1d_noalloc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, 33,
                                  ctypes.c_void_p(16), None)
    assert rc == native.MC_EINVAL
    assert b"n_payoff" in L.mc_last_error()
