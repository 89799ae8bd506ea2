"""The C-ABI library builds, loads without a GPU, exports every entry point
include/mc.h declares, and rejects bad arguments on the host (these checks run
before any CUDA call, so they need no device)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mc_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_02818_gb300 import native
    return native.lib()


def test_exports_every_declared_symbol(lib):
    from paper_1906_02818_gb300 import native
    names = declared_functions()
    assert "mc_price" in names and "mc_simulate" in names
    for n in names:
        assert hasattr(lib, n), n
    # the binding marshals exactly the declared surface
    assert sorted(s[0] for s in native.SIGNATURES) == names


def test_version_and_error_string(lib):
    assert lib.mc_version() == 10000
    assert isinstance(lib.mc_last_error(), bytes)


def _structs(kind="gbm", d=1, **over):
    from paper_1906_02818_gb300 import api
    if kind == "gbm":
        model = dict(kind="gbm", s0=np.full(d, 100.0), sigma=np.full(d, 0.2), r=0.05)
    else:
        model = dict(kind="heston", s0=100.0, v0=0.04, r=0.05, kappa=2.0, theta=0.04, xi=0.5, rho=-0.7)
    model.update({k: v for k, v in over.items()
                  if k in ("s0", "sigma", "corr", "weights", "r", "rho", "xi", "v0", "loadings")})
    cfg = dict(steps=4, T=1.0, paths=16)
    cfg.update({k: v for k, v in over.items()
                if k in ("steps", "T", "paths", "scheme", "precision", "path_offset", "monitoring")})
    pays = over.get("payoffs", [dict(kind="call", strike=100.0)])
    return api._Marshalled(model, cfg, pays)


@pytest.mark.parametrize("over,needle", [
    (dict(steps=0), "steps"),
    (dict(T=-1.0), "T must"),
    (dict(paths=0), "paths"),
    (dict(path_offset=-1), "path range"),
    (dict(s0=np.array([-1.0])), "s0[0]"),
    (dict(sigma=np.array([np.nan])), "sigma[0]"),
    (dict(payoffs=[dict(kind="call", strike=float("nan"))]), "strike"),
    (dict(d=2, corr=np.array([[1.0, 0.5], [0.4, 1.0]])), "symmetric"),
    (dict(d=2, corr=np.array([[2.0, 0.5], [0.5, 1.0]])), "unit diagonal"),
])
def test_price_rejects_bad_arguments_on_host(lib, over, needle):
    from paper_1906_02818_gb300 import native
    mm = _structs(**over)
    out = (native.McResult * 1)()
    rc = lib.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out, None)
    assert rc == native.MC_EINVAL
    assert needle in lib.mc_last_error().decode()


@pytest.mark.parametrize("over,needle", [
    (dict(sigma=np.full(3, 0.2)), "sigma"),
    (dict(corr=np.eye(3)), "corr"),
    (dict(weights=np.full(5, 0.25)), "weights"),
    (dict(loadings=np.full((2, 4), 0.3)), "loadings"),
    (dict(loadings=np.full(6, 0.3)), "loadings"),
])
def test_binding_checks_array_sizes(over, needle):
    """The library reads d, d x d or d x k doubles through the model's
    pointers; the binding refuses arrays of other sizes before any call."""
    with pytest.raises(ValueError, match=needle):
        _structs(d=4, **over)
    _structs(d=4, loadings=np.full((4, 2), 0.3))  # [d, k] passes
    _structs(d=4, loadings=np.zeros((4, 0)))      # no factors passes


def test_heston_argument_checks(lib):
    from paper_1906_02818_gb300 import native
    for over, needle in [(dict(rho=1.0), "rho"), (dict(xi=-0.1), ">= 0"), (dict(precision="bf16"), "precision")]:
        mm = _structs(kind="heston", **over)
        out = (native.McResult * 1)()
        rc = lib.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out, None)
        assert rc == native.MC_EINVAL, over
        assert needle in lib.mc_last_error().decode()


def test_null_and_count_checks(lib):
    from paper_1906_02818_gb300 import native
    mm = _structs()
    out = (native.McResult * 1)()
    assert lib.mc_price(None, ctypes.byref(mm.cfg), mm.payoffs, 1, out, None) == native.MC_EINVAL
    assert lib.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, 33, out, None) == native.MC_EINVAL
    h = ctypes.c_void_p()
    assert lib.mc_plan_create(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, 0,
                              ctypes.byref(h), None) == native.MC_EINVAL
    assert lib.mc_simulate(ctypes.byref(mm.model), ctypes.byref(mm.cfg), 3, ctypes.c_void_p(1), None) == native.MC_EINVAL
    assert lib.mc_plan_execute(None, ctypes.c_void_p(1), None) == native.MC_EINVAL


def test_bridge_monitoring_checks(lib):
    from paper_1906_02818_gb300 import native
    out = (native.McResult * 1)()
    pays = [dict(kind="uo_call", strike=100.0, barrier=130.0)]
    for over, code, needle in [(dict(monitoring="bridge", scheme="euler"), native.MC_EUNSUPPORTED, "bridge"),
                               (dict(d=3, monitoring="bridge"), native.MC_EUNSUPPORTED, "bridge")]:
        mm = _structs(payoffs=pays, **over)
        rc = lib.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out, None)
        assert rc == code, over
        assert needle in lib.mc_last_error().decode().lower()
    mm = _structs(payoffs=pays)
    mm.cfg.monitoring = 7
    rc = lib.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out, None)
    assert rc == native.MC_EINVAL and "monitoring" in lib.mc_last_error().decode()


def test_two_level_estimator_checks(lib):
    from paper_1906_02818_gb300 import native
    out = (native.McMlmcResult * 12)()
    for over, np_, ref, code, needle in [
            (dict(d=4, precision="fp32"), 1, 64, native.MC_EINVAL, "reduced precision"),
            (dict(d=1, precision="bf16"), 1, 64, native.MC_EUNSUPPORTED, "2 <= d"),
            (dict(d=4, precision="bf16"), 11, 64, native.MC_EINVAL, "n_payoff"),
            (dict(d=4, precision="bf16"), 1, 1, native.MC_EINVAL, "paths_ref")]:
        mm = _structs(payoffs=[dict(kind="call", strike=100.0)] * np_, **over)
        rc = lib.mc_price_mlmc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, np_, ref, out, None)
        assert rc == code, (over, np_, ref)
        assert needle in lib.mc_last_error().decode()
    assert lib.mc_price_mlmc(None, None, None, 1, 64, out, None) == native.MC_EINVAL


def test_quasi_monte_carlo_checks(lib):
    from paper_1906_02818_gb300 import native
    out = (native.McResult * 2)()
    for over, reps, code, needle in [(dict(d=33), 8, native.MC_EUNSUPPORTED, "d <= 32"),
                                     (dict(d=4, steps=9), 8, native.MC_EUNSUPPORTED, "Sobol dimensions"),
                                     (dict(d=4), 1, native.MC_EINVAL, "replications"),
                                     (dict(d=4, paths=1 << 23, path_offset=1), 8, native.MC_EINVAL, "2^23"),
                                     (dict(d=4, precision="bf16"), 8, native.MC_EUNSUPPORTED, "FP32")]:
        mm = _structs(**over)
        rc = lib.mc_price_qmc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, reps, out,
                              None, None)
        assert rc == code, over
        assert needle in lib.mc_last_error().decode(), (over, lib.mc_last_error())


def test_factor_model_checks(lib):
    from paper_1906_02818_gb300 import native
    out = (native.McResult * 1)()
    d = 4
    good = np.full((d, 2), 0.5)
    for over, code, needle in [
            (dict(d=d, loadings=good, corr=np.eye(d)), native.MC_EINVAL, "either corr or loadings"),
            (dict(d=d, loadings=np.full((d, 17), 0.1)), native.MC_EUNSUPPORTED, "n_factors"),
            (dict(d=d, loadings=np.full((d, 2), 0.8)), native.MC_EINVAL, "norm"),
            (dict(d=513, loadings=np.full((513, 2), 0.1)), native.MC_EUNSUPPORTED, "exceeds 512"),
            (dict(d=d, loadings=good, precision="bf16"), native.MC_EUNSUPPORTED, "FP32")]:
        mm = _structs(**over)
        rc = lib.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out, None)
        assert rc == code, over
        assert needle in lib.mc_last_error().decode(), (over, lib.mc_last_error())


def test_factor_model_greeks_checks(lib):
    """mc_greeks on a factor model takes one European call or put under
    log-Euler with every sigma > 0; the rest is refused before any device
    work."""
    from paper_1906_02818_gb300 import native
    d = 4
    pr, gr = (native.McResult * 2)(), (native.McResult * (2 * (2 * d + 1)))()
    fm = dict(d=d, loadings=np.full((d, 2), 0.5))
    call = [dict(kind="call", strike=100.0)]
    for over, code, needle in [
            (dict(fm, payoffs=[dict(kind="asian_call", strike=100.0)]), native.MC_EUNSUPPORTED, "European"),
            (dict(fm, payoffs=[dict(kind="uo_call", strike=100.0, barrier=130.0)]), native.MC_EUNSUPPORTED,
             "European"),
            (dict(fm, payoffs=call * 2), native.MC_EUNSUPPORTED, "exactly one"),
            (dict(fm, scheme="euler"), native.MC_EUNSUPPORTED, "log-Euler"),
            (dict(fm, sigma=np.array([0.2, 0.0, 0.3, 0.25])), native.MC_EINVAL, "sigma > 0"),
            (dict(fm, precision="bf16"), native.MC_EUNSUPPORTED, "FP32")]:
        mm = _structs(**over)
        rc = lib.mc_greeks(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, pr, gr, None)
        assert rc == code, over
        assert needle in lib.mc_last_error().decode(), (over, lib.mc_last_error())
    mm = _structs(**fm)
    assert lib.mc_greeks(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, 1, pr, None, None) == native.MC_EINVAL
    assert lib.mc_greek_count(ctypes.byref(mm.model)) == 2 * d + 1


def test_correlation_sensitivity_checks(lib):
    from paper_1906_02818_gb300 import native
    pr, dl, dr = native.McResult(), (native.McResult * 4096)(), (native.McResult * 4096)()
    for over, code, needle in [
            (dict(d=1), native.MC_EUNSUPPORTED, "2 <= d <= 512"),
            (dict(d=513), native.MC_EUNSUPPORTED, "2 <= d <= 512"),
            (dict(d=4, loadings=np.full((4, 2), 0.5)), native.MC_EUNSUPPORTED, "2 <= d <= 512"),
            (dict(d=4, scheme="euler"), native.MC_EUNSUPPORTED, "log-Euler"),
            (dict(d=4, precision="bf16"), native.MC_EUNSUPPORTED, "FP32"),
            (dict(d=65, payoffs=[dict(kind="asian_call", strike=100.0)]), native.MC_EUNSUPPORTED, "Asian"),
            (dict(d=4, payoffs=[dict(kind="uo_put", strike=100.0, barrier=130.0)]), native.MC_EUNSUPPORTED,
             "European"),
            (dict(d=4, payoffs=[dict(kind="uo_call", strike=100.0, barrier=130.0)]), native.MC_EUNSUPPORTED,
             "European"),
            (dict(d=2, corr=np.array([[1.0, 0.5], [0.4, 1.0]])), native.MC_EINVAL, "symmetric")]:
        mm = _structs(**over)
        rc = lib.mc_corr_greeks(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, ctypes.byref(pr), dl, dr,
                                None)
        assert rc == code, over
        assert needle in lib.mc_last_error().decode(), (over, lib.mc_last_error())
    mm = _structs(d=4)
    assert lib.mc_corr_greeks(ctypes.byref(mm.model), ctypes.byref(mm.cfg), None, ctypes.byref(pr), dl, dr,
                              None) == native.MC_EINVAL
    assert lib.mc_corr_greeks(None, None, None, None, None, None, None) == native.MC_EINVAL


def test_release_cache_without_work(lib):
    assert lib.mc_release_cache() == 0


@pytest.mark.parametrize("over,needle", [
    (dict(T=float("inf")), "T must"),
    (dict(s0=np.array([np.inf])), "s0[0]"),
    (dict(sigma=np.array([np.inf])), "sigma[0]"),
    (dict(payoffs=[dict(kind="call", strike=float("nan"))]), "strike"),
    (dict(payoffs=[dict(kind="uo_call", strike=100.0, barrier=float("nan"))]), "barrier"),
    (dict(weights=np.array([np.nan])), "weights"),
    (dict(path_offset=(1 << 56) - 8), "path range"),
    (dict(corr=np.array([[0.5]])), "corr"),
    (dict(d=2), "single-asset"),
])
def test_noalloc_rejects_what_mc_price_rejects(lib, over, needle):
    """The allocation-free pricer applies mc_price's argument checks (and
    its own single-asset restriction) before any CUDA call."""
    from paper_1906_02818_gb300 import native
    mm = _structs(**over)
    rc = lib.mc_price_gbm1d_noalloc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff,
                                    ctypes.c_void_p(16), None)
    assert rc == native.MC_EINVAL, (over, lib.mc_last_error())
    assert needle in lib.mc_last_error().decode()
    for n in (0, 33):
        assert lib.mc_price_gbm1d_noalloc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, n,
                                          ctypes.c_void_p(16), None) == native.MC_EINVAL


def test_rng_entry_points_check_arguments_on_host(lib):
    from paper_1906_02818_gb300 import native
    assert lib.mc_philox_words(42, 0, 0, 0, ctypes.c_void_p(16), None) == native.MC_OK  # empty: no launch
    assert lib.mc_philox_words(42, 0, 0, 4, None, None) == native.MC_EINVAL
    assert lib.mc_philox_words(42, 0, 0, 4, ctypes.c_void_p(20), None) == native.MC_EINVAL
    assert b"aligned" in lib.mc_last_error()
    assert lib.mc_philox_words(42, 0, 0, -1, ctypes.c_void_p(16), None) == native.MC_EINVAL
    assert lib.mc_philox_words(42, 0, (1 << 64) - 2, 4, ctypes.c_void_p(16), None) == native.MC_EINVAL
    assert b"wraps" in lib.mc_last_error()
    assert lib.mc_normals(42, 0, 0, 0, ctypes.c_void_p(16), None) == native.MC_OK
    assert lib.mc_normals(42, 0, (1 << 64) - 2, 4, ctypes.c_void_p(16), None) == native.MC_EINVAL
    assert lib.mc_normals(42, 0, 0, 1 << 41, ctypes.c_void_p(16), None) == native.MC_EINVAL


def test_binding_checks_device_tensors():
    """Network and label calls read float32 device memory through their
    pointers: host tensors, other dtypes and other shapes are refused by the
    binding before any library call (checked here on host tensors)."""
    import torch
    from paper_1906_02818_gb300 import api
    with pytest.raises(ValueError, match="CUDA float32"):
        api._rows(torch.zeros((4, 5)), 5, "x")
    with pytest.raises(ValueError, match="CUDA float32"):
        api._count(np.zeros(4, dtype=np.float32), 4, "t")
    with pytest.raises(ValueError, match="CUDA float32"):
        api.surrogate_labels(torch.zeros((4, 5), dtype=torch.float64), 16)
    with pytest.raises(ValueError, match="holds 3 values, 4 expected"):
        api._host_f32(np.zeros(3), 4, "params")
    assert api._host_f32(np.zeros(4), 4, "params").dtype == np.float32


@pytest.mark.parametrize("key,value", [("sigma", np.full(3, 0.2)), ("corr", np.eye(3)), ("barrier", np.full(5, 1e300)),
                                       ("under", np.zeros(7, dtype=np.int32)), ("position", np.ones(2))])
def test_risk_binding_checks_portfolio_sizes(lib, key, value):
    """mc_risk reads n_under, n_under^2 and n_opt values through the
    portfolio's pointers: arrays of other sizes are refused by the binding."""
    import workloads
    from paper_1906_02818_gb300 import api
    pf = workloads.risk_portfolio(n_under=4, per_under=2)
    pf[key] = value
    with pytest.raises(ValueError, match=key):
        api.risk(pf, n_scen=16)


def _payoff_kind(mm, kind):
    mm.payoffs[0].kind = kind
    return mm


def _set(mm, **fields):
    for obj, name, value in ((mm.model if k.startswith("m_") else mm.cfg, k[2:], v) for k, v in fields.items()):
        setattr(obj, name, value)
    return mm


@pytest.mark.parametrize("make,needle", [
    (lambda: _set(_structs(), m_kind=7), "unknown model kind"),
    (lambda: _set(_structs(), m_d=0), "out of range [1, 4096]"),
    (lambda: _set(_structs(), m_d=5000), "out of range [1, 4096]"),
    (lambda: _set(_structs(), m_s0=None), "s0 is NULL"),
    (lambda: _structs(r=float("inf")), "r is not finite"),
    (lambda: _structs(kind="heston", s0=np.array([100.0, 100.0])), "Heston requires d == 1"),
    (lambda: _set(_structs(kind="heston"), m_kappa=float("nan")), "Heston parameters must be finite"),
    (lambda: _set(_structs(), m_sigma=None), "sigma is NULL"),
    (lambda: _structs(d=4, loadings=np.full((4, 2), np.nan)), "loadings must be finite"),
    (lambda: _structs(d=2, corr=np.array([[1.0, np.nan], [np.nan, 1.0]])), "corr must be finite"),
    (lambda: _structs(d=2, corr=np.array([[1.0, 1.5], [1.5, 1.0]])), "outside [-1, 1]"),
    (lambda: _set(_structs(), c_scheme=5), "unknown scheme"),
    (lambda: _set(_structs(), c_precision=9), "unknown precision"),
    (lambda: _set(_structs(), c_ckpt_every=-1), "ckpt_every must be >= 0"),
    (lambda: _payoff_kind(_structs(), 99), "unknown kind"),
])
def test_model_and_config_checks(lib, make, needle):
    """Every model / configuration / payoff check of mc_price that runs before
    any CUDA call: MC_EINVAL with its message, outputs untouched."""
    from paper_1906_02818_gb300 import native
    mm = make()
    out = (native.McResult * 1)(native.McResult(12345.0, -1.0))
    rc = lib.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out, None)
    assert rc == native.MC_EINVAL, (needle, rc, lib.mc_last_error())
    assert needle in lib.mc_last_error().decode(), (needle, lib.mc_last_error())
    assert out[0].price == 12345.0 and out[0].se == -1.0


def test_null_pointer_checks(lib):
    from paper_1906_02818_gb300 import native
    mm = _structs()
    out = (native.McResult * 1)()
    assert lib.mc_price(ctypes.byref(mm.model), None, mm.payoffs, 1, out, None) == native.MC_EINVAL
    assert "cfg is NULL" in lib.mc_last_error().decode()
    assert lib.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), None, 1, out, None) == native.MC_EINVAL
    assert "payoffs is NULL" in lib.mc_last_error().decode()
    hm = _structs(kind="heston")
    hm.model.corr = hm._ptr(hm._arr(np.eye(1)))
    assert lib.mc_price(ctypes.byref(hm.model), ctypes.byref(hm.cfg), hm.payoffs, 1, out, None) == native.MC_EINVAL
    assert "no correlation" in lib.mc_last_error().decode()


def test_greeks_checks(lib):
    """mc_greeks' own host checks (single-asset, basket and Heston forms)."""
    from paper_1906_02818_gb300 import native
    pr, g = (native.McResult * 2)(), (native.McResult * 64)()
    for mm, gp, code, needle in [
            (_structs(payoffs=[dict(kind="uo_call", strike=100.0, barrier=130.0)]), g, native.MC_EUNSUPPORTED,
             "no pathwise Greek"),
            (_structs(d=3, payoffs=[dict(kind="call", strike=100.0)] * 2), g, native.MC_EINVAL, "exactly one payoff"),
            (_structs(d=3, sigma=np.array([0.2, 0.0, 0.3])), g, native.MC_EINVAL, "sigma > 0"),
            (_structs(scheme="euler"), g, native.MC_EUNSUPPORTED, "log-Euler"),
            (_set(_structs(kind="heston"), c_ckpt_every=100), g, native.MC_EINVAL, "outside [1, 64]"),
            (_structs(), None, native.MC_EINVAL, "greeks is NULL")]:
        rc = lib.mc_greeks(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, pr, gp, None)
        assert rc == code, (needle, rc, lib.mc_last_error())
        assert needle in lib.mc_last_error().decode(), (needle, lib.mc_last_error())


def test_moments_and_combine_checks(lib):
    from paper_1906_02818_gb300 import native
    res = (native.McResult * 1)(native.McResult(float("nan"), 1.0))
    mom = (ctypes.c_double * 3)()
    assert lib.mc_moments(res, 1, 10, mom) == native.MC_EINVAL and "not finite" in lib.mc_last_error().decode()
    bad = (ctypes.c_double * 3)(1.0, 1.0, 0.0)
    out = (native.McResult * 1)()
    assert lib.mc_combine(bad, 1, out) == native.MC_EINVAL and "path count" in lib.mc_last_error().decode()


def test_network_label_tail_and_stream_checks(lib):
    """Host checks of the network, label, tail and random-stream entry points
    (NULL handles and buffers, sizes, ranges), all before any CUDA call."""
    from paper_1906_02818_gb300 import native
    p = ctypes.c_void_p(16)  # never dereferenced: every call below is refused first
    res = native.McRiskResult()
    for call, needle in [
            (lambda: lib.mc_mlp_forward(None, p, 4, p, 0, None), "network is NULL"),
            (lambda: lib.mc_mlp_loss_grad(None, p, p, 4, None, None, None), "network is NULL"),
            (lambda: lib.mc_mlp_train(None, p, p, 4, 1, 1, ctypes.c_float(1e-3), None, None), "network is NULL"),
            (lambda: lib.mc_mlp_apply_grad(None, None, ctypes.c_float(1e-3), None), "network is NULL"),
            (lambda: lib.mc_mlp_create(0, 256, 4, None, ctypes.byref(ctypes.c_void_p())), "n_in in [1,64]"),
            (lambda: lib.mc_mlp_create(5, 256, 4, None, None), "out is NULL"),
            (lambda: lib.mc_surrogate_labels(0, p, 16, 252, 42, p, None, None), "n >= 1"),
            (lambda: lib.mc_surrogate_labels(4, p, 0, 252, 42, p, None, None), "paths must lie in [1, 65536]"),
            (lambda: lib.mc_surrogate_labels(4, p, 16, 0, 42, p, None, None), "steps_per_year"),
            (lambda: lib.mc_surrogate_label_greeks(4, p, 16, 252, 42, p, None, None, None), "dev_dlabels"),
            (lambda: lib.mc_tail(None, 4, ctypes.c_double(0.99), ctypes.byref(res), None), "dev_pnl and result"),
            (lambda: lib.mc_tail(p, 0, ctypes.c_double(0.99), ctypes.byref(res), None), "n outside [1, 2^24]"),
            (lambda: lib.mc_tail(p, 4, ctypes.c_double(1.0), ctypes.byref(res), None), "alpha must lie in (0, 1)"),
            (lambda: lib.mc_philox_words(42, 0, 0, 1 << 41, p, None), "blocks outside [0, 2^40]"),
            (lambda: lib.mc_philox_words(42, 0, (1 << 64) - 2, 4, p, None), "wraps past 2^64"),
            (lambda: lib.mc_normals(42, 0, 0, 1 << 41, p, None), "count outside [0, 2^40]")]:
        rc = call()
        assert rc == native.MC_EINVAL, (needle, rc, lib.mc_last_error())
        assert needle in lib.mc_last_error().decode(), (needle, lib.mc_last_error())
    assert lib.mc_mlp_destroy(None) == 0  # destroying nothing is allowed


class _NullStream:
    cuda_stream = 0  # the default stream's handle, for calls refused before any CUDA work


@pytest.mark.parametrize("over,kw,needle", [
    ({}, dict(n_scen=0), "n_scen outside"),
    ({}, dict(n_scen=16, alpha=1.5), "alpha must lie in (0, 1)"),
    ({"horizon": 1.5 / 252}, dict(n_scen=16), "whole number of steps"),
    ({}, dict(n_scen=16, method="surrogate"), "surrogate network not set"),
    ({}, dict(n_scen=16, inner_paths=0), "inner_paths in [1, 65536]"),
    ({"strike": "zero"}, dict(n_scen=16), "strike must be > 0"),
    ({"maturity": "one day"}, dict(n_scen=16), "whole steps beyond the horizon"),
    ({"s0": "negative"}, dict(n_scen=16), "s0 > 0 and sigma >= 0"),
    ({}, dict(n_scen=16, scen_offset=-1), "scenario range"),
])
def test_risk_checks(lib, over, kw, needle):
    import workloads
    from paper_1906_02818_gb300 import api, native
    pf = workloads.risk_portfolio(n_under=4, per_under=2)
    fill = {"zero": 0.0, "one day": 1 / 252, "negative": -1.0}
    for k, v in over.items():
        pf[k] = np.full_like(pf[k], fill[v]) if isinstance(v, str) else v
    with pytest.raises(native.MCError) as e:
        api.risk(pf, stream=_NullStream(), **kw)
    assert e.value.status == native.MC_EINVAL and needle in str(e.value), str(e.value)


def test_risk_binding_refuses_unknown_kinds(lib):
    import workloads
    from paper_1906_02818_gb300 import api
    pf = workloads.risk_portfolio(n_under=4, per_under=2)
    pf["kind"] = np.full_like(pf["kind"], 2)
    with pytest.raises(ValueError, match="option kinds"):
        api.risk(pf, n_scen=16, stream=_NullStream())
