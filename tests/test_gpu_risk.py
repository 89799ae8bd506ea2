"""GPU parity of portfolio risk (mc_risk) and of the surrogate's labels with
the FP64 oracle on identical streams; exactness of the VaR / CVaR selection;
the trained surrogate measured against nested Monte Carlo, and what it gains."""
import math
import time

import numpy as np
import pytest

import workloads
from oracle import risk as orisk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def test_labels_match_oracle(gb, orc):
    import torch
    pts = workloads.surrogate_points(96, seed=11)
    pts[:48, 4] = 0.0  # European half
    got = gb.surrogate_labels(torch.from_numpy(pts).cuda(), 1024).cpu().numpy()
    want = orisk.labels(pts.astype(np.float64), 1024)
    euro = pts[:, 4] == 0
    rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-3)
    print("label rel err: european max %.2e, barrier max %.2e" % (rel[euro].max(), rel[~euro].max()))
    assert np.all(rel[euro] <= 2e-5)
    # barrier labels: a path whose running maximum lies within FP32 rounding of
    # H may knock out on one side only; one flip moves a label by <= 1/1024 * (S_max - K)
    assert np.all(np.abs(got - want)[~euro] <= 2e-5 * np.abs(want[~euro]) + 2.0 / 1024)


def _small_portfolio():
    return workloads.risk_portfolio(n_under=4, per_under=8, seed=7)


def _oracle_pnl(pf, nscen, inner, base_paths):
    S = orisk.scenarios(pf["s0"], pf["sigma"], pf["corr"], pf["mu"], pf["horizon"], nscen)
    steps = np.rint(pf["maturity"] * 252).astype(np.int32)
    rem = steps - 1
    base = orisk.option_values(pf["s0"], pf["sigma"], pf["r"], 1 / 252, 1, -1, pf["under"], pf["kind"],
                               pf["strike"], pf["barrier"], rem, base_paths)
    pnl = np.empty(nscen)
    vals = []
    for s in range(nscen):
        V = orisk.option_values(S[s], pf["sigma"], pf["r"], 1 / 252, 1, s, pf["under"], pf["kind"], pf["strike"],
                                pf["barrier"], rem, inner)
        vals.append(V)
        pnl[s] = pf["position"] @ (V - base)
    return pnl, np.array(vals), base


def test_nested_pnl_matches_oracle(gb, orc):
    pf = _small_portfolio()
    ns, inner, bp = 24, 1024, 4096
    got = gb.risk(pf, alpha=0.9, n_scen=ns, method="nested", inner_paths=inner, base_paths=bp, want_pnl=True)
    pnl, vals, base = _oracle_pnl(pf, ns, inner, bp)
    scale = np.abs(pf["position"]) @ np.abs(vals).max(axis=0)  # sum of |V| over the options
    err = np.abs(got["pnl"] - pnl)
    print("nested PnL max abs err %.3e, scale %.3e" % (err.max(), scale))
    # FP32 inner paths vs FP64: <= 2e-5 of the book's gross value, plus barrier flips
    # (a knock decision within rounding of H moves one option by <= (H - K) / inner)
    flip = np.max(np.where(pf["kind"] == 4, pf["barrier"] - pf["strike"], 0)) / inner
    assert np.all(err <= 2e-5 * scale + 4 * flip)
    assert abs(got["base_value"] - pf["position"] @ base) <= 2e-5 * (np.abs(pf["position"]) @ np.abs(base)) + 4 * flip
    # Sec. VI.B: reduced precision moves VaR / CVaR by less than 1 % against
    # double precision; here FP32 paths against the FP64 oracle on the same
    # scenarios and inner paths
    var_o, cvar_o, _ = orisk.var_cvar(pnl, 0.9)
    print("VaR rel diff %.2e, CVaR rel diff %.2e" % (abs(got["var"] - var_o) / abs(var_o),
                                                     abs(got["cvar"] - cvar_o) / abs(cvar_o)))
    assert abs(got["var"] - var_o) <= 1e-2 * abs(var_o) and abs(got["cvar"] - cvar_o) <= 1e-2 * abs(cvar_o)


def test_var_cvar_selection_is_exact(gb):
    pf = _small_portfolio()
    for alpha, ns in [(0.99, 1000), (0.95, 4096), (0.5, 3)]:
        got = gb.risk(pf, alpha=alpha, n_scen=ns, method="nested", inner_paths=256, base_paths=1024, want_pnl=True)
        var, cvar, nt = orisk.var_cvar(got["pnl"], alpha)
        assert got["var"] == var and got["n_tail"] == nt
        assert abs(got["cvar"] - cvar) <= 1e-12 * abs(cvar)


@pytest.fixture(scope="module")
def trained(gb):
    """A surrogate trained on GPU Monte Carlo labels (2^18 points, 2^11 paths
    each: a reduced version of the 2^20-label training)."""
    import torch
    pts = torch.from_numpy(workloads.surrogate_points(1 << 18)).cuda()
    lab, x = gb.surrogate_labels(pts, 2048, with_inputs=True)
    net = gb.Mlp(5, 256, 4, workloads.mlp_init())
    for lr, ep in workloads.SURROGATE_SCHEDULE:
        loss = net.train(x, lab, epochs=ep, batch=4096, lr=lr)
    print("surrogate final epoch loss %.3e" % loss)
    return net, loss


def test_surrogate_against_nested(gb, trained):
    """The trained surrogate's VaR / CVaR against nested Monte Carlo (the
    yardstick) on the same 2048 scenarios of the full 1024-option book, and the
    time each revaluation takes."""
    import torch
    net, loss = trained
    pf = workloads.risk_portfolio()
    ns = 2048
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nested = gb.risk(pf, n_scen=ns, method="nested", inner_paths=1 << 12, base_paths=1 << 16, want_pnl=True)
    t1 = time.perf_counter()
    sur = gb.risk(pf, n_scen=ns, method="surrogate", surrogate=net, want_pnl=True)
    t2 = time.perf_counter()
    rv = abs(sur["var"] - nested["var"]) / abs(nested["var"])
    rc = abs(sur["cvar"] - nested["cvar"]) / abs(nested["cvar"])
    corr = np.corrcoef(sur["pnl"], nested["pnl"])[0, 1]
    print(f"VaR nested {nested['var']:.3f} surrogate {sur['var']:.3f} (rel {rv:.3%}); "
          f"CVaR nested {nested['cvar']:.3f} surrogate {sur['cvar']:.3f} (rel {rc:.3%}); "
          f"PnL corr {corr:.4f}; time nested {t1 - t0:.3f}s surrogate {t2 - t1:.3f}s")
    # Reduced training (2^18 points, 2^11-path labels) and a 2048-scenario
    # yardstick with 2^12 inner paths (its own PnL noise is ~5 on a PnL standard
    # deviation of ~26): VaR / CVaR within 15 %; the full-size run
    # (2^20 labels x 2^13 paths, risk_report) lands within 3 %.
    assert corr > 0.93
    assert rv < 0.15 and rc < 0.15
    assert t2 - t1 < t1 - t0  # the network revalues faster than the inner simulation


def test_scenario_shards_reproduce_the_full_run(gb, trained):
    """Scenarios are indexed globally: two slices [0, n1) and [n1, n) revalue
    exactly the PnL of the single run (nested and surrogate), and the tail
    statistics of the gathered PnL are the single run's."""
    from paper_1906_02818_gb300 import shard
    net, _ = trained
    pf = workloads.risk_portfolio(n_under=4, per_under=8, seed=7)
    n, n1 = 777, 300
    for kw in (dict(method="nested", inner_paths=256, base_paths=1024),
               dict(method="surrogate", surrogate=net), dict(method="surrogate", surrogate=net,
                                                              surrogate_precision="bf16")):
        full = gb.risk(pf, alpha=0.97, n_scen=n, want_pnl=True, **kw)
        a = gb.risk(pf, alpha=0.97, n_scen=n1, want_pnl=True, **kw)
        b = gb.risk(pf, alpha=0.97, n_scen=n - n1, scen_offset=n1, want_pnl=True, **kw)
        pnl = np.concatenate([a["pnl"], b["pnl"]])
        assert np.array_equal(pnl, full["pnl"]), kw["method"]
        var, cvar, nt = shard.tail_statistics(pnl, 0.97)
        assert var == full["var"] and nt == full["n_tail"] and abs(cvar - full["cvar"]) <= 1e-12 * abs(cvar)


def test_device_tail_selection_matches_oracle_rule(gb):
    """mc_tail (the device VaR / CVaR selection used by mc_risk and by the
    sharded risk path) against the oracle's rule, with ties on purpose and
    sizes that are not powers of two."""
    import torch
    from oracle import risk as orisk
    rng = np.random.default_rng(1)
    for n, alpha in [(1, 0.99), (3, 0.5), (1000, 0.99), (4096, 0.95), (65536, 0.99), (100_003, 0.975)]:
        pnl = np.round(rng.standard_normal(n) * 10.0, 1)
        got = gb.tail(torch.from_numpy(pnl).cuda(), alpha)
        var, cvar, nt = orisk.var_cvar(pnl, alpha)
        assert got["var"] == var and got["n_tail"] == nt, (n, alpha, got, var, nt)
        assert abs(got["cvar"] - cvar) <= 1e-12 * max(1.0, abs(cvar))


def test_label_greeks_match_oracle(gb, orc):
    """Pathwise delta and vega labels (mc_surrogate_label_greeks) against the
    FP64 oracle on the same paths: the labels themselves unchanged (to an
    FP32 rounding); each
    Greek within 2e-5 relative plus the change of the oracle's own Greek
    under a 2e-5 relative move of S/K (the paths whose S_T lies that close to
    K may take the other side of the payoff's kink in FP32); barrier points
    NaN."""
    import torch
    pts = workloads.surrogate_points(96, seed=11)
    pts[:48, 4] = 0.0
    lab, dl = gb.surrogate_label_greeks(torch.from_numpy(pts).cuda(), 1024)
    lab, dl = lab.cpu().numpy(), dl.cpu().numpy()
    plain = gb.surrogate_labels(torch.from_numpy(pts).cuda(), 1024).cpu().numpy()
    assert np.max(np.abs(lab - plain)) <= 1e-6 * np.max(np.abs(plain))  # same paths (the compiler may fuse differently)
    p64 = pts.astype(np.float64)
    ref = orisk.label_greeks(p64, 1024)
    euro = pts[:, 4] == 0
    assert np.all(np.isnan(dl[~euro])) and np.all(np.isnan(ref[~euro]))
    band = np.zeros((96, 2))
    for sgn in (1.0, -1.0):
        q = p64.copy()
        q[:, 0] *= 1.0 + sgn * 2e-5
        band = np.maximum(band, np.abs(orisk.label_greeks(q, 1024)[:, [2, 4]] - ref[:, [2, 4]]))
    for col, k in ((2, 0), (4, 1)):
        err = np.abs(dl[euro, k] - ref[euro, col])
        tol = 2e-5 * np.abs(ref[euro, col]) + band[euro, k] + 1e-7
        print("label greek %d: max err %.2e, max err / tol %.3f" % (k, err.max(), np.max(err / tol)))
        assert np.all(err <= tol)


def test_greek_trained_surrogate_beats_nested_at_a_fraction_of_the_time(gb):
    """What the network gains over plain nested Monte Carlo (Sec. VI.B's
    portfolio revaluation), at equal accuracy.  A surrogate trained by the
    library's kernels on GPU Monte Carlo prices and pathwise Greeks (the
    portfolio workload's 2^20 points of the parameter box, 2^13 paths each;
    delta and vega labels on the European half; BF16 inference) revalues the
    1024-option book on 16384 scenarios.  The yardstick is nested Monte
    Carlo with 2^14 inner paths on the same scenarios.  Against it the
    surrogate must beat nested Monte Carlo with 2^12 inner paths: a smaller
    per-scenario PnL error (nested's taken against the exact revaluation:
    its error against the 2^14-path run, whose first 2^12 paths it shares,
    over sqrt(1 - 2^12 / 2^14)), smaller 99 % VaR and CVaR errors, both below
    2 %, and a revaluation at least 20 times faster."""
    import torch
    pts = torch.from_numpy(workloads.surrogate_points(1 << 20, seed=31)).cuda()
    lab, dl, x = gb.surrogate_label_greeks(pts, 1 << 13, with_inputs=True)
    net = gb.Mlp(5, 256, 4, workloads.mlp_init(seed=5))
    dirs, scales, weights = [0, 1], [1.0 / 0.55, 1.0 / 0.15], [0.2, 0.05]
    for lr, ep in workloads.SURROGATE_SCHEDULE:
        net.train_d(x, lab, dl, dirs, scales, weights, epochs=ep, batch=4096, lr=lr)
    pf = workloads.risk_portfolio()
    ns = 1 << 14

    def timed(**kw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = gb.risk(pf, n_scen=ns, want_pnl=True, base_paths=1 << 16, **kw)
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    ref, _ = timed(method="nested", inner_paths=1 << 14)
    n12, t12 = timed(method="nested", inner_paths=1 << 12)
    gb.risk(pf, n_scen=ns, method="surrogate", surrogate=net, surrogate_precision="bf16")  # warm-up (weight image)
    sur, ts = timed(method="surrogate", surrogate=net, surrogate_precision="bf16")
    rmse = lambda r: float(np.sqrt(np.mean((r["pnl"] - ref["pnl"]) ** 2)))  # noqa: E731
    rel = lambda a, key: abs(a[key] - ref[key]) / abs(ref[key])  # noqa: E731
    e12, es = rmse(n12) / np.sqrt(1.0 - 0.25), rmse(sur)
    print(f"PnL RMSE vs nested 2^14: surrogate {es:.3f}, nested 2^12 {e12:.3f} (exact-corrected); "
          f"VaR err surrogate {rel(sur, 'var'):.2%} nested 2^12 {rel(n12, 'var'):.2%}; "
          f"CVaR err surrogate {rel(sur, 'cvar'):.2%} nested 2^12 {rel(n12, 'cvar'):.2%}; "
          f"time surrogate {ts * 1e3:.1f} ms, nested 2^12 {t12 * 1e3:.1f} ms")
    assert es < e12
    assert rel(sur, "var") < rel(n12, "var") and rel(sur, "cvar") < rel(n12, "cvar")
    assert rel(sur, "var") < 0.02 and rel(sur, "cvar") < 0.02
    assert ts * 20 < t12
    net.close()
