"""Throughput and accuracy of every workload on one GPU (one JSON line per
workload): path-steps/s and priced options/s at the run's standard error,
the error against the FP64 oracle on the same random stream (on a path
prefix the oracle finishes quickly), and the oracle's own throughput on the
host cores.

  python tests/workload_report.py [--only gbm1d,bridge,basket64,mlmc,qmc,heston,basket512,risk]
         [--reps 20] [--oracle-paths N]

Device times are CUDA events around mc_plan_execute (inputs resident, the
set-up excluded); Greeks and risk are timed around the whole call.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))  # repository root
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))  # tests/ (closed forms)


def _events(torch, stream, fn, reps, warmup=3):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with torch.cuda.stream(stream):
        for s, e in ev:
            s.record(stream)
            fn()
            e.record(stream)
    torch.cuda.synchronize()
    return float(np.median([s.elapsed_time(e) for s, e in ev])) * 1e-3


def _plan_time(torch, gb, model, cfg, pays, reps):
    stream = torch.cuda.Stream()
    plan = gb.Plan(model, cfg, pays, stream=stream)
    out = torch.empty((len(pays), 2), dtype=torch.float64, device="cuda")
    t = _events(torch, stream, lambda: plan.execute(out, stream=stream), reps)
    res = out.cpu().numpy()
    plan.close()
    return t, res


def _rel(a, b):
    return float(abs(a - b) / max(abs(b), 1e-12))


def run_gbm1d(torch, gb, orc, a):
    import workloads
    w = workloads.gbm_1d()
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], r=w["r"])
    cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"])
    t, res = _plan_time(torch, gb, model, cfg, w["payoffs"], a.reps)
    t0 = time.perf_counter()
    ref = orc.gbm_payoffs(100.0, 0.2, 0.05, 1.0, 64, w["paths"], w["payoffs"])
    t_orc = time.perf_counter() - t0
    m, se = orc.mean_se(ref[0])
    from math import erf, exp, log, sqrt
    N = lambda x: 0.5 * (1 + erf(x / sqrt(2)))
    d1 = (log(1.0) + 0.07) / 0.2
    bs = 100 * N(d1) - 100 * exp(-0.05) * N(d1 - 0.2)
    ps = w["paths"] * w["steps"]
    return dict(workload="1-D GBM call, 2^20 paths x 64 log-Euler steps", dtype="f32", seconds=t,
                path_steps_per_s=ps / t, options_per_s=1 / t, price=float(res[0, 0]), std_err=float(res[0, 1]),
                oracle_price=m, rel_err_vs_oracle=_rel(res[0, 0], m), black_scholes=bs,
                bs_diff_in_se=float(abs(res[0, 0] - bs) / res[0, 1]),
                oracle_path_steps_per_s=ps / t_orc, oracle_sample="all 2^20 paths")


def run_bridge(torch, gb, orc, a):
    """The paper's "In and Out Put" (Sec. VI.A.1) with Brownian-bridge
    monitoring: S0 100, K 120, H 140, r 0.03, sigma 0.8, T 2; 2^22 paths."""
    model = dict(kind="gbm", s0=np.array([100.0]), sigma=np.array([0.8]), r=0.03)
    pays = [dict(kind="ui_put", strike=120.0, barrier=140.0)]
    out = dict(workload="up-and-in put, Brownian-bridge monitoring, 2^22 paths", paper_value=23.1371783926, steps={})
    for steps in (25, 100):
        cfg = dict(steps=steps, T=2.0, paths=1 << 22, seed=42, monitoring="bridge")
        t, res = _plan_time(torch, gb, model, cfg, pays, a.reps)
        disc, = gb.price(model, dict(cfg, monitoring="discrete"), pays)
        n_or = a.oracle_paths or (1 << 14)
        t0 = time.perf_counter()
        ref = orc.gbm1d_bridge_payoffs(100.0, 0.8, 0.03, 2.0, steps, n_or, pays)[0]
        t_orc = time.perf_counter() - t0
        small, = gb.price(model, dict(cfg, paths=n_or), pays)
        out["steps"][steps] = dict(seconds=t, path_steps_per_s=(1 << 22) * steps / t, price=float(res[0, 0]),
                                   std_err=float(res[0, 1]),
                                   diff_from_paper_in_se=float((res[0, 0] - 23.1371783926) / res[0, 1]),
                                   discrete_monitoring_price=disc[0],
                                   rel_err_vs_oracle_prefix=_rel(small[0], ref.mean()), oracle_prefix_paths=n_or,
                                   oracle_path_steps_per_s=n_or * steps / t_orc)
    return out


def run_basket64(torch, gb, orc, a):
    import workloads
    w = workloads.basket_d64()
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
    n_or = a.oracle_paths or 4096
    t0 = time.perf_counter()
    ref = orc.gbm_payoffs(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], n_or, w["payoffs"], corr=w["corr"],
                          weights=w["weights"])
    t_orc = time.perf_counter() - t0
    out = dict(workload="basket d=64, 2^18 paths x 252 steps, call + up-and-out call", precisions={})
    for prec in ("fp32", "bf16", "fp16", "fp8"):
        cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"], precision=prec)
        t, res = _plan_time(torch, gb, model, cfg, w["payoffs"], a.reps)
        small = gb.price(model, dict(cfg, paths=n_or), w["payoffs"])
        errs = [_rel(small[i][0], orc.mean_se(ref[i])[0]) for i in range(2)]
        out["precisions"][prec] = dict(seconds=t, path_steps_per_s=w["paths"] * w["steps"] / t,
                                       options_per_s=2 / t, prices=res[:, 0].tolist(), std_err=res[:, 1].tolist(),
                                       rel_err_vs_oracle_prefix=errs)
    out["oracle_prefix_paths"] = n_or
    out["oracle_path_steps_per_s"] = n_or * w["steps"] / t_orc
    return out


def run_mlmc(torch, gb, orc, a):
    """Two-level precision estimator on the d = 64 workload: reduced-precision
    coarse level on 2^18 paths plus the FP32 - reduced correction on 2^14."""
    import workloads
    w = workloads.basket_d64()
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
    base = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"])
    fp32 = gb.price(model, base, w["payoffs"])
    out = dict(workload="basket d=64, 2^18 coarse + 2^14 correction paths", fp32=[list(r) for r in fp32], precisions={})
    for prec in ("fp8", "bf16"):
        gb.price_mlmc(model, dict(base, precision=prec), w["payoffs"], 1 << 14)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = gb.price_mlmc(model, dict(base, precision=prec), w["payoffs"], 1 << 14)
        t = time.perf_counter() - t0
        out["precisions"][prec] = dict(
            wall_seconds=t,
            payoffs=[dict(coarse=r["coarse"], correction=r["correction"], two_level=(r["price"], r["se"]),
                          coarse_bias_vs_fp32=r["coarse"][0] - f[0],
                          two_level_minus_fp32_in_corr_se=(r["price"] - f[0]) / r["correction"][1],
                          plain_se_at_2e14=r["ref_level"][1]) for r, f in zip(res, fp32)])
    return out


def run_qmc(torch, gb, orc, a):
    """Randomised Sobol QMC vs Philox Monte Carlo on the 16-asset one-step
    basket call (Sec. VI.D): standard error and time at equal point counts."""
    import workloads
    s0, sg, corr = workloads.basket_market(16, 4)
    w = np.full(16, 1.0 / 16)
    model = dict(kind="gbm", s0=s0, sigma=sg, corr=corr, weights=w, r=0.05)
    pays = [dict(kind="call", strike=float(w @ s0))]
    out = dict(workload="16-asset basket call, one step, randomised Sobol (32 dims) vs Philox", points={})
    for m in (12, 16, 20):
        cfg = dict(steps=1, T=1.0, paths=1 << m, seed=42)
        gb.price_qmc(model, cfg, pays, replications=16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (q,), _ = gb.price_qmc(model, cfg, pays, replications=16)
        tq = time.perf_counter() - t0
        t0 = time.perf_counter()
        (mc,) = gb.price(model, dict(cfg, paths=16 << m), pays)
        tm = time.perf_counter() - t0
        out["points"][m] = dict(qmc=q, qmc_seconds=tq, mc_same_total_points=mc, mc_seconds=tm,
                                se_ratio_mc_over_qmc=mc[1] / q[1])
    return out


def run_heston(torch, gb, orc, a):
    import workloads
    w = workloads.heston()
    model = dict(kind="heston", **w["model"])
    cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"])
    t, res = _plan_time(torch, gb, model, cfg, w["payoffs"], a.reps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, g = gb.greeks(model, cfg, w["payoffs"])
    t_g = time.perf_counter() - t0
    n_or = a.oracle_paths or (1 << 14)
    t0 = time.perf_counter()
    ref = orc.heston_payoffs(w["model"], w["T"], w["steps"], n_or, w["payoffs"])
    t_orc = time.perf_counter() - t0
    small = gb.price(model, dict(cfg, paths=n_or), w["payoffs"])
    errs = [_rel(small[i][0], orc.mean_se(ref[i])[0]) for i in range(len(w["payoffs"]))]
    gref = orc.heston_greeks(w["model"], w["T"], w["steps"], min(n_or, 4096), w["payoffs"][:1])[0]
    _, gs = gb.greeks(model, dict(cfg, paths=min(n_or, 4096)), w["payoffs"][:1])
    gerr = [float(abs(gs[0, k, 0] - gref[k].mean()) / max(abs(gref[k].mean()), 1e-2)) for k in range(7)]
    ps = w["paths"] * w["steps"]
    from closed_forms import heston_call
    h = w["model"]
    semi = {}
    for i, K in enumerate(workloads.HESTON_STRIKES):
        cf = heston_call(h["s0"], K, h["r"], w["T"], h["v0"], h["kappa"], h["theta"], h["xi"], h["rho"])
        semi[str(int(K))] = dict(gpu=float(res[i, 0]), se=float(res[i, 1]), semi_closed_form=cf,
                                 euler_bias_in_se=float((res[i, 0] - cf) / res[i, 1]))
    return dict(workload="Heston, 2^22 paths x 256 steps, 9 strikes x {European, Asian}", dtype="f32",
                european_vs_semi_closed_form=semi,
                seconds=t, path_steps_per_s=ps / t, options_per_s=18 / t,
                max_rel_err_vs_oracle_prefix=max(errs), oracle_prefix_paths=n_or,
                greeks_seconds=t_g, greeks_path_steps_per_s=ps / t_g,
                greeks_call80=dict(zip(("delta", "vega_v0", "rho", "kappa", "theta", "xi", "rho_corr"),
                                       [float(v) for v in g[0, :, 0]])),
                greek_rel_err_vs_oracle_4096=dict(zip(("delta", "vega_v0", "rho", "kappa", "theta", "xi", "rho_corr"),
                                                      gerr)),
                oracle_path_steps_per_s=n_or * w["steps"] / t_orc)


def run_basket512(torch, gb, orc, a):
    import workloads
    w = workloads.basket_d512()
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
    n_or = a.oracle_paths or 1024
    t0 = time.perf_counter()
    ref = orc.gbm_payoffs(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], n_or, w["payoffs"], corr=w["corr"],
                          weights=w["weights"])
    t_orc = time.perf_counter() - t0
    m_or, se_or = orc.mean_se(ref[0])
    out = dict(workload="basket d=512, 2^20 paths x 252 steps, ATM call + 512-delta", precisions={},
               oracle_prefix_paths=n_or, oracle_path_steps_per_s=n_or * w["steps"] / t_orc)
    wf = workloads.basket_d512_factor()
    fmodel = dict(kind="gbm", s0=wf["s0"], sigma=wf["sigma"], loadings=wf["loadings"], weights=wf["weights"], r=wf["r"])
    fcfg = dict(steps=wf["steps"], T=wf["T"], paths=wf["paths"], seed=wf["seed"])
    t, res = _plan_time(torch, gb, fmodel, fcfg, wf["payoffs"], a.reps)
    fref = orc.gbm_factor_payoffs(wf["s0"], wf["sigma"], wf["loadings"], wf["r"], wf["T"], wf["steps"], n_or,
                                  wf["payoffs"], weights=wf["weights"])
    fsmall = gb.price(fmodel, dict(fcfg, paths=n_or), wf["payoffs"])
    out["factor_model_fp32"] = dict(seconds=t, path_steps_per_s=wf["paths"] * wf["steps"] / t, price=float(res[0, 0]),
                                    std_err=float(res[0, 1]), rel_err_vs_oracle_prefix=_rel(fsmall[0][0], fref[0].mean()))
    for prec in ("bf16", "fp8", "fp16", "fp32"):
        cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"], precision=prec)
        reps = a.reps if prec != "fp32" else 1
        t, res = _plan_time(torch, gb, model, cfg, w["payoffs"], reps)
        small = gb.price(model, dict(cfg, paths=n_or), w["payoffs"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, g = gb.greeks(model, dict(cfg, paths=w["paths"] if prec != "fp32" else 1 << 16), w["payoffs"])
        t_g = time.perf_counter() - t0
        out["precisions"][prec] = dict(seconds=t, path_steps_per_s=w["paths"] * w["steps"] / t, price=float(res[0, 0]),
                                       std_err=float(res[0, 1]), rel_err_vs_oracle_prefix=_rel(small[0][0], m_or),
                                       greeks_seconds=t_g, delta_sum=float(g[0, :512, 0].sum()))
    return out


def run_risk(torch, gb, orc, a):
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(os.path.abspath(__file__)), "risk_report.py"), "--scen", str(1 << 16)],
                       capture_output=True, text=True,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    return json.loads(r.stdout.strip().splitlines()[-1])


def main():
    import torch

    import oracle
    import paper_1906_02818_gb300 as gb
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="gbm1d,bridge,basket64,mlmc,qmc,heston,basket512,risk")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--oracle-paths", type=int, default=0)
    a = ap.parse_args()
    oracle.build()
    runs = dict(gbm1d=run_gbm1d, bridge=run_bridge, basket64=run_basket64, mlmc=run_mlmc, qmc=run_qmc,
                heston=run_heston, basket512=run_basket512, risk=run_risk)
    for name in a.only.split(","):
        out = runs[name](torch, gb, oracle, a)
        out["name"] = name
        out["host_cores"] = os.cpu_count()
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
