"""Benchmark of the Monte Carlo hot path.

Headline (the JSON line's `value`): the correlated-basket workload, d = 64
assets (S0 ~ U[50,150], sigma ~ U[0.1,0.4], 4-factor correlation plus
0.05 I), 2^18 paths x 252 log-Euler steps, ATM arithmetic basket call and
up-and-out basket call at 1.3 B(0), Philox4x32-10 stream seed 42, BF16
correlation contraction on the tensor cores with FP32 accumulation and
state.  One step = one mc_plan_execute: RNG + Box-Muller + correlation
contraction + state update + payoffs + reduction over every path (all in the
library's kernels).

At one GPU the same run also measures every other workload (the `configs`
object of the line), each timed with CUDA events, with its results and
standard errors, its error against the FP64 oracle on a path prefix (the
GPU rerun on the same prefix), the oracle's own throughput on the host cores,
and a roofline:
  C1  1-D GBM European call, 2^20 paths x 64 steps
  C2  the headline workload in FP32 (SIMT FMA contraction) and FP16 / E4M3
  C3  Heston, 2^22 paths x 256 steps, 18 options; pathwise Greeks (adjoint)
  C4  portfolio risk: training labels, network training, surrogate and
      nested (2^12 inner paths) revaluation, VaR / CVaR
  C5  d = 512 basket, 2^20 paths x 252 steps: BF16, E4M3, FP32; Greeks

Rooflines.  The path kernels draw their normals with Box-Muller, which needs
lg2, sqrt, sin and cos per pair of normals on the SFU (MUFU) pipe, plus one
ex2 per monitored asset-step; measured on this part, ex2 issues 32 results
per SM per clock and the other four 16.  The SFU roofline of a kernel is the
unit rate at which its algorithmic transcendentals would keep the SFU busy
every cycle: SMs x sm_max_mhz / (SFU cycles per unit).  Contractions are also
reported against the measured tensor peak (MEASURED_PEAKS.json bf16_tflops;
E4M3 at twice that, TF32 at half, the nominal ratios) and the FP32 FMA peak
(SMs x 128 FMA per clock).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|bf16|fp16|fp8] [--configs all|none]
  python bench.py --impl reference   # the FP64 CPU oracle, bounded sample
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "path-steps/s and prices/s at stated std err vs FP64 oracle; roofline fraction"
UNIT = "path-steps/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
WORKLOAD = ("basket d=64 k=4 factors, 2^18 paths x 252 log-Euler steps, ATM basket call + up-and-out call at "
            "1.3 B0, seed 42")

# SFU (MUFU) results per SM per clock on this part (a microbenchmark of
# dependent-free approximate instructions: ex2 32, lg2 / sin / cos / sqrt /
# tanh 16).  Box-Muller: lg2 + sqrt + sin + cos per pair = 2 slow-rate
# results per normal.
SFU_SLOW, SFU_EX2 = 16.0, 32.0
# DRAM bytes (read + write) of one launch of the headline kernel from its ncu
# capture (profiles/basket_tc_bf16_d64_262144paths.md): only the factor tile
# and launch constants are read, whatever the path count.
HEADLINE_DRAM_BYTES = 76288


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.p:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------- rooflines ---------------------------------
class Hw:
    """Peaks of this device: SM count from the device, clocks and measured
    rates from MEASURED_PEAKS.json."""

    def __init__(self, sms: int):
        self.pk, self.kind = peaks()
        self.sms = sms
        self.hz = float(self.pk.get("sm_max_mhz", 2070.0)) * 1e6
        self.bf16 = float(self.pk.get("bf16_tflops", 1900.0)) * 1e12

    def sfu(self, units_per_s, normals=0.0, ex2=0.0, other=0.0, what=""):
        """SFU roofline: normals (2 slow results each), ex2 (fast) and other
        slow results (sqrt, lg2, tanh) per unit."""
        cyc = (2.0 * normals + other) / SFU_SLOW + ex2 / SFU_EX2
        peak = self.sms * self.hz / cyc
        return {"bound": "alu", "pipe": "SFU", "achieved": units_per_s, "peak": peak, "unit": UNIT,
                "frac": units_per_s / peak,
                "basis": f"per unit {what}: {2 * normals + other:g} results at {SFU_SLOW:g}/clk/SM + {ex2:g} ex2 at "
                         f"{SFU_EX2:g}/clk/SM = {cyc:.4g} SM-cycles; peak = {self.sms} SMs x "
                         f"{self.hz / 1e6:g} MHz (sm_max_mhz, {self.kind}) / that"}

    def tensor(self, flops_per_s, dtype="bf16", what=""):
        ratio = {"bf16": 1.0, "fp16": 1.0, "fp8": 2.0, "tf32": 0.5}[dtype]
        peak = self.bf16 * ratio
        return {"bound": "tensor", "achieved": flops_per_s / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": flops_per_s / peak,
                "basis": f"{what}; peak = bf16_tflops ({self.kind}) x {ratio:g} ({dtype}, nominal ratio)"}

    def fma(self, fma_per_s, what=""):
        peak = self.sms * 128 * self.hz
        return {"bound": "alu", "pipe": "FMA", "achieved": fma_per_s / 1e12, "peak": peak / 1e12, "unit": "T FMA/s",
                "frac": fma_per_s / peak,
                "basis": f"{what}; peak = {self.sms} SMs x 128 FP32 FMA/clk x {self.hz / 1e6:g} MHz"}


# --------------------------------- timing ----------------------------------
def time_plan(torch, gb, model, cfg, pays, reps, warmup, flush):
    """Median CUDA-event time (s) of mc_plan_execute on its own stream, L2
    flushed between launches (outside the events); the last results."""
    stream = torch.cuda.Stream()
    plan = gb.Plan(model, cfg, pays, stream=stream)
    out = torch.empty((len(pays), 2), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            plan.execute(out, stream=stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with torch.cuda.stream(stream):
        for s, e in evs:
            flush.fill_(1.0)
            s.record(stream)
            plan.execute(out, stream=stream)
            e.record(stream)
    torch.cuda.synchronize()
    t = float(np.median([s.elapsed_time(e) for s, e in evs])) * 1e-3
    res = out.cpu().numpy()
    plan.close()
    return t, res


def time_call(torch, fn, reps, warmup=1):
    """Median time (s) of a synchronising library call: CUDA events on the
    current stream around it (its work runs on that stream) and wall time."""
    for _ in range(warmup):
        fn()
    ts, walls, r = [], [], None
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.record()
        r = fn()
        e.record()
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
        ts.append(s.elapsed_time(e) * 1e-3)
    return float(np.median(ts)), float(np.median(walls)), r


def _timed_oracle(fn):
    t0 = time.perf_counter()
    r = fn()
    return r, time.perf_counter() - t0


def _prices(res, pays):
    return [{"payoff": p["kind"], "strike": round(float(p["strike"]), 6), "price": float(res[i][0]),
             "std_err": float(res[i][1])} for i, p in enumerate(pays)]


def _errors(orc, got, ref):
    """Per price: GPU minus FP64 oracle on the same paths, relative and in SE."""
    out = []
    for (p, se), row in zip(got, ref):
        m, s = orc.mean_se(row)
        out.append({"gpu": float(p), "oracle": float(m), "rel": float(abs(p - m) / max(abs(m), 1e-12)),
                    "in_se": float(abs(p - m) / s) if s > 0 else None})
    return out


# ------------------------------ the configs --------------------------------
def config_c1(torch, gb, orc, hw, flush, reps):
    w = workloads.gbm_1d()
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], r=w["r"])
    cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"])
    t, res = time_plan(torch, gb, model, cfg, w["payoffs"], reps, 3, flush)
    ref, t_or = _timed_oracle(lambda: orc.gbm_payoffs(100.0, 0.2, 0.05, 1.0, 64, w["paths"], w["payoffs"]))
    from math import erf, exp, sqrt
    N = lambda x: 0.5 * (1 + erf(x / sqrt(2)))  # noqa: E731
    bs = 100 * N(0.35) - 100 * exp(-0.05) * N(0.15)  # Black-Scholes, S0 = K = 100, r .05, sigma .2, T 1
    ps = w["paths"] * w["steps"]
    return {"workload": "1-D GBM European call, S0 = K = 100, r 0.05, sigma 0.2, T 1, 2^20 paths x 64 log-Euler "
                        "steps, FP32, seed 42",
            "value": ps / t, "unit": UNIT, "ms": t * 1e3, "options_per_s": 1 / t, "results": _prices(res, w["payoffs"]),
            "error_vs_oracle": {"paths": w["paths"], "per_price": _errors(orc, [tuple(r) for r in res], ref)},
            "black_scholes": bs, "diff_vs_black_scholes_in_se": float(abs(res[0, 0] - bs) / res[0, 1]),
            "cpu_baseline": {"value": ps / t_or, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "all 2^20 paths x 64 steps"},
            "roofline": hw.sfu(ps / t, normals=1, what="1 normal")}


def config_c2(torch, gb, orc, hw, flush, reps, headline):
    """The headline workload's other contraction precisions, and every
    precision's error against the FP64 oracle on the first 2^14 paths."""
    w = workloads.basket_d64()
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
    base = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"])
    n_or = 1 << 14
    ref, t_or = _timed_oracle(lambda: orc.gbm_payoffs(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], n_or,
                                                      w["payoffs"], corr=w["corr"], weights=w["weights"]))
    ps = w["paths"] * w["steps"]
    d = len(w["s0"])
    out = {"workload": WORKLOAD, "precisions": {},
           "cpu_baseline": {"value": n_or * w["steps"] / t_or, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"first {n_or} of 2^18 paths, all 252 steps"}}
    for prec in ("bf16", "fp32", "fp16", "fp8"):
        c = dict(base, precision=prec)
        if prec == "bf16":
            t, res = headline["s"], headline["res"]
        else:
            t, res = time_plan(torch, gb, model, c, w["payoffs"], reps if prec != "fp32" else max(3, reps // 4), 3,
                               flush)
        small = gb.price(model, dict(c, paths=n_or), w["payoffs"])
        rec = {"value": ps / t, "unit": UNIT, "ms": t * 1e3, "options_per_s": 2 / t,
               "results": _prices(res, w["payoffs"]),
               "error_vs_oracle": {"paths": n_or, "per_price": _errors(orc, small, ref)},
               "roofline": hw.sfu(ps / t, normals=d, ex2=d, what=f"{d} normals + {d} ex2 (monitored basket)")}
        if prec == "fp32":
            rec["roofline_fma"] = hw.fma(ps / t * d * (d + 1) / 2, f"{d * (d + 1) // 2} FMA per path-step "
                                                                     "(triangular contraction)")
        else:
            rec["roofline_tensor"] = hw.tensor(ps / t * d * (d + 1), "fp8" if prec == "fp8" else "bf16",
                                               f"{d * (d + 1)} flop per path-step (triangular contraction)")
        out["precisions"][prec] = rec
    # correlation sensitivities of the ATM basket call on the same paths (FP32)
    tc, _, (cp, _, _) = time_call(torch, lambda: gb.corr_greeks(model, dict(base), w["payoffs"][0]), 3)
    out["corr_greeks"] = {"ms": tc * 1e3, "value": ps / tc, "unit": UNIT, "price": list(cp),
                          "what": f"dP/dLrho and dP/dcorr ({d * (d - 1) // 2} pairs) of the ATM basket call, "
                                  "one mc_corr_greeks call (set-up, path kernel, FP64 Cholesky adjoint per batch)",
                          "roofline": hw.sfu(ps / tc, normals=d, ex2=0, what=f"{d} normals")}
    return out


def config_c3(torch, gb, orc, hw, flush, reps):
    w = workloads.heston()
    model = dict(kind="heston", **w["model"])
    cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"])
    pays = w["payoffs"]
    t, res = time_plan(torch, gb, model, cfg, pays, reps, 3, flush)
    tg, tg_wall, (_, g) = time_call(torch, lambda: gb.greeks(model, cfg, pays), max(2, reps // 4))
    n_or, n_g = 1 << 14, 4096
    ref, t_or = _timed_oracle(lambda: orc.heston_payoffs(w["model"], w["T"], w["steps"], n_or, pays))
    small = gb.price(model, dict(cfg, paths=n_or), pays)
    gref, tg_or = _timed_oracle(lambda: orc.heston_greeks(w["model"], w["T"], w["steps"], n_g, pays[:1])[0])
    _, gs = gb.greeks(model, dict(cfg, paths=n_g), pays[:1])
    names = ("delta", "vega_v0", "rho", "kappa", "theta", "xi", "rho_corr")
    gerr = {}
    for k, nm in enumerate(names):
        m, s = orc.mean_se(gref[k])
        gerr[nm] = {"gpu": float(gs[0, k, 0]), "oracle": float(m), "rel": float(abs(gs[0, k, 0] - m) / max(abs(m), 1e-12)),
                    "in_se": float(abs(gs[0, k, 0] - m) / s) if s > 0 else None}
    ps = w["paths"] * w["steps"]
    return {"workload": "Heston full-truncation Euler, kappa 2, theta 0.04, xi 0.5, rho -0.7, v0 0.04, S0 100, r 0.05, "
                        "T 1, 2^22 paths x 256 steps, European + arithmetic-Asian calls K = 80..120, FP32",
            "value": ps / t, "unit": UNIT, "ms": t * 1e3, "options_per_s": len(pays) / t,
            "results": _prices(res, pays),
            "error_vs_oracle": {"paths": n_or, "max_rel": max(e["rel"] for e in _errors(orc, small, ref)),
                                "per_price": _errors(orc, small, ref)},
            "greeks": {"ms": tg * 1e3, "wall_ms": tg_wall * 1e3, "value": ps / tg, "unit": UNIT,
                       "what": "7 pathwise Greeks of 18 options, adjoint with checkpoints every 32 steps",
                       "call_K80": {nm: [float(g[0, k, 0]), float(g[0, k, 1])] for k, nm in enumerate(names)},
                       "error_vs_oracle_forward_mode": {"paths": n_g, "call_K80": gerr},
                       "cpu_baseline": {"value": n_g * w["steps"] / tg_or, "unit": UNIT, "cores": os.cpu_count(),
                                        "kind": "oracle", "sample": f"forward-mode tangents, first {n_g} paths, one call"}},
            "cpu_baseline": {"value": n_or * w["steps"] / t_or, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"first {n_or} of 2^22 paths, all 256 steps, 18 options"},
            "roofline": hw.sfu(ps / t, normals=2, ex2=1, other=1,
                               what="2 normals + sqrt(v) + ex2 (Asian average)")}


def config_c4(torch, gb, orc, hw, reps):
    """Portfolio risk: labels, training, surrogate and nested revaluation."""
    from oracle import risk as orisk
    pts = torch.from_numpy(workloads.surrogate_points(1 << 20)).cuda()
    lab_paths = 1 << 13
    t_lab, _, (lab, dl, x) = time_call(torch, lambda: gb.surrogate_label_greeks(pts, lab_paths, with_inputs=True), 1)
    epochs = sum(e for _, e in workloads.SURROGATE_SCHEDULE)
    # the surrogate trained on prices and their pathwise delta / vega (FP32 products)
    net = gb.Mlp(5, 256, 4, workloads.mlp_init())
    losses = []

    def train():
        for lr, ep in workloads.SURROGATE_SCHEDULE:
            losses.append(net.train_d(x, lab, dl, [0, 1], [1.0 / 0.55, 1.0 / 0.15], [0.2, 0.05], epochs=ep,
                                      batch=4096, lr=lr))
    t_train, _, _ = time_call(torch, train, 1, warmup=0)
    # the same network, labels and schedule with the width -> width products on
    # the tensor cores (three-pass TF32)
    net_p = gb.Mlp(5, 256, 4, workloads.mlp_init())
    net_p.set_train_mode("tf32x3")
    losses_p = []

    def train_p():
        for lr, ep in workloads.SURROGATE_SCHEDULE:
            losses_p.append(net_p.train_d(x, lab, dl, [0, 1], [1.0 / 0.55, 1.0 / 0.15], [0.2, 0.05], epochs=ep,
                                          batch=4096, lr=lr))
    t_train_p, _, _ = time_call(torch, train_p, 1, warmup=0)
    net_p.close()
    pf = workloads.risk_portfolio()
    n_scen, n_opt = 1 << 16, len(pf["strike"])
    t_sur, _, sur = time_call(torch, lambda: gb.risk(pf, n_scen=n_scen, method="surrogate", surrogate=net,
                                                     surrogate_precision="bf16", want_pnl=True), max(3, reps // 4))
    t_nest, _, nested = time_call(torch, lambda: gb.risk(pf, n_scen=n_scen, method="nested", inner_paths=1 << 12,
                                                         base_paths=1 << 16, want_pnl=True), 1, warmup=0)
    net.close()
    # the oracle's nested revaluation on a few scenarios (its scenario
    # states, every option with 2^12 inner paths)
    S = orisk.scenarios(pf["s0"], pf["sigma"], pf["corr"], pf["mu"], pf["horizon"], 2, seed=42)
    steps_h = int(round(pf["horizon"] * 252))
    rem = np.rint(np.asarray(pf["maturity"]) * 252).astype(np.int32) - steps_h
    _, t_or = _timed_oracle(lambda: [orisk.option_values(S[s], pf["sigma"], pf["r"], 1.0 / 252, steps_h, s,
                                                         pf["under"], pf["kind"], pf["strike"], pf["barrier"], rem,
                                                         1 << 12) for s in range(2)])
    flop_row = 2 * (5 * 256 + 3 * 256 * 256 + 256)
    rows = n_scen * n_opt
    # the inner paths of a (scenario, underlying) are shared by its options
    # and run to the longest of their remaining maturities
    under = np.asarray(pf["under"])
    steps_u = [int(np.max(np.clip(rem[under == u], 1, None))) for u in np.unique(under)]
    inner_path_steps = n_scen * (1 << 12) * float(sum(steps_u))
    return {"workload": "1024 options (512 European, 512 up-and-out daily) on 32 correlated GBMs, 1-day horizon, "
                        "2^16 scenarios, 99% VaR / CVaR; surrogate 5 -> 256 x 4 (SiLU) -> 1 trained on 2^20 Monte "
                        "Carlo labels (2^13 paths each) and their pathwise delta / vega; nested 2^12 inner paths",
            "labels": {"ms": t_lab * 1e3, "points": 1 << 20, "paths_each": lab_paths,
                       "value": (1 << 20) * lab_paths * 252.5 / t_lab, "unit": UNIT},
            "training": {"ms": t_train * 1e3, "epochs": epochs, "batch": 4096,
                         "labels": "prices + pathwise delta and vega (weights 0.2, 0.05)",
                         "arithmetic": "FP32 SIMT (forward with 2 input tangents, reverse through them)",
                         "final_epoch_loss": losses[-1], "samples_per_s": (1 << 20) * epochs / t_train,
                         "roofline_fma": hw.fma((1 << 20) * epochs * 9 * flop_row / 2 / t_train,
                                                f"9 x {flop_row // 2} FMA per sample (3 stacked rows through forward, "
                                                "input and weight gradients)")},
            "training_tf32x3": {"ms": t_train_p * 1e3, "epochs": epochs, "batch": 4096,
                                "labels": "prices + pathwise delta and vega (weights 0.2, 0.05)",
                                "arithmetic": "width -> width products on the tensor cores (three-pass TF32), "
                                              "the rest FP32 SIMT",
                                "final_epoch_loss": losses_p[-1], "samples_per_s": (1 << 20) * epochs / t_train_p,
                                "roofline_tensor": hw.tensor((1 << 20) * epochs * 9 * flop_row / t_train_p, "tf32",
                                                             f"9 x {flop_row} flop per sample (3 stacked rows "
                                                             "through forward, input and weight gradients)")},
            "surrogate": {"ms": t_sur * 1e3, "var": sur["var"], "cvar": sur["cvar"], "value": rows / t_sur,
                          "unit": "option revaluations/s", "precision": "bf16",
                          "roofline": hw.tensor(rows * flop_row / t_sur, "bf16", f"{flop_row} flop per revaluation")},
            "nested": {"ms": t_nest * 1e3, "var": nested["var"], "cvar": nested["cvar"], "value": rows / t_nest,
                       "unit": "option revaluations/s", "inner_paths": 1 << 12,
                       "inner_path_steps_per_s": inner_path_steps / t_nest,
                       "roofline": hw.sfu(inner_path_steps / t_nest, normals=1, ex2=1,
                                          what="inner path-step (1 normal + the ex2 of the barrier test; "
                                               f"{len(steps_u)} underlyings x 2^12 paths per scenario, each to its "
                                               "longest remaining maturity; achieved and peak in inner path-steps/s)"),
                       "cpu_baseline": {"value": 2 * n_opt / t_or, "unit": "option revaluations/s",
                                        "cores": os.cpu_count(), "kind": "oracle",
                                        "sample": "2 scenarios x 1024 options, 2^12 inner paths each"}},
            "surrogate_vs_nested": {"var_rel": abs(sur["var"] - nested["var"]) / abs(nested["var"]),
                                    "cvar_rel": abs(sur["cvar"] - nested["cvar"]) / abs(nested["cvar"]),
                                    "pnl_corr": float(np.corrcoef(sur["pnl"], nested["pnl"])[0, 1]),
                                    "speedup_revaluation": t_nest / t_sur,
                                    "speedup_pipeline": t_nest / (t_lab + t_train + t_sur)}}


def config_c5(torch, gb, orc, hw, flush, reps):
    w = workloads.basket_d512()
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
    base = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"])
    pays = w["payoffs"]
    d, ps = len(w["s0"]), w["paths"] * w["steps"]
    n_or = 1024
    ref, t_or = _timed_oracle(lambda: orc.gbm_payoffs(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], n_or, pays,
                                                      corr=w["corr"], weights=w["weights"]))
    out = {"workload": "basket d=512 k=16 factors, 2^20 paths x 252 log-Euler steps, ATM basket call + 512-entry "
                       "delta vector, seed 42", "precisions": {},
           "cpu_baseline": {"value": n_or * w["steps"] / t_or, "unit": UNIT, "cores": os.cpu_count(),
                            "kind": "oracle", "sample": f"first {n_or} of 2^20 paths, all 252 steps"}}
    for prec in ("bf16", "fp8", "fp32"):
        c = dict(base, precision=prec)
        t, res = time_plan(torch, gb, model, c, pays, 3 if prec != "fp32" else 2, 1, flush)
        small = gb.price(model, dict(c, paths=n_or), pays)
        rec = {"value": ps / t, "unit": UNIT, "ms": t * 1e3, "options_per_s": 1 / t, "results": _prices(res, pays),
               "error_vs_oracle": {"paths": n_or, "per_price": _errors(orc, small, ref)},
               "roofline_sfu": hw.sfu(ps / t, normals=d, what=f"{d} normals")}
        if prec == "fp32":
            rec["roofline"] = hw.fma(ps / t * d * (d + 1) / 2, f"{d * (d + 1) // 2} FMA per path-step (triangular)")
        else:
            rec["roofline"] = hw.tensor(ps / t * d * (d + 1), prec, f"{d * (d + 1)} flop per path-step (triangular)")
            tg, _, (_, g) = time_call(torch, lambda: gb.greeks(model, c, pays), 1)
            rec["greeks"] = {"ms": tg * 1e3, "value": ps / tg, "unit": UNIT,
                             "what": "price + 512 deltas + 512 vegas + rho from the same paths",
                             "delta_sum": float(g[0, :d, 0].sum())}
        out["precisions"][prec] = rec
    # correlation sensitivities (FP32 paths; the wide path's device buffers and products)
    tc, _, (cp, _, _) = time_call(torch, lambda: gb.corr_greeks(model, dict(base), pays[0]), 1)
    out["corr_greeks"] = {"ms": tc * 1e3, "value": ps / tc, "unit": UNIT, "price": list(cp),
                          "what": f"dP/dLrho and dP/dcorr ({d * (d - 1) // 2} pairs) of the ATM basket call, one "
                                  "mc_corr_greeks call (summed normals, two FP32 products, FP64 adjoint per batch)",
                          "roofline": hw.sfu(ps / tc, normals=d, what=f"{d} normals")}
    return out


# --------------------------------- arms ------------------------------------
def oracle_one_core(paths=2048):
    """The FP64 oracle on one host core (OMP_NUM_THREADS=1, a subprocess):
    path-steps/s on the first `paths` paths of the d = 64 workload."""
    code = ("import sys, time; sys.path.insert(0, %r); import workloads, oracle; oracle.build(); "
            "w = workloads.basket_d64(); t0 = time.perf_counter(); "
            "oracle.gbm_payoffs(w['s0'], w['sigma'], w['r'], w['T'], w['steps'], %d, w['payoffs'], corr=w['corr'], "
            "weights=w['weights'], seed=w['seed']); print(time.perf_counter() - t0)") % (ROOT, paths)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    dt = float(r.stdout.strip().splitlines()[-1])
    return {"value": paths * 252 / dt, "unit": UNIT, "cores": 1, "sample": f"first {paths} of 2^18 paths, all 252 steps"}


def oracle_sample(w, target_s=12.0, max_paths=1 << 16):
    """Time the FP64 oracle on a prefix of the workload's paths, doubling the
    prefix until one run takes at least ~1/4 of target_s (bounded)."""
    import oracle
    oracle.build()
    n = 256
    while True:
        t0 = time.perf_counter()
        oracle.gbm_payoffs(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], n, w["payoffs"],
                           corr=w["corr"], weights=w["weights"], seed=w["seed"])
        dt = time.perf_counter() - t0
        if dt * 4 >= target_s or n >= max_paths:
            return n, dt
        n = min(max_paths, n * max(2, int(target_s / 4 / max(dt, 1e-3))))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workloads.basket_d64()
    times = []
    n, _ = oracle_sample(w, target_s=8.0)  # sizes the sample; its runs are the warm-up
    import oracle
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.gbm_payoffs(w["s0"], w["sigma"], w["r"], w["T"], w["steps"], n, w["payoffs"],
                           corr=w["corr"], weights=w["weights"], seed=w["seed"])
        times.append(time.perf_counter() - t0)
    ps = n * w["steps"] / float(np.median(times))
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": ps, "unit": UNIT, "n_gpus": world,
            "device": f"host CPU, {cores} threads (the FP64 oracle uses no GPU)",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.median(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "paths_sampled": n},
            "cpu_baseline": {"value": ps, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {n} of 2^18 paths, all 252 steps"},
            "e2e": {"value": ps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gbmc(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1906_02818_gb300 as gb

    w = workloads.basket_d64()
    P = w["paths"]
    model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
    cfg = dict(steps=w["steps"], T=w["T"], paths=P, seed=w["seed"], path_offset=rank * P,
               precision=args.prec)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    hw = Hw(torch.cuda.get_device_properties(local).multi_processor_count)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    plan = gb.Plan(model, cfg, w["payoffs"], stream=stream)
    out = torch.empty((len(w["payoffs"]), 2), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.execute(out, stream=stream)
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(local)
    with clk:
        barrier()
        with torch.cuda.stream(stream):
            for s, e in evs:
                flush.fill_(1.0)  # L2 flush between timed iterations (outside the events)
                s.record(stream)
                plan.execute(out, stream=stream)
                e.record(stream)
        barrier()
    step_ms = [s.elapsed_time(e) for s, e in evs]
    tt = torch.tensor([float(sum(step_ms))], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ms_step = float(tt.item()) / args.steps
    launches = plan.launches * args.steps
    res = out.cpu().numpy()
    plan.close()
    path_steps = P * w["steps"] * world
    value = path_steps / (ms_step * 1e-3)
    combined = None
    if world > 1:  # the one exchange of the sharded path: all-reduce of the moments
        from paper_1906_02818_gb300 import shard
        combined = shard.allreduce_results([(float(res[i, 0]), float(res[i, 1])) for i in range(len(w["payoffs"]))],
                                           P, device=torch.device("cuda", local))

    # End to end through the public C-ABI call with host buffers: model
    # upload, Cholesky, kernels, results back to the host, every step.
    e2e_times = []
    for i in range(args.warmup + max(3, min(args.steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gb.price(model, cfg, w["payoffs"], stream=stream)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_s = float(np.median(e2e_times))
    d = len(w["s0"])
    h2d = d * d * 8 + d * 8
    d2h = 4 + d * (d + 1) // 2 * 4 + d * 4 + len(w["payoffs"]) * 16

    per_gpu = P * w["steps"] / (ms_step * 1e-3)
    roof = hw.sfu(per_gpu, normals=d, ex2=d, what=f"{d} normals + {d} ex2 (monitored basket)")
    roof.update(kernel="basket_tc_acc_kernel" if args.prec in ("bf16", "fp16") else
                ("basket_tc_kernel" if args.prec == "fp8" else "basket_fp32_kernel"),
                traffic=HEADLINE_DRAM_BYTES if args.prec == "bf16" else None)
    contraction = (hw.fma(per_gpu * d * (d + 1) / 2, f"{d * (d + 1) // 2} FMA per path-step") if args.prec == "fp32"
                   else hw.tensor(per_gpu * d * (d + 1), "fp8" if args.prec == "fp8" else "bf16",
                                  f"{d * (d + 1)} flop per path-step (triangular contraction)"))

    configs = None
    if world == 1 and args.configs == "all":
        import oracle
        oracle.build()
        reps = max(3, min(args.steps, 20))
        headline = {"s": ms_step * 1e-3, "res": res}
        configs = {}
        for name, fn in (("C1", lambda: config_c1(torch, gb, oracle, hw, flush, reps)),
                         ("C2", lambda: config_c2(torch, gb, oracle, hw, flush, reps, headline)),
                         ("C3", lambda: config_c3(torch, gb, oracle, hw, flush, reps)),
                         ("C4", lambda: config_c4(torch, gb, oracle, hw, reps)),
                         ("C5", lambda: config_c5(torch, gb, oracle, hw, flush, reps))):
            t0 = time.perf_counter()
            try:
                configs[name] = fn()
            except Exception as exc:  # reported, never fatal to the headline line
                configs[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            configs[name]["bench_seconds"] = time.perf_counter() - t0

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            n, dt = oracle_sample(w)
            cpu = {"value": n * w["steps"] / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"first {n} of 2^18 paths, all 252 steps, one run"}
            try:
                cpu["one_core"] = oracle_one_core()
            except Exception as exc:  # reported, never fatal to the GPU line
                cpu["one_core"] = {"unavailable": str(exc)[:200]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else f"{args.prec}+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "paths_per_gpu": P, "time_steps": w["steps"], "d": d,
                       "contraction": args.prec, "l2": "flushed between timed iterations (512 MB write)",
                       "parallelism": f"path shards x{world}"},
            "prices_per_s": len(w["payoffs"]) * world / (ms_step * 1e-3),
            "results": [{"payoff": p["kind"], "price": float(res[i, 0]), "std_err": float(res[i, 1])}
                        for i, p in enumerate(w["payoffs"])],
            "results_all_ranks": None if combined is None else [
                {"payoff": p["kind"], "price": combined[i][0], "std_err": combined[i][1]}
                for i, p in enumerate(w["payoffs"])],
            "e2e": {"value": P * w["steps"] / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s},
            "gpu_launches": launches,
            "roofline": roof,
            "roofline_contraction": contraction,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "step_ms_min_max": [min(step_ms), max(step_ms)],
            "configs": configs,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbmc", choices=["gbmc", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16", "fp16", "fp8"])
    ap.add_argument("--configs", default="all", choices=["all", "none"],
                    help="at one GPU, also measure every workload (C1-C5) after the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gbmc(args)


if __name__ == "__main__":
    main()
