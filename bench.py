"""Benchmark of the Monte Carlo hot path on the correlated-basket workload:
d = 64 assets (S0 ~ U[50,150], sigma ~ U[0.1,0.4], 4-factor correlation plus
0.05 I), 2^18 paths x 252 log-Euler steps, ATM arithmetic basket call and
up-and-out basket call at 1.3 B(0), Philox4x32-10 stream seed 42.

One step = one mc_plan_execute: RNG + Box-Muller + correlation contraction +
state update + payoffs + reduction over every path (all in the library's
kernels).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|bf16|fp16|fp8]
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

# Warp instructions the basket kernel issues per path-step (smsp__inst_executed.sum
# divided by paths x steps) from the ncu capture of the same kernel build,
# recorded in profiles/.  None where no capture of the current build exists.
WORKLOAD = ("basket d=64 k=4 factors, 2^18 paths x 252 log-Euler steps, ATM basket call + up-and-out call at "
            "1.3 B0, seed 42")
INST_PER_PATH_STEP = {"fp32": None, "bf16": 48.38, "fp16": None, "fp8": None}
# DRAM bytes (read + write) of one launch of that kernel in the same capture:
# only the factor tile and launch constants are read, whatever the path count.
DRAM_BYTES_PER_LAUNCH = {"bf16": 76288}


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

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, clock_sampler=None):
        c = dict(cfg, precision=prec)
        plan = gb.Plan(model, c, w["payoffs"], stream=stream)
        out = torch.empty((len(w["payoffs"]), 2), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                plan.execute(out, stream=stream)
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with (clock_sampler or _Null()):
            barrier()
            with torch.cuda.stream(stream):
                for s, e in evs:
                    flush.fill_(1.0)  # L2 flush between timed iterations (outside the events)
                    s.record(stream)
                    plan.execute(out, stream=stream)
                    e.record(stream)
            barrier()
        step_ms = [s.elapsed_time(e) for s, e in evs]
        t = torch.tensor([float(sum(step_ms))], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        launches = plan.launches * args.steps
        res = out.cpu().numpy()
        plan.close()
        return float(t.item()) / args.steps, step_ms, res, launches

    clk = ClockSampler(local)
    ms_step, step_ms, res, launches = timed(args.prec, clk)
    fp32 = timed("fp32") if args.prec != "fp32" else None
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
        r = gb.price(model, cfg, w["payoffs"], stream=stream)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_s = float(np.median(e2e_times))
    d = len(w["s0"])
    h2d = d * d * 8 + d * 8
    d2h = 4 + d * (d + 1) // 2 * 4 + d * 4 + len(w["payoffs"]) * 16

    pk, pk_kind = peaks()
    clocks = clk.summary()
    inst = INST_PER_PATH_STEP.get(args.prec)
    issue_peak = 152 * 4 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12  # T warp-inst/s
    if inst is not None:
        achieved = inst * P * w["steps"] / (ms_step * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": issue_peak, "unit": "Twarp-inst/s",
                "frac": achieved / issue_peak, "traffic": DRAM_BYTES_PER_LAUNCH.get(args.prec),
                "kernel": ("basket_tc_acc_kernel" if args.prec in ("bf16", "fp16") else "basket_tc_kernel")
                if args.prec != "fp32" else "basket_fp32_kernel",
                "basis": f"{inst} warp instructions per path-step (ncu, profiles/) x path-steps / CUDA-event "
                         f"time; peak = 152 SMs x 4 issue slots x {pk.get('sm_max_mhz', 2070.0)} MHz "
                         f"(issue rate; sm_max_mhz from MEASURED_PEAKS.json, {pk_kind})"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": issue_peak, "unit": "Twarp-inst/s", "frac": None,
                "traffic": None, "basis": "instruction count per path-step not yet measured for this precision"}
    # the contraction's own FP32 FMA-pipe fraction (algorithmic: d(d+1) flop per path-step)
    fma_peak = 152 * 128 * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    contraction_tflops = d * (d + 1) * P * w["steps"] / (ms_step * 1e-3) / 1e12

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
            "contraction_fp32_tflops": {"achieved": contraction_tflops, "peak": fma_peak,
                                        "frac": contraction_tflops / fma_peak},
            "clocks": clocks,
            "fp32_contraction": None if fp32 is None else {
                "value": path_steps / (fp32[0] * 1e-3), "ms_per_step": fp32[0],
                "results": [{"payoff": p["kind"], "price": float(fp32[2][i, 0]), "std_err": float(fp32[2][i, 1])}
                            for i, p in enumerate(w["payoffs"])],
                "diff_vs_headline_in_se": [float(abs(res[i, 0] - fp32[2][i, 0]) / fp32[2][i, 1])
                                           for i in range(len(w["payoffs"]))]},
            "cpu_baseline": cpu,
            "step_ms_min_max": [min(step_ms), max(step_ms)],
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
