"""Portfolio-risk run of the surrogate pipeline on one GPU, as a JSON line:
Monte Carlo training labels over the surrogate's parameter box, native
training of the network, VaR / CVaR of the 1024-option book by the
surrogate, and the same by nested Monte Carlo (the yardstick), with timings.

  python tests/risk_report.py [--labels 1048576] [--label-paths 8192]
         [--scen 65536] [--inner 4096] [--prec fp32|bf16] [--train fp32|tf32x3] [--alpha 0.99]
         [--accuracy-sweep]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch

    import workloads
    import paper_1906_02818_gb300 as gb

    ap = argparse.ArgumentParser()
    ap.add_argument("--labels", type=int, default=1 << 20)
    ap.add_argument("--label-paths", type=int, default=1 << 13)
    ap.add_argument("--scen", type=int, default=1 << 16)
    ap.add_argument("--inner", type=int, default=1 << 12)
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--train", default="tf32x3", choices=["fp32", "tf32x3"])
    ap.add_argument("--alpha", type=float, default=0.99)
    ap.add_argument("--skip-nested", action="store_true")
    ap.add_argument("--accuracy-sweep", action="store_true",
                    help="nested runs at 2^8 .. 2^14 inner paths; errors against the 2^14 run")
    a = ap.parse_args()

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    pts = torch.from_numpy(workloads.surrogate_points(a.labels)).cuda()
    (lab, x), t_lab = wall(lambda: gb.surrogate_labels(pts, a.label_paths, with_inputs=True))
    net = gb.Mlp(5, 256, 4, workloads.mlp_init())
    net.set_train_mode(a.train)
    losses = []

    def train():
        for lr, ep in workloads.SURROGATE_SCHEDULE:
            losses.append(net.train(x, lab, epochs=ep, batch=4096, lr=lr))
    _, t_train = wall(train)
    pf = workloads.risk_portfolio()
    sur, t_sur = wall(lambda: gb.risk(pf, alpha=a.alpha, n_scen=a.scen, method="surrogate", surrogate=net,
                                      surrogate_precision=a.prec, want_pnl=True))
    out = {
        "workload": "1024 options (512 European, 512 up-and-out daily) on 32 correlated GBMs, 1-day horizon",
        "alpha": a.alpha, "scenarios": a.scen,
        "labels": {"points": a.labels, "paths_each": a.label_paths, "seconds": t_lab,
                   "path_steps_per_s": float(a.labels * a.label_paths * 252.5 / t_lab)},
        "training": {"epochs": sum(e for _, e in workloads.SURROGATE_SCHEDULE), "seconds": t_train, "arithmetic": a.train,
                     "final_epoch_mse": losses[-1]},
        "surrogate": {"var": sur["var"], "cvar": sur["cvar"], "seconds": t_sur, "precision": a.prec,
                      "revaluations_per_s": a.scen * 1024 / t_sur},
        "surrogate_pipeline_seconds": t_lab + t_train + t_sur,
    }
    if not a.skip_nested:
        nested, t_nest = wall(lambda: gb.risk(pf, alpha=a.alpha, n_scen=a.scen, method="nested", inner_paths=a.inner,
                                              base_paths=1 << 16, want_pnl=True))
        out["nested"] = {"var": nested["var"], "cvar": nested["cvar"], "seconds": t_nest, "inner_paths": a.inner,
                         "revaluations_per_s": a.scen * 1024 / t_nest}
        out["surrogate_error_vs_nested"] = {
            "var_rel": abs(sur["var"] - nested["var"]) / abs(nested["var"]),
            "cvar_rel": abs(sur["cvar"] - nested["cvar"]) / abs(nested["cvar"]),
            "pnl_corr": float(np.corrcoef(sur["pnl"], nested["pnl"])[0, 1]),
            "pnl_rmse": float(np.sqrt(np.mean((sur["pnl"] - nested["pnl"]) ** 2))),
            "pnl_std_nested": float(np.std(nested["pnl"])),
            "speedup": t_nest / t_sur}
    if a.accuracy_sweep:
        # Plain nested Monte Carlo at several inner path counts on the same
        # scenarios; the 2^14-path run is the reference for every error.
        runs = {}
        for inner in (1 << 8, 1 << 10, 1 << 12, 1 << 14):
            r, t = wall(lambda: gb.risk(pf, alpha=a.alpha, n_scen=a.scen, method="nested", inner_paths=inner,
                                        base_paths=1 << 16, want_pnl=True))
            runs[inner] = (r, t)
        ref = runs[1 << 14][0]

        def errs(r):
            return {"var_rel": abs(r["var"] - ref["var"]) / abs(ref["var"]),
                    "cvar_rel": abs(r["cvar"] - ref["cvar"]) / abs(ref["cvar"]),
                    "pnl_rmse": float(np.sqrt(np.mean((r["pnl"] - ref["pnl"]) ** 2)))}
        # a nested run with N inner paths uses the first N of the reference's
        # paths: its error against the reference is sqrt(1 - N / 2^14) of its
        # error against the exact revaluation; pnl_rmse_exact undoes that
        sweep = {}
        for k, (r, t) in runs.items():
            if k == 1 << 14:
                continue
            e = errs(r)
            e["pnl_rmse_exact"] = e["pnl_rmse"] / np.sqrt(1.0 - k / float(1 << 14))
            sweep[str(k)] = dict(seconds=t, **e)
        se = errs(sur)  # includes the reference's own noise: conservative for the surrogate
        match = [int(k) for k, v in sweep.items() if v["pnl_rmse_exact"] <= se["pnl_rmse"]]
        out["accuracy_vs_nested_2^14"] = {
            "reference_seconds": runs[1 << 14][1], "nested": sweep,
            "surrogate": dict(seconds=t_sur, **se),
            "cheapest_nested_at_surrogate_pnl_rmse": min(match) if match else None}
    print(json.dumps(out), flush=True)
    net.close()


if __name__ == "__main__":
    main()
