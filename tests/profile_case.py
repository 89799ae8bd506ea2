"""Run one workload a fixed number of times (for profilers).

  python tests/profile_case.py basket64 --paths 16384 --reps 2 [--prec fp32]
  python tests/profile_case.py gbm1d --paths 1048576
  python tests/profile_case.py heston --paths 65536
  python tests/profile_case.py basket512 --paths 32768 --prec bf16
  python tests/profile_case.py heston_greeks --paths 65536
  python tests/profile_case.py mlp --paths 1048576 --prec bf16   (paths = network rows)
  python tests/profile_case.py labels --paths 4096              (paths = label points)
  python tests/profile_case.py risk_nested --paths 256          (paths = scenarios)
  python tests/profile_case.py train --paths 262144            (paths = samples, 1 epoch;
                                                                                 --prec tf32x3: tensor-core training)
  python tests/profile_case.py train_d --paths 262144          (derivative-label training: prices + 2
                                                                input-gradient labels, 1 epoch;
                                                                --prec tf32x3: tensor-core products)
  python tests/profile_case.py bridge --paths 1048576          (the In and Out Put, 25 steps)
  python tests/profile_case.py qmc --paths 262144              (points x 16 replications)
  python tests/profile_case.py mlmc --paths 16384              (correction paths, d = 64, bf16)
  python tests/profile_case.py factor512 --paths 65536
  python tests/profile_case.py corr64 --paths 65536          (correlation sensitivities, d = 64)
  python tests/profile_case.py corr512 --paths 65536         (correlation sensitivities, d = 512)
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch

    import workloads
    import paper_1906_02818_gb300 as gb

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["gbm1d", "basket64", "basket512", "heston", "heston_greeks", "mlp", "labels",
                                     "risk_nested", "train", "train_d", "bridge", "qmc", "mlmc", "factor512", "corr64", "corr512"])
    ap.add_argument("--paths", type=int, default=None)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--prec", default="fp32")
    a = ap.parse_args()
    if a.case in ("mlp", "labels", "risk_nested", "train", "train_d", "bridge", "qmc", "mlmc", "factor512", "corr64", "corr512"):
        _other(a, torch, workloads, gb)
        return
    if a.case in ("heston", "heston_greeks"):
        w = workloads.heston(paths=a.paths or (1 << 16))
        model = dict(kind="heston", **w["model"])
    else:
        w = {"gbm1d": workloads.gbm_1d, "basket64": workloads.basket_d64, "basket512": workloads.basket_d512}[a.case]()
        if a.paths:
            w["paths"] = a.paths
        model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w.get("corr"), weights=w.get("weights"), r=w["r"])
    cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"], precision=a.prec)
    if a.case == "heston_greeks":
        for _ in range(a.reps):
            _, g = gb.greeks(model, cfg, w["payoffs"])
        print(a.case, w["paths"], g[0, :, 0].tolist())
        return
    with gb.Plan(model, cfg, w["payoffs"]) as plan:
        for _ in range(a.reps):
            out = plan.execute()
        torch.cuda.synchronize()
        print(a.case, w["paths"], out.cpu().numpy().tolist())


def _other(a, torch, workloads, gb):
    if a.case == "mlp":
        n = a.paths or (1 << 20)
        net = gb.Mlp(5, 256, 4, workloads.mlp_init())
        x = torch.rand((n, 5), device="cuda", generator=torch.Generator("cuda").manual_seed(1)) * 2 - 1
        for _ in range(a.reps):
            y = net.forward(x, precision=a.prec)
        torch.cuda.synchronize()
        print(a.case, n, a.prec, float(y.sum()))
        net.close()
    elif a.case == "bridge":
        import numpy as np
        model = dict(kind="gbm", s0=np.array([100.0]), sigma=np.array([0.8]), r=0.03)
        cfg = dict(steps=25, T=2.0, paths=a.paths or (1 << 20), seed=42, monitoring="bridge")
        for _ in range(a.reps):
            r = gb.price(model, cfg, [dict(kind="ui_put", strike=120.0, barrier=140.0)])
        print(a.case, r)
    elif a.case == "qmc":
        import numpy as np
        s0, sg, corr = workloads.basket_market(16, 4)
        w = np.full(16, 1 / 16)
        model = dict(kind="gbm", s0=s0, sigma=sg, corr=corr, weights=w, r=0.05)
        for _ in range(a.reps):
            r, _ = gb.price_qmc(model, dict(steps=1, T=1.0, paths=a.paths or (1 << 18), seed=42),
                                [dict(kind="call", strike=float(w @ s0))], replications=16)
        print(a.case, r)
    elif a.case == "mlmc":
        w = workloads.basket_d64(paths=1 << 14)
        model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
        cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"], precision="bf16")
        for _ in range(a.reps):
            r = gb.price_mlmc(model, cfg, w["payoffs"], a.paths or (1 << 14))
        print(a.case, r[0]["price"], r[0]["correction"])
    elif a.case == "corr64":
        w = workloads.basket_d64(paths=a.paths or (1 << 18))
        model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
        for _ in range(a.reps):
            r = gb.corr_greeks(model, dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=42), w["payoffs"][0])
        print(a.case, r[0])
    elif a.case == "corr512":
        import time
        w = workloads.basket_d512(paths=a.paths or (1 << 16))
        model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w["corr"], weights=w["weights"], r=w["r"])
        for _ in range(a.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = gb.corr_greeks(model, dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=42), w["payoffs"][0])
            dt = time.perf_counter() - t0
        print(a.case, w["paths"], r[0], f"{dt:.3f} s per call")
    elif a.case == "factor512":
        w = workloads.basket_d512_factor(paths=a.paths or (1 << 16))
        model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], loadings=w["loadings"], weights=w["weights"], r=w["r"])
        for _ in range(a.reps):
            r = gb.price(model, dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=42), w["payoffs"])
        print(a.case, r)
    elif a.case == "train":
        import time
        n = a.paths or (1 << 18)
        net = gb.Mlp(5, 256, 4, workloads.mlp_init())
        net.set_train_mode("tf32x3" if a.prec == "tf32x3" else "fp32")
        g = torch.Generator("cuda").manual_seed(2)
        x = torch.rand((n, 5), device="cuda", generator=g) * 2 - 1
        t = torch.rand(n, device="cuda", generator=g)
        for _ in range(a.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss = net.train(x, t, epochs=1, batch=4096, lr=1e-3)
            dt = time.perf_counter() - t0
        print(a.case, n, loss, f"{dt:.4f} s/epoch, {dt / (n // 4096) * 1e3:.3f} ms/step")
        net.close()
    elif a.case == "train_d":
        import time
        n = a.paths or (1 << 18)
        net = gb.Mlp(5, 256, 4, workloads.mlp_init())
        net.set_train_mode("tf32x3" if a.prec == "tf32x3" else "fp32")
        g = torch.Generator("cuda").manual_seed(2)
        x = torch.rand((n, 5), device="cuda", generator=g) * 2 - 1
        t = torch.rand(n, device="cuda", generator=g)
        dl = torch.rand((n, 2), device="cuda", generator=g)
        for _ in range(a.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss = net.train_d(x, t, dl, [0, 1], [1.0, 1.0], [0.2, 0.05], epochs=1, batch=4096, lr=1e-3)
            dt = time.perf_counter() - t0
        print(a.case, n, loss, f"{dt:.4f} s/epoch, {dt / (n // 4096) * 1e3:.3f} ms/step")
        net.close()
    elif a.case == "labels":
        pts = torch.from_numpy(workloads.surrogate_points(a.paths or 4096)).cuda()
        for _ in range(a.reps):
            lab = gb.surrogate_labels(pts, 1 << 13)
        torch.cuda.synchronize()
        print(a.case, pts.shape[0], float(lab.sum()))
    else:
        pf = workloads.risk_portfolio()
        for _ in range(a.reps):
            r = gb.risk(pf, n_scen=a.paths or 256, method="nested", inner_paths=1 << 12, base_paths=1 << 16)
        print(a.case, r["var"], r["cvar"])


if __name__ == "__main__":
    main()
