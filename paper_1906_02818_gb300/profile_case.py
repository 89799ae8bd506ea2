"""Run one workload's plan a fixed number of times (for profilers).

  python -m paper_1906_02818_gb300.profile_case basket64 --paths 16384 --reps 2 [--prec fp32]
  python -m paper_1906_02818_gb300.profile_case gbm1d --paths 1048576
  python -m paper_1906_02818_gb300.profile_case heston --paths 65536
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
    ap.add_argument("case", choices=["gbm1d", "basket64", "basket512", "heston"])
    ap.add_argument("--paths", type=int, default=None)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--prec", default="fp32")
    a = ap.parse_args()
    if a.case == "heston":
        w = workloads.heston(paths=a.paths or (1 << 16))
        model = dict(kind="heston", **w["model"])
    else:
        w = {"gbm1d": workloads.gbm_1d, "basket64": workloads.basket_d64, "basket512": workloads.basket_d512}[a.case]()
        if a.paths:
            w["paths"] = a.paths
        model = dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w.get("corr"), weights=w.get("weights"), r=w["r"])
    cfg = dict(steps=w["steps"], T=w["T"], paths=w["paths"], seed=w["seed"], precision=a.prec)
    with gb.Plan(model, cfg, w["payoffs"]) as plan:
        for _ in range(a.reps):
            out = plan.execute()
        torch.cuda.synchronize()
        print(a.case, w["paths"], out.cpu().numpy().tolist())


if __name__ == "__main__":
    main()
