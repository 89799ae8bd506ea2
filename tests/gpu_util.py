"""Helpers shared by the GPU parity tests: conversion of the seeded workloads
into the binding's and the oracle's argument forms, and the tolerance rules.

Tolerances (FP32 path vs FP64 oracle on the identical random stream):
  smooth payoffs (European, Asian, basket) and their Greeks: 1e-5 relative;
  barrier payoffs: 1e-5 relative plus the payoff mass of the paths whose
  monitored extreme lies within the FP32 path error band of the barrier (the
  knock decision of those paths may legitimately differ); the count of such
  paths is reported.
"""
import numpy as np

REL = 1e-5
BAND = 2e-5  # relative FP32 error bound of a monitored underlying over <= 256 steps


def gbm_model(w):
    return dict(kind="gbm", s0=w["s0"], sigma=w["sigma"], corr=w.get("corr"), weights=w.get("weights"), r=w["r"])


def cfg_of(w, paths=None, **kw):
    c = dict(steps=w["steps"], T=w["T"], paths=paths or w["paths"], seed=w.get("seed", 42))
    c.update(kw)
    return c


def oracle_gbm(orc, w, paths, payoffs, scheme="log_euler", path_offset=0, steps=None):
    return orc.gbm_payoffs(w["s0"], w["sigma"], w["r"], w["T"], steps or w["steps"], paths, payoffs,
                           corr=w.get("corr"), weights=w.get("weights"), scheme=scheme,
                           seed=w.get("seed", 42), path_offset=path_offset)


def assert_price_close(got, per_path, payoffs, band_mass=None, label=""):
    """got: list of (price, se) from the library; per_path: oracle [n_pay, N]."""
    import oracle
    for i, p in enumerate(payoffs):
        want, se = oracle.mean_se(per_path[i])
        tol = REL * max(abs(want), 1e-3 * se if se > 0 else 1e-12)
        if band_mass is not None and band_mass[i] is not None:
            tol += band_mass[i]
        assert abs(got[i][0] - want) <= tol, (label, p, got[i], want, tol)
        if se > 0:
            assert abs(got[i][1] - se) <= 1e-3 * se, (label, p, got[i][1], se)
