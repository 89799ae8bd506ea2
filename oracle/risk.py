"""FP64 portfolio-risk reference: scenarios, nested revaluation (oracle.c),
PnL, and the VaR / CVaR estimators.

TEST INFRASTRUCTURE ONLY (see the oracle package docstring).

Reading of Sec. VI.B (its printed VaR formula is garbled): with losses
l = -PnL over n scenarios sorted in decreasing order, VaR_alpha is the k-th
largest loss, k = ceil((1 - alpha) n), and CVaR_alpha the mean of the losses
strictly above VaR_alpha (VaR_alpha itself when none is), the conditional
expectation of the loss beyond VaR.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _dptr, _f64, _load, OracleError


def var_cvar(pnl, alpha):
    l = np.sort(-np.asarray(pnl, dtype=np.float64))[::-1]
    k = max(1, math.ceil((1.0 - alpha) * l.size - 1e-9))
    var = l[k - 1]
    tail = l[:k][l[:k] > var]
    return float(var), float(tail.mean()) if tail.size else float(var), int(tail.size)


def scenarios(s0, sigma, corr, mu, h, nscen, seed=42):
    lib = _load()
    s0, sigma, corr = _f64(s0), _f64(sigma), _f64(corr)
    d = s0.size
    out = np.empty((nscen, d))
    lib.orc_risk_scenarios.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_double)] * 3 + [
        ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    rc = lib.orc_risk_scenarios(d, _dptr(s0), _dptr(sigma), _dptr(corr), mu, h, nscen, seed, _dptr(out))
    if rc:
        raise OracleError(f"orc_risk_scenarios: {rc}")
    return out


def option_values(state, sigma, r, dt, hsteps, scen, under, kind, K, H, rem, inner, seed=42):
    """Values of every option at `state` (scenario `scen`, or the base date
    when scen < 0); kind codes: 0 call, 1 put, 4 up-and-out call."""
    lib = _load()
    i32 = ctypes.POINTER(ctypes.c_int)
    lib.orc_risk_values.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                    i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), i32,
                                    ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    state, sigma, K, H = _f64(state), _f64(sigma), _f64(K), _f64(H)
    under, kind, rem = (np.ascontiguousarray(a, dtype=np.int32) for a in (under, kind, rem))
    V = np.empty(K.size)
    lib.orc_risk_values(state.size, _dptr(state), _dptr(sigma), r, dt, hsteps, scen, K.size,
                        under.ctypes.data_as(i32), kind.ctypes.data_as(i32), _dptr(K), _dptr(H),
                        rem.ctypes.data_as(i32), inner, seed, _dptr(V))
    return V


def labels(points, paths, spy=252, seed=42):
    lib = _load()
    pts = _f64(points).reshape(-1, 5)
    out = np.empty(pts.shape[0])
    lib.orc_surrogate_labels.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    lib.orc_surrogate_labels(pts.shape[0], _dptr(pts), paths, spy, seed, _dptr(out))
    return out


def label_greeks(points, paths, spy=252, seed=42):
    """Pathwise price, delta (d/d S/K) and vega (d/d sigma) of the European
    training points, each (mean, se): shape [n, 6]; NaN rows for barrier
    points (orc_surrogate_label_greeks)."""
    lib = _load()
    pts = _f64(points).reshape(-1, 5)
    out = np.empty((pts.shape[0], 6))
    lib.orc_surrogate_label_greeks.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                               ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    lib.orc_surrogate_label_greeks(pts.shape[0], _dptr(pts), paths, spy, seed, _dptr(out))
    return out
