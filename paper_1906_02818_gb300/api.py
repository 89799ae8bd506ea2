"""Python binding of the C ABI (include/mc.h): argument marshalling only.

PyTorch provides device memory and streams; every simulation step runs in the
library's CUDA kernels.  Model and configuration are plain keyword arguments:

  model:  kind="gbm", s0, sigma, corr=None, weights=None, r
          kind="heston", s0, v0, r, kappa, theta, xi, rho
  cfg:    steps, T, paths, seed=42, scheme="log_euler", precision="fp32",
          path_offset=0, ckpt_every=0
  payoff: dict(kind=<name in native.PAYOFF>, strike=K, barrier=H)
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native
from .native import McModel, McPayoff, McResult, McSimCfg, check


class _Marshalled:
    """Keeps the numpy arrays alive while the C structs point at them."""

    def __init__(self, model: dict, cfg: dict, payoffs=None):
        kind = model.get("kind", "gbm")
        self.arrays = []
        m = McModel()
        m.kind = native.MODEL[kind]
        s0 = self._arr(np.atleast_1d(model["s0"]))
        m.d = s0.size
        m.s0 = self._ptr(s0)
        if kind == "gbm":
            m.sigma = self._ptr(self._arr(np.atleast_1d(model["sigma"])))
            if model.get("corr") is not None:
                m.corr = self._ptr(self._arr(model["corr"]))
            if model.get("weights") is not None:
                m.weights = self._ptr(self._arr(model["weights"]))
        else:
            for k in ("v0", "kappa", "theta", "xi", "rho"):
                setattr(m, k, float(model[k]))
        m.r = float(model["r"])
        self.model = m
        c = McSimCfg()
        c.scheme = native.SCHEME[cfg.get("scheme", "log_euler")]
        c.steps = int(cfg["steps"])
        c.T = float(cfg["T"])
        c.paths = int(cfg["paths"])
        c.path_offset = int(cfg.get("path_offset", 0))
        c.seed = int(cfg.get("seed", 42))
        c.precision = native.PRECISION[cfg.get("precision", "fp32")]
        c.ckpt_every = int(cfg.get("ckpt_every", 0))
        self.cfg = c
        self.n_payoff = 0
        self.payoffs = None
        if payoffs is not None:
            n = len(payoffs)
            arr = (McPayoff * max(n, 1))()
            for i, p in enumerate(payoffs):
                arr[i].kind = native.PAYOFF[p["kind"]]
                arr[i].strike = float(p.get("strike", 0.0))
                arr[i].barrier = float(p.get("barrier", float("inf")))
            self.payoffs = arr
            self.n_payoff = n

    def _arr(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.arrays.append(a)
        return a

    @staticmethod
    def _ptr(a):
        return a.ctypes.data_as(native.c_double_p)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def price(model: dict, cfg: dict, payoffs, stream=None):
    """Discounted prices and standard errors: list of (price, se)."""
    L = native.lib()
    mm = _Marshalled(model, cfg, payoffs)
    out = (McResult * mm.n_payoff)()
    check(L.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out,
                     _stream_handle(stream)))
    return [(r.price, r.se) for r in out]


def greeks(model: dict, cfg: dict, payoffs, stream=None):
    """Pathwise Greeks: (prices, greeks) with prices a list of (price, se) and
    greeks an array [n_payoff, G, 2] of (mean, se); G = 7 for Heston
    (S0, v0, r, kappa, theta, xi, rho), 3 for single-asset GBM (S0, sigma, r)."""
    L = native.lib()
    mm = _Marshalled(model, cfg, payoffs)
    G = L.mc_greek_count(ctypes.byref(mm.model))
    pr = (McResult * mm.n_payoff)()
    gr = (McResult * (mm.n_payoff * G))()
    check(L.mc_greeks(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, pr, gr,
                      _stream_handle(stream)))
    g = np.array([[r.price, r.se] for r in gr]).reshape(mm.n_payoff, G, 2)
    return [(r.price, r.se) for r in pr], g


def simulate(model: dict, cfg: dict, save_every: int = 1, stream=None):
    """Simulated paths as a CUDA float32 tensor [steps/save_every + 1, D, paths]."""
    import torch
    L = native.lib()
    mm = _Marshalled(model, cfg)
    D = 2 if model.get("kind", "gbm") == "heston" else mm.model.d
    nsave = mm.cfg.steps // save_every + 1 if save_every > 0 else 0
    out = torch.empty((nsave, D, mm.cfg.paths), dtype=torch.float32, device="cuda")
    check(L.mc_simulate(ctypes.byref(mm.model), ctypes.byref(mm.cfg), int(save_every),
                        ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


class Plan:
    """A set-up computation (mc_plan_create) executable asynchronously."""

    def __init__(self, model: dict, cfg: dict, payoffs, stream=None):
        self._lib = native.lib()
        mm = _Marshalled(model, cfg, payoffs)
        self.n_payoff = mm.n_payoff
        h = ctypes.c_void_p()
        check(self._lib.mc_plan_create(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs,
                                       mm.n_payoff, ctypes.byref(h), _stream_handle(stream)))
        self._h = h

    def execute(self, out=None, stream=None):
        """Launch on `stream`; returns the CUDA float64 tensor [n_payoff, 2] of
        (price, se) that the launch will fill."""
        import torch
        if out is None:
            out = torch.empty((self.n_payoff, 2), dtype=torch.float64, device="cuda")
        check(self._lib.mc_plan_execute(self._h, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    @property
    def launches(self) -> int:
        return self._lib.mc_plan_launches(self._h)

    def close(self):
        if self._h:
            self._lib.mc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
