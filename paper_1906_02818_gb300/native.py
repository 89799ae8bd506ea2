"""ctypes mirror of include/mc.h and the loader of libgbmc.so.

Argument marshalling only: every simulation step runs in the library's CUDA
kernels.  There is no fallback: if the library is missing or cannot be
loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# GBMC_LIBRARY selects another build of the same library (the sanitizer
# build of the tests); by default the in-tree release build.
LIB_PATH = os.environ.get("GBMC_LIBRARY") or os.path.join(_PKG, "libgbmc.so")

c_double_p = ctypes.POINTER(ctypes.c_double)

# enums of mc.h
MC_OK, MC_EINVAL, MC_ENOTPSD, MC_ENOMEM, MC_ECUDA, MC_ETIMEOUT, MC_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
MC_MLP_TRAIN_FP32, MC_MLP_TRAIN_TF32X3 = 0, 1
STATUS_NAMES = {0: "MC_OK", -1: "MC_EINVAL", -2: "MC_ENOTPSD", -3: "MC_ENOMEM", -4: "MC_ECUDA",
                -5: "MC_ETIMEOUT", -6: "MC_EUNSUPPORTED"}
MODEL = {"gbm": 0, "heston": 1}
SCHEME = {"log_euler": 0, "euler": 1}
PRECISION = {"fp32": 0, "bf16": 1, "fp16": 2, "fp8": 3}
MONITORING = {"discrete": 0, "bridge": 1}
PAYOFF = {"call": 0, "put": 1, "asian_call": 2, "asian_put": 3,
          "uo_call": 4, "ui_call": 5, "uo_put": 6, "ui_put": 7,
          "do_call": 8, "di_call": 9, "do_put": 10, "di_put": 11}
MAX_PAYOFFS = 32


class McModel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("d", ctypes.c_int32),
                ("s0", c_double_p), ("sigma", c_double_p), ("corr", c_double_p), ("weights", c_double_p),
                ("r", ctypes.c_double), ("v0", ctypes.c_double), ("kappa", ctypes.c_double),
                ("theta", ctypes.c_double), ("xi", ctypes.c_double), ("rho", ctypes.c_double),
                ("n_factors", ctypes.c_int32), ("loadings", c_double_p)]


class McSimCfg(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("steps", ctypes.c_int32), ("T", ctypes.c_double),
                ("paths", ctypes.c_int64), ("path_offset", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("ckpt_every", ctypes.c_int32), ("monitoring", ctypes.c_int32)]


class McPayoff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("strike", ctypes.c_double), ("barrier", ctypes.c_double)]


class McResult(ctypes.Structure):
    _fields_ = [("price", ctypes.c_double), ("se", ctypes.c_double)]


class McMlmcResult(ctypes.Structure):
    _fields_ = [("price", ctypes.c_double), ("se", ctypes.c_double), ("coarse", McResult),
                ("correction", McResult), ("ref_level", McResult), ("coarse_level", McResult)]


class McPortfolio(ctypes.Structure):
    _fields_ = [("n_under", ctypes.c_int32), ("s0", c_double_p), ("sigma", c_double_p), ("corr", c_double_p),
                ("r", ctypes.c_double), ("mu", ctypes.c_double), ("n_opt", ctypes.c_int32),
                ("under", ctypes.POINTER(ctypes.c_int32)), ("kind", ctypes.POINTER(ctypes.c_int32)),
                ("strike", c_double_p), ("barrier", c_double_p), ("maturity", c_double_p),
                ("position", c_double_p)]


class McRiskCfg(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("horizon", ctypes.c_double), ("n_scen", ctypes.c_int64),
                ("steps_per_year", ctypes.c_int32), ("method", ctypes.c_int32), ("inner_paths", ctypes.c_int32),
                ("base_paths", ctypes.c_int32), ("seed", ctypes.c_uint64), ("surrogate", ctypes.c_void_p),
                ("surrogate_precision", ctypes.c_int32), ("scen_offset", ctypes.c_int64)]


class McRiskResult(ctypes.Structure):
    _fields_ = [("var", ctypes.c_double), ("cvar", ctypes.c_double), ("base_value", ctypes.c_double),
                ("n_tail", ctypes.c_int64)]


RISK_METHOD = {"nested": 0, "surrogate": 1}


class McMlpDloss(ctypes.Structure):
    _fields_ = [("n_dir", ctypes.c_int32), ("dir", ctypes.c_int32 * 4), ("scale", ctypes.c_float * 4),
                ("weight", ctypes.c_float * 4)]

# name, restype, argtypes  (the complete exported surface of mc.h)
SIGNATURES = [
    ("mc_version", ctypes.c_int, []),
    ("mc_last_error", ctypes.c_char_p, []),
    ("mc_release_cache", ctypes.c_int, []),
    ("mc_simulate", ctypes.c_int, [ctypes.POINTER(McModel), ctypes.POINTER(McSimCfg), ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_price", ctypes.c_int, [ctypes.POINTER(McModel), ctypes.POINTER(McSimCfg), ctypes.POINTER(McPayoff),
                                ctypes.c_int32, ctypes.POINTER(McResult), ctypes.c_void_p]),
    ("mc_price_mlmc", ctypes.c_int, [ctypes.POINTER(McModel), ctypes.POINTER(McSimCfg), ctypes.POINTER(McPayoff),
                                     ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(McMlmcResult), ctypes.c_void_p]),
    ("mc_price_qmc", ctypes.c_int, [ctypes.POINTER(McModel), ctypes.POINTER(McSimCfg), ctypes.POINTER(McPayoff),
                                    ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(McResult),
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("mc_greek_count", ctypes.c_int32, [ctypes.POINTER(McModel)]),
    ("mc_greeks", ctypes.c_int, [ctypes.POINTER(McModel), ctypes.POINTER(McSimCfg), ctypes.POINTER(McPayoff),
                                 ctypes.c_int32, ctypes.POINTER(McResult), ctypes.POINTER(McResult),
                                 ctypes.c_void_p]),
    ("mc_corr_greeks", ctypes.c_int, [ctypes.POINTER(McModel), ctypes.POINTER(McSimCfg), ctypes.POINTER(McPayoff),
                                      ctypes.POINTER(McResult), ctypes.POINTER(McResult), ctypes.POINTER(McResult),
                                      ctypes.c_void_p]),
    ("mc_plan_create", ctypes.c_int, [ctypes.POINTER(McModel), ctypes.POINTER(McSimCfg),
                                      ctypes.POINTER(McPayoff), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    ("mc_plan_execute", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_plan_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("mc_plan_launches", ctypes.c_int, [ctypes.c_void_p]),
    ("mc_mlp_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]),
    ("mc_mlp_param_count", ctypes.c_int64, [ctypes.c_void_p]),
    ("mc_mlp_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_mlp_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_mlp_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int32, ctypes.c_void_p]),
    ("mc_mlp_loss_grad", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_mlp_train", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("mc_mlp_apply_grad", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p]),
    ("mc_mlp_set_train_mode", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("mc_mlp_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("mc_risk", ctypes.c_int, [ctypes.POINTER(McPortfolio), ctypes.POINTER(McRiskCfg),
                               ctypes.POINTER(McRiskResult), ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_surrogate_labels", ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_debug_status", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_int64)]),
    ("mc_moments", ctypes.c_int, [ctypes.POINTER(McResult), ctypes.c_int32, ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_double)]),
    ("mc_combine", ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.POINTER(McResult)]),
    ("mc_tail", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(McRiskResult),
                               ctypes.c_void_p]),
    ("mc_mlp_loss_grad_sums", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_mlp_apply_grad_sums", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                                              ctypes.c_void_p]),
    ("mc_surrogate_label_greeks", ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
    ("mc_mlp_loss_grad_d", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.POINTER(McMlpDloss), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_mlp_train_d", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.POINTER(McMlpDloss), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_float, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("mc_philox_words", ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_normals", ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    ("mc_price_gbm1d_noalloc", ctypes.c_int, [ctypes.POINTER(McModel), ctypes.POINTER(McSimCfg),
                                              ctypes.POINTER(McPayoff), ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_void_p]),
]

_lib = None


class MCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib(build: bool = True):
    """Load libgbmc.so (building it first if needed and `build` is true)."""
    global _lib
    if _lib is not None:
        return _lib
    if build and not os.environ.get("GBMC_LIBRARY"):
        from . import build as _build
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"the CUDA library {LIB_PATH} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(rc: int):
    if rc != MC_OK:
        raise MCError(rc, lib(build=False).mc_last_error().decode())
