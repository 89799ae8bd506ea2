"""gbmc: GB300-native financial Monte Carlo (Belletti et al., 2019, the
data-parallel path: Philox normals, correlated Euler / log-Euler steps, path
payoffs, FP64-finished estimator with standard errors).

The compute path is the CUDA library libgbmc.so (C ABI in include/mc.h); this
package is its thin binding.  Importing it does not load CUDA; the first call
loads the library and raises if it is missing.
"""
from .native import MCError, PAYOFF, PRECISION, SCHEME  # noqa: F401


def __getattr__(name):
    if name in ("price", "price_mlmc", "price_qmc", "simulate", "greeks", "corr_greeks", "Plan", "Mlp", "risk",
                "surrogate_labels", "surrogate_label_greeks", "philox_words", "normals", "moments", "combine", "tail"):
        from . import api
        return getattr(api, name)
    if name in ("HestonPricer", "GbmPricer", "BasketPricer"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
