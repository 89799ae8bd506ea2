"""Seeded synthetic inputs for the Monte Carlo workloads.

This module only draws and shapes input data (spot prices, volatilities,
factor-model correlation matrices, strike grids, portfolios, parameter points).
It holds none of the method's arithmetic: no random-number stream of the
simulation, no Cholesky factor, no time step, no payoff.  Both the CUDA path and
the oracle take their inputs from here.

The paper's basket, VaR and QMC experiments use a historical Russell-3000
covariance that is not available (Sec. VI.A.2, VI.B.1); the seeded factor
model below stands in for it with the same shapes (ATM baskets of correlated
names priced near 100, r = 0.05).
"""
from __future__ import annotations

import numpy as np

SEED = 42


def factor_correlation(d: int, k: int, rng: np.random.Generator, ridge: float = 0.05) -> np.ndarray:
    """Correlation matrix from a k-factor model plus ridge*I, normalised to a
    unit diagonal: C = F F^T / k + ridge I, rho = D^-1/2 C D^-1/2 (PSD, in
    fact positive definite because of the ridge)."""
    F = rng.standard_normal((d, k))
    C = F @ F.T / k + ridge * np.eye(d)
    s = 1.0 / np.sqrt(np.diag(C))
    rho = C * s[:, None] * s[None, :]
    np.fill_diagonal(rho, 1.0)
    return rho


def basket_market(d: int, k: int, seed: int = SEED):
    """Spot prices S0 ~ U[50, 150], vols ~ U[0.1, 0.4] and a k-factor
    correlation, drawn in that order from numpy's PCG64 with `seed`."""
    rng = np.random.default_rng(seed)
    s0 = rng.uniform(50.0, 150.0, size=d)
    sigma = rng.uniform(0.1, 0.4, size=d)
    corr = factor_correlation(d, k, rng)
    return s0, sigma, corr


def gbm_1d(paths: int = 1 << 20, steps: int = 64):
    """Single-asset Black-Scholes GBM, European call at the money."""
    return dict(s0=np.array([100.0]), sigma=np.array([0.2]), corr=None, r=0.05, T=1.0,
                steps=steps, paths=paths, seed=SEED,
                payoffs=[dict(kind="call", strike=100.0)])


def basket_d64(paths: int = 1 << 18, steps: int = 252, d: int = 64, k: int = 4):
    """Correlated GBM basket: equal weights, ATM basket call K = sum w S0 and
    an up-and-out basket call knocked out when the basket value reaches
    1.3 times its initial value, monitored at every step."""
    s0, sigma, corr = basket_market(d, k)
    w = np.full(d, 1.0 / d)
    b0 = float(w @ s0)
    return dict(s0=s0, sigma=sigma, corr=corr, weights=w, r=0.05, T=1.0, steps=steps,
                paths=paths, seed=SEED,
                payoffs=[dict(kind="call", strike=b0),
                         dict(kind="uo_call", strike=b0, barrier=1.3 * b0)])


def basket_d512(paths: int = 1 << 20, steps: int = 252, d: int = 512, k: int = 16):
    """Large correlated basket: ATM arithmetic basket call."""
    s0, sigma, corr = basket_market(d, k)
    w = np.full(d, 1.0 / d)
    b0 = float(w @ s0)
    return dict(s0=s0, sigma=sigma, corr=corr, weights=w, r=0.05, T=1.0, steps=steps,
                paths=paths, seed=SEED, payoffs=[dict(kind="call", strike=b0)])


HESTON_PARAMS = dict(s0=100.0, v0=0.04, r=0.05, kappa=2.0, theta=0.04, xi=0.5, rho=-0.7)
HESTON_STRIKES = tuple(float(k) for k in range(80, 121, 5))


def heston(paths: int = 1 << 22, steps: int = 256):
    """Heston model, European and arithmetic-Asian calls on K = 80..120."""
    pays = [dict(kind="call", strike=K) for K in HESTON_STRIKES]
    pays += [dict(kind="asian_call", strike=K) for K in HESTON_STRIKES]
    return dict(model=dict(HESTON_PARAMS), T=1.0, steps=steps, paths=paths, seed=SEED, payoffs=pays)
