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


def basket_market_factors(d: int, k: int, seed: int = SEED, ridge: float = 0.05):
    """The market of basket_market(d, k, seed) (same draws, same order) with
    its correlation given by factor loadings: rho = B B^T + diag(e^2),
    B_aj = F_aj / sqrt(k C_aa), e_a^2 = ridge / C_aa, C = F F^T / k + ridge I.
    Returns (s0, sigma, B [d, k])."""
    rng = np.random.default_rng(seed)
    s0 = rng.uniform(50.0, 150.0, size=d)
    sigma = rng.uniform(0.1, 0.4, size=d)
    F = rng.standard_normal((d, k))
    caa = (F * F).sum(axis=1) / k + ridge
    return s0, sigma, F / np.sqrt(k * caa)[:, None]


def basket_d512_factor(paths: int = 1 << 20, steps: int = 252, d: int = 512, k: int = 16):
    """The d = 512 market of basket_d512 with its 16-factor correlation given
    by loadings (factor-model simulation): ATM arithmetic basket call."""
    s0, sigma, B = basket_market_factors(d, k)
    w = np.full(d, 1.0 / d)
    b0 = float(w @ s0)
    return dict(s0=s0, sigma=sigma, loadings=B, weights=w, r=0.05, T=1.0, steps=steps, paths=paths, seed=SEED,
                payoffs=[dict(kind="call", strike=b0)])


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


def mlp_init(n_in: int = 5, width: int = 256, hidden: int = 4, seed: int = SEED) -> np.ndarray:
    """Packed initial parameters of the surrogate (per layer W [in x out]
    row-major then b [out]): W ~ N(0, 1/in) (variance-preserving for SiLU
    nets), b = 0; float32."""
    rng = np.random.default_rng(seed)
    sizes = [n_in] + [width] * hidden + [1]
    parts = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        parts.append((rng.standard_normal((a, b)) / np.sqrt(a)).ravel())
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


RISK_K_OVER_S0 = (0.8, 0.9, 1.0, 1.1, 1.2)
RISK_T_DAYS = (63, 126, 252, 504)


def risk_portfolio(n_under: int = 32, per_under: int = 32, seed: int = SEED, barriers: bool = True):
    """1024 options on 32 correlated GBM underlyings (basket_market(32, 4)):
    per underlying, half European calls / puts (K/S0 on {0.8 .. 1.2}, T on
    {63, 126, 252, 504} days), half up-and-out calls (K/S0 on {0.8, 0.9, 1.0},
    H/S0 ~ U[1.2, 1.5], daily monitoring); positions +-1.  With
    barriers=False every option is European."""
    s0, sigma, corr = basket_market(n_under, 4, seed=seed)
    rng = np.random.default_rng(seed + 1)
    under, kind, K, H, T, pos = [], [], [], [], [], []
    for u in range(n_under):
        for j in range(per_under):
            barrier = barriers and j >= per_under // 2
            if barrier:
                k = 4  # up-and-out call
                kk = rng.choice(RISK_K_OVER_S0[:3])
                hh = rng.uniform(1.2, 1.5)
            else:
                k = int(rng.integers(0, 2))  # 0 call, 1 put
                kk = rng.choice(RISK_K_OVER_S0)
                hh = np.inf
            under.append(u)
            kind.append(k)
            K.append(kk * s0[u])
            H.append(hh * s0[u])
            T.append(rng.choice(RISK_T_DAYS) / 252.0)
            pos.append(float(rng.choice([-1.0, 1.0])))
    return dict(s0=s0, sigma=sigma, corr=corr, r=0.05, mu=0.05, under=np.array(under, dtype=np.int32),
                kind=np.array(kind, dtype=np.int32), strike=np.array(K), barrier=np.array(H),
                maturity=np.array(T), position=np.array(pos), horizon=1.0 / 252, steps_per_year=252)


def surrogate_points(n: int, seed: int = SEED + 2) -> np.ndarray:
    """Training points of the surrogate over its parameter box: S/K ~ U[0.5, 1.6],
    sigma ~ U[0.1, 0.4], tau = days / 252 with days ~ U{1..504}, r ~ U[0, 0.08],
    K/H = 0 (European) for half of them, ~ U[0.5, 0.9] for the rest; float32 [n, 5]."""
    rng = np.random.default_rng(seed)
    x = np.empty((n, 5))
    x[:, 0] = rng.uniform(0.5, 1.6, n)
    x[:, 1] = rng.uniform(0.1, 0.4, n)
    x[:, 2] = rng.integers(1, 505, n) / 252.0
    x[:, 3] = rng.uniform(0.0, 0.08, n)
    x[:, 4] = np.where(rng.uniform(size=n) < 0.5, 0.0, rng.uniform(0.5, 0.9, n))
    return x.astype(np.float32)


# Adam learning-rate schedule of the surrogate: (lr, epochs) phases.
SURROGATE_SCHEDULE = ((1e-3, 30), (3e-4, 20), (1e-4, 20))
