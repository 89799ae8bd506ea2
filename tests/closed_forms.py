"""Textbook closed forms used to pin the oracle (and, through it, the CUDA path).

Each is written from its mathematical definition, independently of the
oracle's code.  None of them is used by the library.
"""
from __future__ import annotations

from math import erf, exp, log, pi, sqrt

import numpy as np


def ncdf(x: float) -> float:
    return 0.5 * (1.0 + erf(x / sqrt(2.0)))


def npdf(x: float) -> float:
    return exp(-0.5 * x * x) / sqrt(2.0 * pi)


def bs_d1d2(S, K, r, sigma, T):
    d1 = (log(S / K) + (r + 0.5 * sigma * sigma) * T) / (sigma * sqrt(T))
    return d1, d1 - sigma * sqrt(T)


def bs_call(S, K, r, sigma, T):
    d1, d2 = bs_d1d2(S, K, r, sigma, T)
    return S * ncdf(d1) - K * exp(-r * T) * ncdf(d2)


def bs_put(S, K, r, sigma, T):
    d1, d2 = bs_d1d2(S, K, r, sigma, T)
    return K * exp(-r * T) * ncdf(-d2) - S * ncdf(-d1)


def bs_call_greeks(S, K, r, sigma, T):
    """(delta, vega = d/dsigma, rho = d/dr) of the Black-Scholes call."""
    d1, d2 = bs_d1d2(S, K, r, sigma, T)
    return ncdf(d1), S * npdf(d1) * sqrt(T), K * T * exp(-r * T) * ncdf(d2)


def lognormal_call(mu, s2, K):
    """E[(e^Y - K)^+] for Y ~ N(mu, s2)."""
    s = sqrt(s2)
    d2 = (mu - log(K)) / s
    return exp(mu + 0.5 * s2) * ncdf(d2 + s) - K * ncdf(d2)


def geometric_asian_call(S, K, r, sigma, T, M):
    """Discrete geometric-average call, average of S(t_i) at t_i = iT/M,
    i = 1..M (Kemna-Vorst with discrete monitoring): log G is normal with
    mean log S + (r - sigma^2/2) T (M+1)/(2M) and variance
    sigma^2 T (M+1)(2M+1)/(6 M^2)."""
    mu = log(S) + (r - 0.5 * sigma * sigma) * T * (M + 1) / (2.0 * M)
    s2 = sigma * sigma * T * (M + 1) * (2 * M + 1) / (6.0 * M * M)
    return exp(-r * T) * lognormal_call(mu, s2, K)


def geometric_basket_call(s0, sigma, corr, w, K, r, T):
    """Call on prod S_a(T)^{w_a} (sum w = 1) for correlated GBM: the log is
    normal with mean sum w_a (log S0_a + (r - sigma_a^2/2) T) and variance
    T w^T Sigma w, Sigma = diag(sigma) corr diag(sigma)."""
    s0, sigma, w = map(np.asarray, (s0, sigma, w))
    cov = np.diag(sigma) @ np.asarray(corr) @ np.diag(sigma)
    mu = float(np.sum(w * (np.log(s0) + (r - 0.5 * sigma ** 2) * T)))
    s2 = float(T * w @ cov @ w)
    return exp(-r * T) * lognormal_call(mu, s2, K)


def one_step_up_and_out_call(S, K, H, r, sigma, T):
    """Up-and-out call monitored only at T (H > K): payoff
    (S_T - K) 1{K < S_T < H} = (S_T - K)^+ - (S_T - H)^+ - (H - K) 1{S_T >= H}."""
    _, d2H = bs_d1d2(S, H, r, sigma, T)
    return bs_call(S, K, r, sigma, T) - bs_call(S, H, r, sigma, T) - (H - K) * exp(-r * T) * ncdf(d2H)


def up_and_in_put_continuous(S, K, H, r, sigma, T):
    """Continuously monitored up-and-in put, no dividends, S < H, K <= H
    (reflection principle: the put that knocks in equals the image term)."""
    mu = (r - 0.5 * sigma * sigma) / (sigma * sigma)
    sT = sigma * sqrt(T)
    y1 = log(H * H / (S * K)) / sT + (1.0 + mu) * sT
    # phi = -1 (put), eta = -1 (up barrier)
    return (-S * (H / S) ** (2.0 * (mu + 1.0)) * ncdf(-y1)
            + K * exp(-r * T) * (H / S) ** (2.0 * mu) * ncdf(-y1 + sT))


def down_and_in_call_continuous(S, K, H, r, sigma, T):
    """Continuously monitored down-and-in call, no dividends, H < S, H <= K
    (reflection principle, the image of the call in the barrier)."""
    mu = (r - 0.5 * sigma * sigma) / (sigma * sigma)
    sT = sigma * sqrt(T)
    y1 = log(H * H / (S * K)) / sT + (1.0 + mu) * sT
    return (S * (H / S) ** (2.0 * (mu + 1.0)) * ncdf(y1)
            - K * exp(-r * T) * (H / S) ** (2.0 * mu) * ncdf(y1 - sT))


def heston_call(S, K, r, T, v0, kappa, theta, xi, rho):
    """Heston (1993) European call by Fourier inversion:
    C = S P1 - K e^{-rT} P2, P_j = 1/2 + (1/pi) int_0^inf Re[e^{-i u ln K}
    f_j(u) / (i u)] du, with the characteristic functions written in the
    rotation-free form (Albrecher et al., 'The little Heston trap')."""
    from scipy.integrate import quad
    x = np.log(S)

    def f(u, j):
        b = kappa - rho * xi if j == 1 else kappa
        uj = 0.5 if j == 1 else -0.5
        a = kappa * theta
        d = np.sqrt((rho * xi * 1j * u - b) ** 2 - xi * xi * (2 * uj * 1j * u - u * u))
        g = (b - rho * xi * 1j * u - d) / (b - rho * xi * 1j * u + d)
        e = np.exp(-d * T)
        C = r * 1j * u * T + a / (xi * xi) * ((b - rho * xi * 1j * u - d) * T - 2.0 * np.log((1 - g * e) / (1 - g)))
        D = (b - rho * xi * 1j * u - d) / (xi * xi) * (1 - e) / (1 - g * e)
        return np.exp(C + D * v0 + 1j * u * x)

    def P(j):
        integrand = lambda u: (np.exp(-1j * u * np.log(K)) * f(u, j) / (1j * u)).real
        val, _ = quad(integrand, 1e-10, 200.0, limit=400)
        return 0.5 + val / np.pi

    return S * P(1) - K * np.exp(-r * T) * P(2)
