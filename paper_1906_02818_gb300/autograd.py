"""torch.autograd.Function wrappers: prices in the forward pass (mc_price),
pathwise Greeks from the library's adjoint kernels in the backward pass
(mc_greeks).  Gradients flow to the model parameters; inputs and outputs are
float64 CPU tensors (the library returns host results).

  HestonPricer.apply(params, cfg, payoffs)
      params = tensor [7]: (s0, v0, r, kappa, theta, xi, rho)
  GbmPricer.apply(params, cfg, payoffs)
      params = tensor [3]: (s0, sigma, r)  (single asset, log-Euler)
Both return the tensor [n_payoff] of discounted prices.

  BasketPricer.apply(s0, sigma, r, corr, cfg, payoff, weights=None)
      s0, sigma: [d]; r: []; corr: [d, d] (2 <= d <= 512); one European
      basket call or put, log-Euler, FP32.  Returns the price [].  Backward:
      d/ds0, d/dsigma, d/dr from mc_greeks and d/dcorr from mc_corr_greeks;
      the gradient of a correlation entry pair is split evenly between
      corr[a][b] and corr[b][a] (so a symmetric perturbation of both sees the
      pair's derivative) and the diagonal, fixed at 1, gets 0.
"""
from __future__ import annotations

import torch

from . import api

HESTON_PARAMS = ("s0", "v0", "r", "kappa", "theta", "xi", "rho")
GBM_PARAMS = ("s0", "sigma", "r")


def _heston_model(p):
    v = [float(x) for x in p.detach().cpu().numpy()]
    return dict(kind="heston", **dict(zip(HESTON_PARAMS, v)))


def _gbm_model(p):
    s0, sigma, r = [float(x) for x in p.detach().cpu().numpy()]
    return dict(kind="gbm", s0=[s0], sigma=[sigma], r=r)


def _forward(ctx, model, params, cfg, payoffs):
    res = api.price(model, cfg, payoffs)
    ctx.model, ctx.cfg, ctx.payoffs = model, cfg, payoffs
    ctx.dtype, ctx.device = params.dtype, params.device
    return torch.tensor([r[0] for r in res], dtype=params.dtype, device=params.device)


def _backward(ctx, grad_out):
    _, g = api.greeks(ctx.model, ctx.cfg, ctx.payoffs)  # [n_payoff, G, 2]
    J = torch.tensor(g[:, :, 0], dtype=ctx.dtype, device=ctx.device)
    return grad_out @ J, None, None


class HestonPricer(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, cfg, payoffs):
        return _forward(ctx, _heston_model(params), params, cfg, payoffs)

    @staticmethod
    def backward(ctx, grad_out):
        return _backward(ctx, grad_out)


class GbmPricer(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, cfg, payoffs):
        return _forward(ctx, _gbm_model(params), params, cfg, payoffs)

    @staticmethod
    def backward(ctx, grad_out):
        return _backward(ctx, grad_out)


def _basket_model(s0, sigma, r, corr, weights):
    def arr(t):
        return t.detach().cpu().double().numpy()
    w = arr(weights) if torch.is_tensor(weights) else weights
    return dict(kind="gbm", s0=arr(s0), sigma=arr(sigma), r=float(r), corr=arr(corr), weights=w)


class BasketPricer(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s0, sigma, r, corr, cfg, payoff, weights=None):
        model = _basket_model(s0, sigma, r, corr, weights)
        (p, _), = api.price(model, cfg, [payoff])
        ctx.model, ctx.cfg, ctx.payoff = model, cfg, payoff
        ctx.dtype, ctx.device = s0.dtype, s0.device
        return torch.tensor(p, dtype=s0.dtype, device=s0.device)

    @staticmethod
    def backward(ctx, grad_out):
        d = len(ctx.model["s0"])
        _, g = api.greeks(ctx.model, ctx.cfg, [ctx.payoff])      # [1, 2d + 1, 2]
        _, _, dr = api.corr_greeks(ctx.model, ctx.cfg, ctx.payoff)

        def t(x):
            return torch.as_tensor(x, dtype=ctx.dtype, device=ctx.device) * grad_out
        return (t(g[0, :d, 0]), t(g[0, d:2 * d, 0]), t(g[0, 2 * d, 0]), t(0.5 * dr[..., 0]), None, None, None)
