"""torch.autograd.Function wrappers: prices in the forward pass (mc_price),
pathwise Greeks from the library's adjoint kernels in the backward pass
(mc_greeks).  Gradients flow to the model parameters; inputs and outputs are
float64 CPU tensors (the library returns host results).

  HestonPricer.apply(params, cfg, payoffs)
      params = tensor [7]: (s0, v0, r, kappa, theta, xi, rho)
  GbmPricer.apply(params, cfg, payoffs)
      params = tensor [3]: (s0, sigma, r)  (single asset, log-Euler)
Both return the tensor [n_payoff] of discounted prices.
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
