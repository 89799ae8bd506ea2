"""Path-range sharding across processes (one GPU each).

Paths are independent and the random stream is indexed by the global path
number, so a run over [0, N) splits into contiguous ranges run with
`path_offset` and nothing is exchanged until the end: one all-reduce of
(n * mean, n * second moment, n) per payoff combines the ranges into the
estimator of Eq. 3 and its standard error, as if one device had run them.
The moments and their combination are the library's (mc_moments,
mc_combine); VaR / CVaR of gathered scenario PnLs is the library's device
selection (mc_tail).  This module only moves data: tensors live on the
process group's device (CUDA for NCCL, host memory for gloo).
"""
from __future__ import annotations

import numpy as np


def shard_range(rank: int, world: int, paths: int) -> tuple[int, int]:
    """Contiguous, balanced [offset, offset + count) of rank `rank`."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    base, extra = divmod(paths, world)
    offset = rank * base + min(rank, extra)
    return offset, base + (1 if rank < extra else 0)


def group_device(group=None):
    """The device collectives of `group` run on: the current CUDA device for
    NCCL, the host for gloo."""
    import torch
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def moments(results, n: int) -> np.ndarray:
    """Per payoff [n * mean, n * mean(f^2), n] (discounted units) from the
    (price, se) pairs of a run over n paths (mc_moments)."""
    from . import api
    return api.moments(results, n)


def combine(mom: np.ndarray):
    """(price, se) per payoff from summed moments (mc_combine)."""
    from . import api
    return api.combine(mom)


def allreduce_results(results, n: int, group=None, device=None):
    """Combine this rank's (price, se) list over n paths with every other
    rank's through one torch.distributed all-reduce (float64)."""
    import torch
    import torch.distributed as dist
    dev = device if device is not None else group_device(group)
    t = torch.tensor(moments(results, n), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return combine(t.cpu().numpy())


# ----------------------------- portfolio risk ------------------------------
# Outer scenarios are independent and indexed globally (mc_risk_cfg
# scen_offset), so each rank revalues a contiguous slice; the PnL vector
# (8 bytes per scenario) is gathered and the tail statistics are taken on it.

def gather_ordered(local, group=None):
    """Concatenation of every rank's 1-D float64 tensor (or array) in rank
    order, on the group's device (the slices may differ in length by one)."""
    import torch
    import torch.distributed as dist
    dev = group_device(group)
    x = torch.as_tensor(np.asarray(local) if not torch.is_tensor(local) else local, dtype=torch.float64).to(dev)
    world = dist.get_world_size(group)
    n = torch.tensor([x.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    counts = [int(s.item()) for s in sizes]
    buf = torch.zeros(max(counts), dtype=torch.float64, device=dev)
    buf[:x.numel()] = x
    parts = [torch.zeros(max(counts), dtype=torch.float64, device=dev) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])


def tail_statistics(pnl, alpha: float):
    """(VaR, CVaR, n_tail) of the loss -PnL (Sec. VI.B) by the library's
    device selection (mc_tail) on a CUDA copy of `pnl`."""
    import torch
    from . import api
    r = api.tail(torch.as_tensor(pnl, dtype=torch.float64).cuda(), alpha)
    return r["var"], r["cvar"], r["n_tail"]


def risk_sharded(portfolio, n_scen: int, group=None, **kw):
    """VaR / CVaR over n_scen scenarios revalued by every rank on its slice
    (gb.risk with scen_offset), PnL gathered to every rank.  Returns the dict
    of gb.risk for the whole scenario set (var, cvar, n_tail, pnl)."""
    import torch.distributed as dist
    from . import api
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    off, cnt = shard_range(rank, world, n_scen)
    alpha = kw.get("alpha", 0.99)
    local = api.risk(portfolio, n_scen=cnt, scen_offset=off, want_pnl=True, **kw)
    pnl = gather_ordered(local["pnl"], group)
    var, cvar, nt = tail_statistics(pnl, alpha)
    return dict(var=var, cvar=cvar, n_tail=nt, pnl=pnl.cpu().numpy(), base_value=local["base_value"])


# -------------------------- surrogate training -----------------------------
# Data-parallel mini-batch Adam: every rank holds the same parameters and its
# own slice of each global batch.  Each rank writes the gradient of its
# slice's SUMMED loss and that sum into one device buffer
# (mc_mlp_loss_grad_sums); one all-reduce adds the buffers, and every rank
# applies the same Adam step with the sum scaled by 1 / global batch
# (mc_mlp_apply_grad_sums): the mean gradient of the global batch, without a
# host round trip.

def dp_train(net, x_local, t_local, epochs: int, batch: int, lr: float, group=None):
    """Train `net` (gb.Mlp, or anything with loss_grad_sums(x, t) -> tensor
    [count + 1] and apply_grad_sums(g, scale, lr)) on the union of the ranks'
    data: the global batch of `batch` samples takes batch / world rows from
    every rank's slice in order.  Returns the mean global-batch loss of the
    last epoch."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    b = batch // world
    if b < 1:
        raise ValueError(f"a global batch of {batch} leaves no sample for each of {world} ranks")
    steps = len(t_local) // b
    n_global = b * world
    last = 0.0
    for _ in range(epochs):
        losses = []  # summed losses stay on the device until the epoch ends
        for s in range(steps):
            buf = net.loss_grad_sums(x_local[s * b:(s + 1) * b], t_local[s * b:(s + 1) * b])
            dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
            net.apply_grad_sums(buf, 1.0 / n_global, lr)
            losses.append(buf[-1:])
        if losses:
            import torch
            last = float(torch.cat(losses).double().sum()) / (steps * n_global)
    return last
