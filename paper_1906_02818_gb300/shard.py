"""Path-range sharding across processes (one GPU each).

Paths are independent and the random stream is indexed by the global path
number, so a run over [0, N) splits into contiguous ranges run with
`path_offset` and nothing is exchanged until the end: one all-reduce of
(n * mean, n * second moment, n) per payoff combines the ranges into the
estimator of Eq. 3 and its standard error, as if one device had run them.
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


def moments(results, n: int) -> np.ndarray:
    """Per payoff [n * mean, n * mean(f^2), n] (discounted units) from the
    (price, se) pairs of a run over n paths."""
    out = np.zeros((len(results), 3))
    for i, (m, se) in enumerate(results):
        m2 = se * se * (n - 1) + m * m if n > 1 else m * m
        out[i] = (n * m, n * m2, n)
    return out


def combine(mom: np.ndarray):
    """(price, se) per payoff from summed moments."""
    res = []
    for s, s2, n in mom:
        m = s / n
        var = max(s2 / n - m * m, 0.0)
        res.append((m, float(np.sqrt(var / (n - 1))) if n > 1 else 0.0))
    return res


def allreduce_results(results, n: int, group=None, device=None):
    """Combine this rank's (price, se) list over n paths with every other
    rank's through one torch.distributed all-reduce (float64)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(moments(results, n), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return combine(t.cpu().numpy())


# ----------------------------- portfolio risk ------------------------------
# Outer scenarios are independent and indexed globally (mc_risk_cfg
# scen_offset), so each rank revalues a contiguous slice; the PnL vector
# (8 bytes per scenario) is gathered and the tail statistics are taken on it.

def gather_ordered(local: np.ndarray, group=None) -> np.ndarray:
    """Concatenation of every rank's 1-D float64 array in rank order (the
    slices may differ in length by one)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([local.size], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    m = int(max(s.item() for s in sizes))
    buf = torch.zeros(m, dtype=torch.float64)
    buf[:local.size] = torch.from_numpy(np.ascontiguousarray(local, dtype=np.float64))
    parts = [torch.zeros(m, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return np.concatenate([p[:int(s.item())].numpy() for p, s in zip(parts, sizes)])


def tail_statistics(pnl: np.ndarray, alpha: float):
    """(VaR, CVaR, n_tail) of the loss -PnL (Sec. VI.B): VaR is the k-th
    largest loss, k = ceil((1 - alpha) n); CVaR the mean of the losses strictly
    above it (VaR itself when there are none)."""
    loss = -np.asarray(pnl, dtype=np.float64)
    n = loss.size
    k = min(n, max(1, int(np.ceil((1.0 - alpha) * n - 1e-9))))
    var = float(np.partition(loss, n - k)[n - k])  # k-th largest
    above = loss[loss > var]
    return var, (float(above.mean()) if above.size else var), int(above.size)


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
    return dict(var=var, cvar=cvar, n_tail=nt, pnl=pnl, base_value=local["base_value"])


# -------------------------- surrogate training -----------------------------
# Data-parallel mini-batch Adam: every rank holds the same parameters and its
# own slice of each global batch; the batch gradient of the mean loss is the
# size-weighted average of the ranks' gradients (one all-reduce of ~0.2 M
# floats per step), after which every rank applies the same Adam step.

def allreduce_grad(g: np.ndarray, n_local: int, group=None) -> np.ndarray:
    """sum_r n_r g_r / sum_r n_r over the ranks (float64 reduction)."""
    import torch
    import torch.distributed as dist
    t = torch.zeros(g.size + 1, dtype=torch.float64)
    t[:-1] = torch.from_numpy(np.asarray(g, dtype=np.float64).ravel() * n_local)
    t[-1] = float(n_local)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return (t[:-1] / t[-1]).numpy().astype(g.dtype)


def dp_train(net, x_local, t_local, epochs: int, batch: int, lr: float, group=None):
    """Train `net` (gb.Mlp or anything with loss_grad(x, t) -> (loss, grad)
    and apply_grad(grad, lr)) on the union of the ranks' data: the global
    batch of `batch` samples takes batch / world rows from every rank's slice
    in order.  Returns the mean global-batch loss of the last epoch."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    b = batch // world
    steps = len(t_local) // b
    last = 0.0
    for _ in range(epochs):
        tot = 0.0
        for s in range(steps):
            xs, ts = x_local[s * b:(s + 1) * b], t_local[s * b:(s + 1) * b]
            loss, g = net.loss_grad(xs, ts)
            gsum = allreduce_grad(np.append(g, loss).astype(np.float64), b, group)
            net.apply_grad(gsum[:-1].astype(np.asarray(g).dtype), lr)  # the net's own gradient type
            tot += float(gsum[-1])
        last = tot / max(steps, 1)
    return last
