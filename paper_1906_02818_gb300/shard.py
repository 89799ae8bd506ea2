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
