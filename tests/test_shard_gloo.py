"""Multi-process path sharding on the CPU (world size 2, gloo): each rank
prices its contiguous path range with the oracle (standing in for its GPU),
one all-reduce combines the moments, and the result equals the single-run
estimator over the whole range."""
import os
import socket

import numpy as np
import pytest

from paper_1906_02818_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    pays = [dict(kind="call", strike=100.0), dict(kind="asian_put", strike=105.0)]
    N = 10_001
    off, cnt = shard.shard_range(rank, world, N)
    per = oracle.gbm_payoffs(100.0, 0.25, 0.05, 1.0, 16, cnt, pays, path_offset=off)
    res = [oracle.mean_se(row) for row in per]
    q.put((rank, shard.allreduce_results(res, cnt)))
    dist.destroy_process_group()


def test_shard_range_covers_exactly():
    for N in (1, 7, 1000, 10_001):
        for W in (1, 2, 3, 8):
            r = [shard.shard_range(k, W, N) for k in range(W)]
            assert r[0][0] == 0 and sum(c for _, c in r) == N
            assert all(r[k][0] + r[k][1] == r[k + 1][0] for k in range(W - 1))
            assert max(c for _, c in r) - min(c for _, c in r) <= 1


def test_two_rank_gloo_combine_equals_single_run(orc):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    pays = [dict(kind="call", strike=100.0), dict(kind="asian_put", strike=105.0)]
    full = orc.gbm_payoffs(100.0, 0.25, 0.05, 1.0, 16, 10_001, pays)
    for i in range(2):
        m, se = orc.mean_se(full[i])
        for r in range(2):
            assert abs(got[r][i][0] - m) <= 1e-12 * abs(m)
            assert abs(got[r][i][1] - se) <= 1e-9 * se


def test_moments_and_combine_through_the_library(orc):
    """mc_moments / mc_combine (host code of the library, no device): three
    disjoint path ranges of one stream combine into the single-range
    estimator and standard error; non-finite input is rejected."""
    from paper_1906_02818_gb300 import api, native
    pays = [dict(kind="call", strike=100.0), dict(kind="put", strike=90.0)]
    cuts = [0, 1, 4000, 10_001]
    tot = np.zeros((len(pays), 3))
    for a, b in zip(cuts, cuts[1:]):
        per = orc.gbm_payoffs(100.0, 0.25, 0.05, 1.0, 16, b - a, pays, path_offset=a)
        tot += api.moments([orc.mean_se(row) for row in per], b - a)
    got = api.combine(tot)
    full = orc.gbm_payoffs(100.0, 0.25, 0.05, 1.0, 16, 10_001, pays)
    for i in range(len(pays)):
        m, se = orc.mean_se(full[i])
        assert abs(got[i][0] - m) <= 1e-12 * abs(m) and abs(got[i][1] - se) <= 1e-9 * se
    with pytest.raises(native.MCError):
        api.moments([(float("nan"), 1.0)], 10)
    with pytest.raises(native.MCError):
        api.combine(np.array([[1.0, 2.0, 0.0]]))


def test_data_parallel_training_needs_a_sample_per_rank():
    """A global batch smaller than the world leaves a rank nothing to train
    on: refused before any collective (one-rank gloo group)."""
    import torch.distributed as dist
    if dist.is_initialized():
        pytest.skip("a process group is already initialised in this process")
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1)
    try:
        with pytest.raises(ValueError, match="no sample"):
            shard.dp_train(object(), np.zeros((4, 5)), np.zeros(4), epochs=1, batch=0, lr=1e-3)
    finally:
        dist.destroy_process_group()
