"""Multi-process host logic of the risk workload on the CPU (world size 2,
gloo): the scenario-sharded PnL gather and its tail statistics against the
oracle's VaR / CVaR, and data-parallel Adam training of the surrogate (each
rank a slice of every global batch, one gradient all-reduce per step) against
single-process full-batch training, with the FP64 oracle network standing in
for each rank's GPU."""
import socket

import numpy as np

from paper_1906_02818_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


N_SCEN = 10_001


def _global_pnl():
    return np.random.default_rng(5).standard_normal(N_SCEN) * 26.0 + 3.0


class OracleNet:
    """The network on the FP64 oracle: loss_grad / apply_grad as gb.Mlp."""

    def __init__(self, flat, sizes):
        from oracle import mlp as omlp
        self.omlp, self.sizes = omlp, sizes
        self.P = omlp.unpack(flat.astype(np.float64), sizes)
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in self.P]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in self.P]
        self.step = 0

    def loss_grad(self, x, t):
        loss, G = self.omlp.loss_and_grads(self.P, x, t)
        return loss, self.omlp.pack(G)

    def apply_grad(self, g, lr):
        self.step += 1
        G = self.omlp.unpack(np.asarray(g, dtype=np.float64), self.sizes)
        self.P, self.m, self.v = self.omlp.adam_step(self.P, G, self.m, self.v, self.step, lr)


def _data(n):
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, size=(n, 3))
    return x, np.sin(x[:, 0]) + x[:, 1] * x[:, 2]


def _init(sizes):
    rng = np.random.default_rng(11)
    from oracle import mlp as omlp
    return omlp.pack([(rng.normal(0, 1 / np.sqrt(i), size=(i, o)), np.zeros(o)) for i, o in zip(sizes, sizes[1:])])


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    off, cnt = shard.shard_range(rank, world, N_SCEN)
    pnl = shard.gather_ordered(_global_pnl()[off:off + cnt])
    stats = shard.tail_statistics(pnl, 0.99)
    sizes = [3, 16, 16, 1]
    net = OracleNet(_init(sizes), sizes)
    x, t = _data(512)
    xs, ts = x[rank::world], t[rank::world]  # this rank's rows: global batch s = rows of both ranks' slices s
    loss = shard.dp_train(net, xs, ts, epochs=2, batch=64, lr=1e-2)
    q.put((rank, pnl, stats, net.omlp.pack(net.P), loss))
    dist.destroy_process_group()


def test_two_rank_risk_gather_and_data_parallel_training():
    import torch.multiprocessing as mp
    from oracle import risk as orisk
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = {}
    for _ in range(2):
        r, *rest = q.get(timeout=300)
        got[r] = rest
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = _global_pnl()
    var, cvar, nt = orisk.var_cvar(full, 0.99)
    for r in range(2):
        pnl, stats, params, _ = got[r]
        assert np.array_equal(pnl, full)
        assert stats[0] == var and stats[2] == nt and abs(stats[1] - cvar) <= 1e-12 * abs(cvar)
    # single process: the same global batches (rank 0 rows, then rank 1 rows of each slice), full-batch gradient
    sizes = [3, 16, 16, 1]
    ref = OracleNet(_init(sizes), sizes)
    x, t = _data(512)
    x0, t0, x1, t1 = x[0::2], t[0::2], x[1::2], t[1::2]
    for _ in range(2):
        for s in range(256 // 32):
            xb = np.concatenate([x0[s * 32:(s + 1) * 32], x1[s * 32:(s + 1) * 32]])
            tb = np.concatenate([t0[s * 32:(s + 1) * 32], t1[s * 32:(s + 1) * 32]])
            _, g = ref.loss_grad(xb, tb)
            ref.apply_grad(g, 1e-2)
    want = ref.omlp.pack(ref.P)
    for r in range(2):
        assert np.max(np.abs(got[r][2] - want)) <= 1e-9 * np.max(np.abs(want))
    assert np.array_equal(got[0][2], got[1][2])


def test_tail_statistics_matches_oracle_rule():
    from oracle import risk as orisk
    rng = np.random.default_rng(1)
    for n, alpha in [(1, 0.99), (3, 0.5), (1000, 0.99), (4096, 0.95), (65536, 0.99)]:
        pnl = np.round(rng.standard_normal(n) * 10.0, 1)  # ties on purpose
        a = shard.tail_statistics(pnl, alpha)
        b = orisk.var_cvar(pnl, alpha)
        assert a[0] == b[0] and a[2] == b[2] and abs(a[1] - b[1]) <= 1e-12 * max(1.0, abs(b[1]))
