"""Multi-process host logic of the risk workload on the CPU (world size 2,
gloo): the scenario-sharded PnL gather (rank order, ragged slices), and
data-parallel Adam training of the surrogate (each
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
    """The network on the FP64 oracle with gb.Mlp's data-parallel interface
    (loss_grad_sums / apply_grad_sums on host float64 tensors, the gloo
    group's device)."""

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

    def loss_grad_sums(self, x, t):
        import torch
        loss, g = self.loss_grad(x, t)  # mean loss and its gradient
        n = len(t)
        return torch.from_numpy(np.append(n * g, n * loss))

    def apply_grad_sums(self, buf, scale, lr):
        self.apply_grad(buf.numpy()[:-1] * scale, lr)


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
    pnl = shard.gather_ordered(_global_pnl()[off:off + cnt]).numpy()
    sizes = [3, 16, 16, 1]
    net = OracleNet(_init(sizes), sizes)
    x, t = _data(512)
    xs, ts = x[rank::world], t[rank::world]  # this rank's rows: global batch s = rows of both ranks' slices s
    loss = shard.dp_train(net, xs, ts, epochs=2, batch=64, lr=1e-2)
    q.put((rank, pnl, net.omlp.pack(net.P), loss))
    dist.destroy_process_group()


def test_two_rank_risk_gather_and_data_parallel_training():
    import torch.multiprocessing as mp
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
    for r in range(2):
        pnl, params, _ = got[r]
        assert np.array_equal(pnl, full)
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
        assert np.max(np.abs(got[r][1] - want)) <= 1e-9 * np.max(np.abs(want))
    assert np.array_equal(got[0][1], got[1][1])
