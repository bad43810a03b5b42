"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own run
time; the whole-job throughput uses the slowest rank (max over ranks)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [2.0, 5.0][rank]               # rank 1 is the slow one
    value, total = bench.rank_aggregate(local, 1000, 10, world)
    out[rank] = (value, total)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, total = res[r]
        assert total == 5.0
        assert value == pytest.approx(2 * 1000 * 10 / 5.0)


def test_single_rank_needs_no_collective():
    import bench
    value, total = bench.rank_aggregate(4.0, 100, 3, 1)
    assert total == 4.0 and value == pytest.approx(75.0)


# --- the particle-sharded single run (paper_1108_1954_gb300.shard) ----------

class _OracleShardRun:
    """A stand-in for one rank's run on the CPU: its particles are float32
    cell coordinates, its push moves them all by a fixed step and deposits
    them with the oracle's fixed-point deposit into a CPU int64 density, its
    solve records the density it consumed.  Every call is logged."""

    def __init__(self, u, ng, sort_interval):
        import numpy as np
        self.np = np
        self.u = u.copy()
        self.ng = ng
        self.step = 0
        self.log = []
        self.consumed = []
        self.rho = torch.zeros(ng, dtype=torch.int64)
        self.pending = False

        class P:
            pass
        self.p = P()
        self.p.sort_interval = sort_interval

    def _deposit(self):
        import oracle as O
        self.rho += torch.from_numpy(O.deposit_fixed(self.ng, self.u))

    def set_shard(self, n):
        self.log.append(("shard", n))

    def density(self):
        return self.rho

    def init(self, x, v):
        self.log.append("init")
        self.rho.zero_()
        self._deposit()
        self.rho.zero_()                     # pic_init's own solve consumes it

    def deposit(self):
        self.log.append("deposit")
        self.rho.zero_()
        self._deposit()

    def sort(self):
        self.log.append("sort")

    def push(self):
        self.log.append("push")
        np = self.np
        self.u = np.mod(self.u + np.float32(0.37), np.float32(self.ng)).astype(np.float32)
        self._deposit()
        self.pending = True

    def solve_field(self):
        self.log.append("solve")
        self.consumed.append(self.rho.clone())
        self.rho.zero_()
        if self.pending:
            self.step += 1
            self.pending = False


def _shard_rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    from paper_1108_1954_gb300 import shard
    n, ng, S = 10007, 64, 2
    u = np.random.default_rng(5).uniform(0, ng, n).astype(np.float32)
    lo, hi = shard.split(n, world, rank)
    run = _OracleShardRun(u[lo:hi], ng, S)
    sh = shard.Shard(run.p, n, shard.torch_allreduce(), run=run)
    sh.init(None, None)
    sh.step_n(5)
    out[rank] = ([t.numpy().tolist() for t in run.consumed], run.log)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_shards_solve_the_whole_density():
    # Each of two ranks deposits its half of the particles; the int64
    # all-reduce gives both the density of all of them bit for bit, at the
    # start and at every step, and each step runs sort (when due), push,
    # all-reduce, solve in that order.
    import numpy as np
    import oracle as O
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    n, ng = 10007, 64
    u = np.random.default_rng(5).uniform(0, ng, n).astype(np.float32)
    want = [O.deposit_fixed(ng, u).tolist()]
    for _ in range(5):
        u = np.mod(u + np.float32(0.37), np.float32(ng)).astype(np.float32)
        want.append(O.deposit_fixed(ng, u).tolist())
    for r in (0, 1):
        consumed, log = res[r]
        assert consumed == want
        assert log[0] == ("shard", n)
        assert log[1:4] == ["init", "deposit", "solve"]
        steps = log[4:]
        assert steps == ["push", "solve", "push", "solve", "sort", "push", "solve",
                         "push", "solve", "sort", "push", "solve"]
