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
