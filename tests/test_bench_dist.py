"""The multi-rank path of bench.py (independent replicas, one per GPU): the
timing aggregation takes the slowest rank and sums the work of all ranks.
Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate(10.0 + 5.0 * rank, 1000, 20, world, "cpu")
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0  # the slower rank's 15 ms
        assert abs(value - 1000 * 20 * 2 / 15e-3) < 1e-6 * value


def test_single_rank_aggregation_is_identity():
    import bench
    ms, value = bench.aggregate(4.0, 100, 10, 1, "cpu")
    assert ms == 4.0 and abs(value - 100 * 10 / 4e-3) < 1e-9
