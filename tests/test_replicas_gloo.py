"""CPU, two gloo ranks: the replica path of the benchmark takes the slowest
rank's time and counts the units of every rank (weak scaling; the path has
no data exchange, so replicas share nothing but this reduction)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 * (rank + 1)  # rank 1 is the slower replica
    total = bench.max_over_ranks(ms, world, device="cpu")
    rate = bench.whole_job_rate(32.0, world, 10, total)
    q.put((rank, total, rate))
    dist.destroy_process_group()


def test_two_replicas_take_slowest_time_and_sum_units():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, rate in out:
        assert total == 200.0
        assert rate == pytest.approx(2 * 32 * 10 / 0.2)


def test_single_rank_is_identity():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(32, 1, 10, 1000.0) == 320.0
