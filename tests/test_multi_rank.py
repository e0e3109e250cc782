"""The multi-GPU path of the benchmark on the CPU: independent replicas, one
stream per rank, no collective on the data path; the job's throughput is
the units of all ranks over the slowest rank's time.  Two gloo ranks run the
same aggregation helpers bench.py uses under torchrun (NCCL there)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.barrier(world)
        # rank r processed (r + 1) * 1e9 units in (r + 1) * 100 ms
        value, ms_max = bench.weak_scaling_value(world, (rank + 1) * 1e9, (rank + 1) * 100.0)
        total = bench.sum_over_ranks(world, rank + 1)
        worst = bench.max_over_ranks(world, -rank)
        out.put((rank, value, ms_max, total, worst, bench.stream_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate_as_weak_scaling():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_rank_main, args=(world, _free_port(), q), nprocs=world, join=True,
                       start_method="spawn")
    res = sorted(q.get() for _ in range(world))
    for rank, value, ms_max, total, worst, seed in res:
        assert ms_max == 200.0                       # the slowest rank's time
        assert value == pytest.approx(3e9 / 0.2 / 1e9)  # all units over that time
        assert total == 3 and worst == 0
    assert res[0][5] != res[1][5]                    # each replica its own stream


def test_single_process_needs_no_process_group():
    import bench
    value, ms = bench.weak_scaling_value(1, 5e9, 250.0)
    assert ms == 250.0 and value == pytest.approx(20.0)
    assert bench.max_over_ranks(1, 3.0) == 3.0 and bench.sum_over_ranks(1, 3.0) == 3.0
