"""The multi-rank path of the benchmark on CPU (gloo, world size 2): every rank runs its own
replica of the workload; the job time is the slowest rank's and the value counts every
rank's receiver-steps (weak scaling, no data collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                      # the second replica is slower
    ms_max = bench.slowest_rank_ms(ms, dist, torch.device("cpu"))
    value = bench.weak_scaling_value(1_000_000, world, ms_max)
    q.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_report_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms_max, value in out:
        assert ms_max == 15.0
        assert value == pytest.approx(2 * 1_000_000 / 0.015)


def test_single_process_is_unchanged():
    import bench
    assert bench.slowest_rank_ms(12.5) == 12.5
    assert bench.weak_scaling_value(10, 1, 1000.0) == 10.0
