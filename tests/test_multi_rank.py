"""The multi-rank paths on CPU (gloo, world size 2): the job time is the slowest rank's and
the value counts every rank's receiver-steps; and the receiver split -- balanced ranges of
points, bands of grid rows with the parent's FP32 cell centres, results gathered on rank
0 in rank order -- reassembles the single-rank layout."""
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


def _shard_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    from paper_1907_04435_gb300 import shard
    # each rank's "results" are the global receiver indices of its share, as a library
    # call on its own receivers would return them in its own (input) order
    grid = (0.0, 0.0, 1.0, 37, 23)
    x0, y0, dx, nx, rows, r0 = shard.grid_band(grid, rank, world)
    ground = (r0 * nx + np.arange(rows * nx)).astype(np.int64)
    a, b = shard.split(101, rank, world)
    facades = np.arange(a, b, dtype=np.int64)
    got = shard.gather_to_root([ground, facades], dist)
    q.put((rank, None if got is None else [g.tolist() for g in got]))
    dist.barrier()
    dist.destroy_process_group()


def test_receiver_split_gathers_to_the_single_rank_layout():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[1] is None
    ground, facades = out[0]
    assert ground == list(range(37 * 23)) and facades == list(range(101))


def test_split_and_grid_bands():
    import numpy as np
    from paper_1907_04435_gb300 import shard
    for n in (0, 1, 7, 100, 4194304):
        for world in (1, 2, 3, 8):
            parts = [shard.split(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    # the district's grid splits exactly; bands of a 0.7 m grid from an odd origin would
    # not keep the parent's FP32 centres and are refused
    bands = [shard.grid_band((0.0, 0.0, 1.0, 2048, 2048), r, 8) for r in range(8)]
    assert sum(b[4] for b in bands) == 2048 and bands[3][1] == 768.0
    with pytest.raises(ValueError):
        [shard.grid_band((-3.3, -2.1, 0.7, 101, 77), r, 3) for r in range(3)]
