"""The benchmark's N > 1 path without GPUs: two gloo ranks on the CPU exchange their
timings; every rank sees the slowest rank's time and the whole-job throughput counts
the paths of all ranks (weak scaling, no data-path collective)."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench._env_rank()
    t = bench.max_over_ranks(100.0 + 50.0 * rank, w)     # rank 1 is the slow one
    v = bench.weak_scaling_value(1000, w, 10, t)
    dist.barrier()
    q.put((r, w, t, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
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
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 150.0 for o in out)
    assert all(o[3] == pytest.approx(1000 * 2 * 10 / 0.150) for o in out)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.weak_scaling_value(100, 1, 4, 400.0) == pytest.approx(1000.0)
