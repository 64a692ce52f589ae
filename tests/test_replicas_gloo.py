"""The multi-process bench path on the CPU: two ranks over gloo (one process per
GPU on the GPU machine, replicas with no collective on the data path) agree on the
slowest rank's time, and the whole-job rate counts both ranks' units over it."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 3.0 * rank, world, device="cpu")
    rate = bench.whole_job_rate(world, 5, t)
    dist.barrier()
    q.put((rank, t, rate))
    dist.destroy_process_group()


def test_two_rank_timing_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == [0, 1]
    for _, t, rate in out:
        assert t == 13.0                     # the slower rank's time on both ranks
        assert rate == pytest.approx(2 * 5 / 13.0)


def test_single_rank_is_local():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0
