"""Host logic of the multi-rank benchmark path, run as two gloo ranks on CPU:
the barriers that bracket the timed region and the max-over-ranks reduction
of the step time (the work split itself is tested in test_shard_cpu.py).
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # each rank's own step time: the job is as slow as the slowest rank
        t_local = 10.0 + 5.0 * rank
        t_max = bench.allmax(t_local, world)
        value = bench.job_value(1000, world, t_max)
        bench.barrier(world)
        q.put((rank, t_local, t_max, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_time_and_job_value():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[2] for o in out] == [15.0, 15.0]                  # every rank sees the max
    assert all(abs(o[3] - 2 * 1000 / 15e-3) < 1e-6 for o in out)  # N x units / max time


def test_single_rank_is_identity():
    import bench
    assert bench.allmax(3.5, 1) == 3.5
    assert bench.job_value(10, 1, 2.0) == 10 / 2e-3
