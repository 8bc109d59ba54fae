"""The multi-rank timing of bench.py on CPU (gloo, two ranks): each rank runs
an independent replica, the job's time is the slowest rank's, and the job's
throughput counts every rank's states (weak scaling)."""

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


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local = [120.0, 150.0][rank]          # rank 1 is the slow one
    ms = bench.job_ms(local, dist, "cpu")
    q.put((rank, ms, bench.job_value(world, 4, 5, ms)))
    dist.destroy_process_group()


def test_job_time_is_slowest_rank_and_value_counts_all_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 150.0
        assert value == pytest.approx(2 * 4 * 5 / 0.150)


def test_single_process_is_local_time():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.job_ms(80.0, None, "cpu") == 80.0
    assert bench.job_value(1, 1, 2, 1000.0) == 2.0
