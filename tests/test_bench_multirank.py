"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
runs its own replica, the job's time is the slowest rank's, and the value
counts the units of all ranks.  Ranks other than 0 of the reference arm
exit without work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dt = bench.reduce_max_seconds(1.0 + 0.5 * rank)        # rank 1 is the slowest
        out[rank] = (dt, bench.whole_job_gstencil(3e9, world, dt))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        dt, value = out[r]
        assert dt == 1.5
        assert abs(value - 2 * 3e9 / 1.5 / 1e9) < 1e-9


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.main() == 0


def test_single_rank_time_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_seconds(2.5) == 2.5
