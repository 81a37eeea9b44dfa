"""bench.py's multi-rank logic on CPU: with two gloo ranks the whole-job value counts every
rank's solves over the slowest rank's time; the reference arm's other ranks exit without work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms, value = bench.aggregate(100.0 * (rank + 1), 120, ws)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_slowest_rank_and_all_solves():
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
    for rank, ms, value in out:
        assert ms == 200.0  # the slower rank's 200 ms
        assert value == pytest.approx(2 * 120 / 0.2)  # both ranks' 240 solves in 0.2 s


def test_single_rank_aggregation_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(500.0, 120, 1) == (500.0, pytest.approx(240.0))


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(Args) == 0  # returns at once, no oracle work
