"""Replicas-only multi-GPU path of bench.py on CPU: two gloo ranks, the whole-job rate from the
slowest rank's time, and the reference arm running on rank 0 only."""
import os
import socket
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 1 + r seconds for 5e9 units: the job rate is 2 * 5e9 / 2 s on every rank
    rate = bench.whole_job_rate(5e9, 1.0 + rank, world, dist, "cpu")
    slowest = bench.max_over_ranks(0.25 * (rank + 1), dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rate, slowest))


def test_whole_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, slowest in res:
        assert rate == pytest.approx(5e9)
        assert slowest == pytest.approx(0.5)


def test_single_rank_rate_needs_no_process_group():
    import bench

    assert bench.whole_job_rate(1e9, 0.5, 1) == pytest.approx(2e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup = 1, 1

    assert bench.run_reference(Args()) == 0
