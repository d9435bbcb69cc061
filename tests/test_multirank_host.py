"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2).

Every rank solves its own problems (no collective on the data path). The whole-job rate
takes the slowest rank's time, by a MAX all-reduce, and counts the units of all ranks. The
reference arm runs on rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_worker(rank, world, port, q):
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [100.0, 150.0][rank]          # rank 1 is the slow one
        rate, ms = bench.whole_job_rate(local_ms, 5, world, device="cpu")
        q.put((rank, rate, ms))
        torch.distributed.barrier()
    finally:
        torch.distributed.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank_and_all_units():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = [q.get(timeout=120) for _ in procs]
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert sorted(r for r, _, _ in res) == [0, 1]
    for _, rate, ms in res:
        assert ms == 150.0                        # every rank sees the slowest time
        assert rate == pytest.approx(world * 5 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    rate, ms = bench.whole_job_rate(200.0, 4, 1)
    assert ms == 200.0 and rate == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only():
    import bench

    class Args:
        steps = 1
        warmup = 0

    assert bench.run_reference(Args(), 1, 2) is None
