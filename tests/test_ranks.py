"""The multi-rank path of bench.py on CPU: world_size-2 gloo ranks, each an
independent replica ("replicas only": the path has no exchange step).  The job's
time is the slowest rank's, element by element, and the whole-job rate counts
the units of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed its replica at (10 + r) ms and its end-to-end leg at (30 - r) ms
        got = bench.max_over_ranks([10.0 + rank, 30.0 - rank], world, torch.device("cpu"))
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r] == [11.0, 30.0]


def test_single_rank_and_job_rate():
    assert bench.max_over_ranks([3.5, 7.0], 1, None) == [3.5, 7.0]
    # 2 replicas of 200 sweeps, slowest rank 250 ms: 1600 sweeps/s for the job
    assert bench.job_rate(200, 2, 250.0) == pytest.approx(1600.0)
