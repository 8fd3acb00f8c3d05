"""The multi-GPU path is replicas only (each rank renders its own step, no exchange): the
benchmark's job time is the slowest rank's and its rate counts every rank's rays.  Checked with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist, r, n, local = bench._dist("gloo")
    assert (r, n, local) == (rank, world, rank)
    seconds = 1.5 + rank                       # rank 1 is the slow one
    worst = bench._max_over_ranks(dist, seconds, device="cpu")
    rate = bench._job_rate(1000, n, 10, worst)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, worst, rate))


def test_two_replicas_time_is_the_slowest_and_rate_counts_both():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, worst, rate in got:
        assert worst == pytest.approx(2.5)
        assert rate == pytest.approx(1000 * 2 * 10 / 2.5 / 1e6)


def test_single_process_needs_no_group():
    import bench
    assert bench._max_over_ranks(None, 3.0) == 3.0
    assert bench._job_rate(2_000_000, 1, 5, 2.0) == pytest.approx(5.0)
