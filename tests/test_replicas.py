"""The replica path of the benchmark on two CPU ranks (gloo): the job's time is
the slowest rank's and its throughput counts every rank's cells; each rank
draws its own grid."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2406_17284_gb300 import inputs
        ms_local = [120.0, 200.0][rank]                       # rank 1 is the slow one
        ms_step, rate = bench.job_rate(ms_local, 1_000_000, 4, world, dist)
        grid = inputs.bernoulli(64, 64, bench.P_ALIVE, bench.SEED + rank)
        q.put((rank, ms_step, rate, bench.dist_env(), int(grid.sum()), grid.tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_all_cells():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_step, rate, env, _, _ in out:
        assert env == (rank, world, 0) or env[:2] == (rank, world)
        assert ms_step == pytest.approx(200.0 / 4)             # the slowest rank's time
        assert rate == pytest.approx(2 * 1_000_000 / 0.05)     # both ranks' cells
    assert out[0][5] != out[1][5], "replicas must draw different grids"


def test_single_rank_needs_no_process_group():
    import bench
    ms_step, rate = bench.job_rate(80.0, 500, 4, 1)
    assert ms_step == 20.0 and rate == pytest.approx(500 / 0.02)
