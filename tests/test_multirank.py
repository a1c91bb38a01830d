"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The path shards right-hand sides over ranks (replicas of the factor, no data-path
collective): each rank's incidence angles must be disjoint from the other's and lie in
[0, 180); the job time is the maximum over ranks, taken by an all-reduce.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        phis = bench.shard_angles(rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, [float(p) for p in phis])
        ms = bench.max_over_ranks(10.0 + rank, world, "cpu")
        if rank == 0:
            out.put((gathered, ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_angles_and_take_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, ms = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = (np.array(g) for g in gathered)
    assert len(a) == len(b) == 256
    assert np.all((a >= 0) & (a < 180)) and np.all((b >= 0) & (b < 180))
    assert len(np.intersect1d(np.round(a, 9), np.round(b, 9))) == 0
    assert ms == 11.0


def test_single_rank_angles_are_the_workload_angles():
    import bench
    import workloads as W
    np.testing.assert_array_equal(bench.shard_angles(0, 1), W.incidence_angles_deg(W.SEMICIRCLE_N262144))
