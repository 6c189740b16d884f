"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The beamforming path shards by frames with no data-path collective
(replicas); the only cross-rank operations are the barrier and the
max-over-ranks time.  These run as two gloo processes here.
"""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        frames = bench.rank_frames(rank, 4)
        dist.barrier()
        t_local = 1.0 + rank  # rank 1 is the slow one
        t_job = bench.max_over_ranks(t_local, dist)
        value = bench.job_value(1e9, world, 10, t_job)
        gathered = [None] * world
        dist.all_gather_object(gathered, frames)
        q.put((rank, t_job, value, gathered))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_frames_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_job, value, gathered in res:
        assert t_job == pytest.approx(2.0)  # max over ranks
        assert value == pytest.approx(1e9 * 2 * 10 / 2.0 / 1e9)
        assert gathered[0] == [0, 1, 2, 3] and gathered[1] == [4, 5, 6, 7]  # disjoint frames


def test_single_rank_helpers():
    import bench

    assert bench.rank_frames(0, 3) == [0, 1, 2]
    assert bench.max_over_ranks(1.25, None) == 1.25
    assert bench.job_value(33554432 * 32, 1, 400, 0.4) == pytest.approx(33554432 * 32 * 400 / 0.4 / 1e9)
