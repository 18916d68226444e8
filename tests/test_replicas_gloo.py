"""Replica timing aggregation of bench.py on two CPU ranks (gloo, world size 2).

The multi-GPU bench runs independent replicas (no collective on the data
path); the only cross-rank step is the max of the elapsed times, and the job
value is elapsed_max / (world * steps).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local = 100.0 + 50.0 * rank            # rank 1 is the slow replica
    mx = bench.max_over_ranks(local)
    bench.barrier()
    q.put((rank, mx, bench.job_ms_per_unit(mx, 10, world), bench.dist_env()))
    dist.destroy_process_group()


def test_two_rank_max_and_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val, env in res:
        assert mx == 150.0
        assert val == pytest.approx(150.0 / 20)
        assert env == (rank, 2, rank)


def test_single_process_defaults():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_ms_per_unit(30.0, 10, 1) == 3.0
