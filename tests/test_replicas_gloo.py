"""Multi-process host logic of the benchmark on CPU (gloo, world size 2).

The workload shards into independent replicas (one problem per rank, no
data-path collective); the job's step time is the slowest rank's.  This runs
the same reduction bench.py uses, on two CPU processes.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ws, r, local = bench.dist_env()
    step = 0.25 + 0.5 * rank  # rank 1 is the slow replica
    job = bench.job_step_seconds(step)
    q.put((r, ws, job))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_step_time_is_max_over_ranks():
    import socket

    import torch.multiprocessing as mp

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[2] == pytest.approx(0.75) for o in out)


def test_single_process_step_time_unchanged():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_step_seconds(0.3) == 0.3
