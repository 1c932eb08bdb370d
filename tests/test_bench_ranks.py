"""The multi-rank timing path of bench.py on CPU (gloo, world size 2).

With N replicas the bench reports the units all ranks processed over the
slowest rank's time; every rank must see the same maximum, and the
reference arm runs on rank 0 only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [2.0, 3.0][rank]
        m = bench.max_over_ranks(secs, world)
        rate = bench.job_rate(6.0, secs, world)
        r_env = bench.dist_env()

        class A:
            workload, steps, warmup = "rmat20", 1, 0
        ref = bench.run_reference(A(), rank, world) if rank == 1 else "skipped"
        q.put((rank, m, rate, r_env, ref))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    by = {o[0]: o for o in out}
    for r in (0, 1):
        _, m, rate, env, _ = by[r]
        assert m == 3.0            # the slowest rank's time on every rank
        assert rate == 6.0 * 2 / 3.0
        assert env == (r, 2, r)
    assert by[1][4] is None        # the reference arm: rank 1 does no work


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.job_rate(10.0, 2.0, 1) == 5.0
