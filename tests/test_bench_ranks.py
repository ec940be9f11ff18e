"""The benchmark's whole-job figures over N replicas (one process per GPU, exchanging nothing but
these two reductions): the slowest rank's time and the work summed over the ranks.  Run here as a
world of two `gloo` ranks on the CPU (the GPU runs use NCCL; the reduction logic is the same)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units, e2e = bench.whole_job(10.0 + rank, 1000 * (rank + 1), 5.0 * (rank + 1), "cpu", world)
        out.put((rank, ms, units, e2e))
    finally:
        dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, e2e in res:
        assert ms == 11.0                # the slowest rank
        assert units == 3000.0           # work of both replicas
        assert e2e == 15.0


def test_whole_job_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(7.5, 123, 4.0, "cpu", 1) == (7.5, 123, 4.0)
