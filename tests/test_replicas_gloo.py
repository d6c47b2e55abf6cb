"""The N > 1 path of bench.py on the CPU: two gloo ranks.

bench.py runs one independent replica per rank (seed = rank, no exchange on
the data path); the only collectives are the barrier around the timed region
and the maximum of the per-rank step times.  Checked here: the ranks build
different problems of the same shape, the timing reduction returns the
slowest rank's time on every rank, and the whole-job figure divides it by the
number of replicas.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from inputs.grid_ls import workload

        prob, depth = workload("grid2d_64", seed=rank)
        dist.barrier()
        t = bench.reduce_max(0.5 + rank)  # rank 1 is the slowest
        out.put((rank, prob.m, prob.n, depth, float(prob.b[:16].sum()), t, bench.job_seconds(t, world)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_of_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    (r0, m0, n0, d0, b0, t0, v0), (r1, m1, n1, d1, b1, t1, v1) = res
    assert (m0, n0, d0) == (m1, n1, d1)  # same workload shape on every replica
    assert b0 != b1  # independent problems (seed = rank)
    assert t0 == t1 == pytest.approx(1.5)
    assert v0 == v1 == pytest.approx(0.75)
