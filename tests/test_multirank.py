"""Host logic of the multi-rank bench path on CPU (gloo, world size 2).

The FSI path shards by games with no exchange step: each rank explains its
own 16 instances and the job's time is its slowest rank.  These tests run
two gloo ranks on the CPU: the max-over-ranks reduction, the whole-job rate,
and that the ranks' instance shards are disjoint slices of one seeded
stream."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [2.0, 5.0][rank]
        m = bench.max_over_ranks(ms, "cpu")
        rate = bench.whole_job_rate(1000.0, world, m)
        x = bench.shard_workload(rank).x
        dist.barrier()
        q.put((rank, m, rate, x))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        r, m, rate, x = q.get(timeout=120)
        got[r] = (m, rate, x)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert got[r][0] == 5.0                      # the slowest rank's time
        assert got[r][1] == pytest.approx(2 * 1000.0 / 5e-3)
    x0, x1 = got[0][2], got[1][2]
    assert x0.shape == x1.shape == (16, 20)
    assert not np.allclose(x0, x1)                   # disjoint instances
    from paper_2601_01903_gb300 import synthetic
    both = synthetic.gaussian_instances(32, 20, 2)
    assert np.array_equal(np.vstack([x0, x1]), both)  # slices of one stream


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
