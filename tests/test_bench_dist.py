"""The multi-replica bookkeeping of bench.py on CPU with the gloo backend,
world size 2: every rank times its own replica; the job's time is the slowest
rank's and the rate counts the cells of all replicas."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is slower
    mx = bench.reduce_max_ms(ms)
    rate = bench.aggregate_rate(1000, 4, world, mx)
    q.put((rank, mx, rate))
    dist.destroy_process_group()


def test_replica_timing_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rate in out:
        assert mx == 15.0
        assert rate == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_single_process_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_ms(7.5) == 7.5
    assert bench.aggregate_rate(10, 2, 1, 1.0) == pytest.approx(20 / 1e-3)
