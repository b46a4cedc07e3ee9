"""The N-replica path of bench.py on CPU ranks (gloo, world size 2): the timed region is
the maximum over ranks, and the whole-job value counts the units of every rank."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        value, ms = bench.job_rate(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world)
        q.put((rank, value, ms))
    finally:
        dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's 15 ms; each counts world x its own units
    for rank, value, ms in out:
        assert ms == 15.0
        assert value == pytest.approx(2 * 1000.0 * (rank + 1) / 15e-3)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(20.0, 500.0, 1) == (500.0 / 20e-3, 20.0)
