"""Multi-rank host logic of bench.py on CPU with the gloo backend
(world size 2): the timed window is the slowest rank's, and the whole-job
throughput counts every rank's replica."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    mx = bench.max_over_ranks(ms)
    val = bench.whole_job_throughput(units_per_rank_step=1000, steps=4, world=world, max_ms=mx)
    out.put((rank, mx, val))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val in res:
        assert mx == 150.0
        assert abs(val - 1000 * 4 * 2 / 0.150) < 1e-6


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_throughput(10, 3, 1, 1000.0) == 30.0
