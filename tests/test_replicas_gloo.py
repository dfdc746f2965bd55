"""The N > 1 path of bench.py (independent replicas, one per rank) on CPU with the gloo
backend: the timed region is the maximum over ranks, the throughput counts all ranks'
points, and the two ranks agree on both numbers."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [120.0, 150.0][rank]            # rank 1 is the slower replica
        total, value = bench.whole_job_value(local_ms, 10, 4 << 20, world)
        q.put((rank, total, value))
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    for _, total, value in res:
        assert total == 150.0
        assert value == pytest.approx(world * 10 * (4 << 20) / 0.150)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    total, value = bench.whole_job_value(200.0, 5, 1000, 1)
    assert total == 200.0 and value == pytest.approx(5 * 1000 / 0.2)
