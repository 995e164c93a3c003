"""The replicas path of bench.py (one process per GPU, no data-path collective) on CPU: two gloo
ranks with different times and counts reduce to the slowest time and the total count."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, count = [(812.5, 300), (1044.0, 299)][rank]
        q.put((rank,) + bench.reduce_over_ranks(ms, count, "cpu"))
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_to_slowest_time_and_total_count():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, count in out:
        assert ms == 1044.0 and count == 599
