"""Multi-rank host logic on CPU (gloo, world size 2): the 8-byte exchange of a
sharded count and the max-over-ranks job timing used by bench.py."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, partials, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2309_09064_gb300 import shard
        total = shard.sum_partials(partials[rank])
        slowest = shard.max_over_ranks(times[rank])
        out.put((rank, total, slowest))
    finally:
        dist.destroy_process_group()


def test_sharded_exchange_and_job_timing_world2():
    world = 2
    partials = [7_000_000_123, 3_285_451_828]  # uint64-sized partial counts
    times = [412.5, 433.25]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, partials, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, total, slowest in res:
        assert total == sum(partials)
        assert slowest == max(times)
