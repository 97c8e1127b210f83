"""The N>1 host logic of bench.py on CPU with two gloo ranks: each rank renders
its own views (independent replicas, no data-path collective) and the timing
reduction takes the slowest rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    views = bench.rank_views(rank, views_per_rank=2)
    slowest = bench.max_over_ranks(10.0 + rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, views)
    q.put((rank, views, slowest, gathered))
    dist.destroy_process_group()


def test_two_ranks_render_disjoint_views_and_report_the_slowest():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, views, slowest, gathered in out:
        assert slowest == 11.0
        flat = [v for vs in gathered for v in vs]
        assert len(set(flat)) == len(flat) == 4
    assert sorted(v for _, views, _, _ in out for v in views) == [0.0, 45.0, 90.0, 135.0]
