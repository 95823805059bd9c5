"""Multi-rank host logic on CPU: two gloo ranks shard the items and reduce
timings the way bench.py does under torchrun (no GPU)."""
import os
import socket

import torch.multiprocessing as mp

from paper_2407_11388_b300.dist import shard_range


def test_shards_partition_items():
    for n in (0, 1, 5, 16, 257, 16384):
        for world in (1, 2, 3, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2407_11388_b300.dist import max_over_ranks, shard_range, sum_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start, stop = shard_range(1000, rank, world)
        t = 1.0 + rank  # this rank's "time"
        out[rank] = (start, stop, max_over_ranks(t), sum_over_ranks(stop - start))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    res = [out[r] for r in range(world)]
    assert res[0][:2] == (0, 500) and res[1][:2] == (500, 1000)
    assert all(r[2] == 2.0 for r in res)       # slowest rank's time everywhere
    assert all(r[3] == 1000.0 for r in res)    # every item counted once
