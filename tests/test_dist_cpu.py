"""Multi-rank host logic on CPU (gloo, world size 2): problem sharding, max/sum timing
reduction and the eigenvalue gather used when k-points are split across GPUs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1806_10284_gb300.sharding import shard, shard_indices, reduce_timing, gather_results


def test_shard_partition():
    items = list(range(23))
    for world in (1, 2, 3, 8):
        parts = [shard(items, r, world) for r in range(world)]
        flat = sorted(x for p in parts for x in p)
        assert flat == items
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        shard(items, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard_indices(60, rank, world)
        # each rank "solves" its problems: eigenvalues encoded from the index
        local = {i: [float(i), float(i) + 0.5] for i in mine}
        merged = gather_results(local)
        t, w = reduce_timing(10.0 + rank, float(len(mine) * 100))
        out_q.put((rank, sorted(merged), t, w))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, keys, t, w in res:
        assert keys == list(range(60))          # every problem gathered exactly once
        assert t == 11.0                         # max over ranks
        assert w == 6000.0                       # sum over ranks
