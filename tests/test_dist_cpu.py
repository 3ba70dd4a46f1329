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


def _bench_worker(rank, world, port, out_q):
    """One rank of the benchmark's multi-GPU host path on CPU: its share of the bench's
    problem list (bench.my_problems, the sharding module's round robin), each problem
    solved here by the oracle on a small FCC grid in place of the GPU, then the
    benchmark's own gather and max/sum reductions."""
    import numpy as np
    import bench
    from oracle.eigs import eigs_dense
    from oracle.lattice import make_lattice
    from paper_1806_10284_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.WORKLOADS[bench.WORKLOAD]
        local = {}
        for idx, red in bench.my_problems(rank, world):
            lat = make_lattice(w["vectors"], (4, 4, 4), W.bloch_from_reduced(w["vectors"], red))
            invB = np.ones((3,) + lat.shape) / 3.0
            lam, _ = eigs_dense(lat, invB, 4)
            local[idx] = [float(x) for x in lam]
        merged = gather_results(local)
        t, work = reduce_timing(5.0 * (rank + 1), float(len(local)))
        out_q.put((rank, merged, t, work))
    finally:
        dist.destroy_process_group()


def test_bench_multi_rank_path_two_ranks():
    import numpy as np
    import bench
    from oracle.eigs import eigs_dense
    from oracle.lattice import make_lattice
    from paper_1806_10284_gb300 import workloads as W
    world = 2
    # one problem per rank, the first being the workload's own Bloch vector
    assert [len(bench.my_problems(r, world)) for r in range(world)] == [1, 1]
    assert np.allclose(bench.my_problems(0, world)[0][1], W.WORKLOADS[bench.WORKLOAD]["reduced_k"][0])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = W.WORKLOADS[bench.WORKLOAD]
    serial = {}
    for idx, red in enumerate(bench.problem_list(world)):
        lat = make_lattice(w["vectors"], (4, 4, 4), W.bloch_from_reduced(w["vectors"], red))
        serial[idx] = [float(x) for x in eigs_dense(lat, np.ones((3,) + lat.shape) / 3.0, 4)[0]]
    for rank, merged, t, work in res:
        assert merged == serial                 # every problem once, identical to one process
        assert t == 10.0 and work == 2.0        # max of the times, sum of the work
