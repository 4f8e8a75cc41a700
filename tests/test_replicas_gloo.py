"""Multi-rank host logic on CPU: world-size-2 gloo process groups (127.0.0.1).

The data path has no collective: each rank propagates its own share of independent fields (here
with the FP64 oracle, standing in for its GPU), and the union of the shares equals the
single-process result; only the timing reduction (max over ranks) and the tally are collective."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1107_5578_gb300 import replicas, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_items, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        share = replicas.item_range(n_items, world, rank)
        outs = {}
        for i in share:
            u = synth.random_field(32, seed=replicas.rank_seed(7, 0) + i)
            outs[i] = oracle.propagate(u, 8e-6, 8e-6, 532e-9, 0.01 + 0.002 * i, oracle.ANGULAR)
        t_max = replicas.max_over_ranks(1.0 + rank)          # rank 1 is the slowest
        total = replicas.sum_over_ranks(len(share))
        gathered = [None] * world
        dist.all_gather_object(gathered, outs)
        routes = replicas.route([256, 4096, 512, 2048, 256, 1024, 4096, 256], world)
        all_routes = [None] * world
        dist.all_gather_object(all_routes, routes)
        q.put((rank, t_max, total, gathered if rank == 0 else None, all_routes))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_reduce_and_route():
    import oracle
    oracle.build()
    world, n_items = 2, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_items, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    for rank, t_max, total, _, routes in res:
        assert t_max == 2.0                                  # max over ranks, seen by every rank
        assert total == n_items                              # every item handled exactly once
    assert res[0][4][0] == res[0][4][1]                      # all ranks compute the same routing
    gathered = res[0][3]
    merged = {}
    for d in gathered:
        assert not (set(d) & set(merged))                    # shares are disjoint
        merged.update(d)
    assert sorted(merged) == list(range(n_items))
    for i in range(n_items):                                 # sharded == single-process
        u = synth.random_field(32, seed=replicas.rank_seed(7, 0) + i)
        want = oracle.propagate(u, 8e-6, 8e-6, 532e-9, 0.01 + 0.002 * i, oracle.ANGULAR)
        assert np.array_equal(merged[i], want)


def test_item_range_partitions():
    for n in range(0, 40):
        for w in range(1, 9):
            rs = [replicas.item_range(n, w, r) for r in range(w)]
            assert sum(len(r) for r in rs) == n
            assert [i for r in rs for i in r] == list(range(n))
            assert max(len(r) for r in rs) - min(len(r) for r in rs) <= 1
    with pytest.raises(ValueError):
        replicas.item_range(4, 2, 2)


def test_router_balances_cost():
    sizes = synth.serving_requests(2000, seed=3)["n"]
    routes = replicas.route(sizes, 4)
    assert sorted(i for r in routes for i in r) == list(range(2000))
    loads = [sum(replicas.request_cost(sizes[i]) for i in r) for r in routes]
    assert max(loads) - min(loads) <= replicas.request_cost(4096)
    assert all(r == sorted(r) for r in routes)
    assert replicas.job_rate(16, 4, 0.5) == 128.0
