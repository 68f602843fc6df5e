"""Multi-rank host logic on the CPU: ensemble sharding (no data-path
collective) and the bench's barrier / max-over-ranks timing, with gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1801_03863_gb300 import workloads as wl
from paper_1801_03863_gb300.partition import imbalance, partition


def test_partition_covers_and_balances():
    members = wl.cavity_ensemble(count=64 * 8, seed=0)
    costs = [m.side * m.side for m in members]
    for n in (1, 2, 4, 8):
        shares = partition(costs, n)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(members)))
        assert imbalance(costs, shares) < 1.02
    assert partition(costs, 4) == partition(costs, 4)


def test_partition_edge_cases():
    assert partition([], 3) == [[], [], []]
    assert partition([5.0], 2) == [[0], []]
    with pytest.raises(ValueError):
        partition([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench
    import torch
    import torch.distributed as dist
    d = bench.Dist()
    # each rank builds its own share of the ensemble, as bench.py does
    wk = bench.Workload("tubes4096", rank, world)
    mine = torch.tensor([wk.nodes, len(wk.dims)], dtype=torch.int64)
    got = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, mine)
    d.barrier()
    t = d.reduce(10.0 + rank, "max")
    total = d.reduce(float(wk.nodes), "sum")
    q.put((rank, [g.tolist() for g in got], t, total))
    d.close()


def test_two_gloo_ranks_shard_without_overlap():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    members = wl.tube_ensemble(count=4096 * world, seed=1)
    full = sum(m.n for m in members)
    for rank, got, t, total in res:
        assert t == 11.0                       # max over ranks
        assert int(total) == full              # shares cover the ensemble once
        assert sum(g[1] for g in got) == 4096 * world
        assert max(g[0] for g in got) / (full / world) < 1.01
