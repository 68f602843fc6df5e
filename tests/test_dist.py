"""Multi-rank host logic on the CPU: ensemble sharding (no data-path
collective) and the bench's barrier / max-over-ranks timing, with gloo ranks."""
import os
import socket

import numpy as np
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


# ----------------------------------------------------------------------------
# Each rank advances its share of an ensemble (through the oracle on the CPU):
# the gathered per-member results equal the one-rank run, so the share ->
# member mapping (order, nu, u_lid, initial fields) is right.
# ----------------------------------------------------------------------------
def _spawn(world, target, extra=()):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + tuple(extra))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return sorted(res, key=lambda r: r[0])


def _share_results(name, rank, world, per_gpu, steps):
    """Run the oracle on every member of this rank's share of the workload;
    -> {global member id: (totals, populations)}."""
    import numpy as np

    import bench
    import oracle
    wk = bench.Workload(name, rank, world, members_per_gpu=per_gpu)
    out, k = {}, 0
    for j, mid in enumerate(wk.member_ids):
        nx, ny = wk.dims[j]
        n = nx * ny
        if wk.lattice == "d2q9":
            sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(wk.nu[j]), oracle.BC_CAVITY,
                             u_lid=wk.u_lid[j])
            sim.init(wk.rho[k:k + n], wk.ux[k:k + n], wk.uy[k:k + n])
        else:
            sim = oracle.Sim(oracle.D1Q3, nx, 1, oracle.tau_from_nu(wk.nu[j]),
                             oracle.BC_ZERO_GRADIENT)
            sim.init(wk.rho[k:k + n], wk.ux[k:k + n])
        k += n
        sim.step(steps)
        out[mid] = (sim.conservation(), np.asarray(sim.get_f()))
    return out


def _share_main(rank, world, port, q, name, per_gpu, steps):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "OMP_NUM_THREADS": "2"})
    import bench
    from paper_1801_03863_gb300.partition import gather_totals
    d = bench.Dist()
    res = _share_results(name, rank, world, per_gpu, steps)
    ids = sorted(res)
    # the one collective of the sharded path: every rank gets all totals
    table = gather_totals([res[m][0] for m in ids], ids, per_gpu * world, d.pg)
    d.barrier()
    q.put((rank, {"members": res, "table": table}))
    d.close()


@pytest.mark.parametrize("name,per_gpu,steps", [("ensemble64", 3, 2), ("tubes4096", 24, 40)])
def test_ranks_advance_their_share_like_one_rank(name, per_gpu, steps):
    world = 2
    res = _spawn(world, _share_main, (name, per_gpu, steps))
    got = {}
    for _, part in res:
        assert not set(part["members"]) & set(got)  # no member on two ranks
        got.update(part["members"])
    want = _share_results(name, 0, 1, per_gpu * world, steps)
    assert sorted(got) == sorted(want) == list(range(per_gpu * world))
    for mid in want:
        assert np.array_equal(got[mid][0], want[mid][0]), mid
        assert np.array_equal(got[mid][1], want[mid][1]), mid
    # the gathered totals table is the same on every rank and equals the
    # one-rank totals bit for bit
    want_table = np.array([want[m][0] for m in range(per_gpu * world)])
    for _, part in res:
        assert np.array_equal(part["table"], want_table)


# ----------------------------------------------------------------------------
# Row-slab decomposition of one lattice: gloo ranks run the oracle on their
# slabs, exchanging one row of three planes per face per step; the gathered
# lattice equals the one-rank run bit for bit.
# ----------------------------------------------------------------------------
SLAB_CASES = {
    # name: (nx, ny, bc, nu, u_lid, collision, steps)
    "taylor_green": (20, 26, "periodic", 0.01, 0.0, "minxent4", 30),
    "cavity": (18, 23, "cavity", 0.02, 0.08, "minxent4", 30),
    "cavity_mrt": (14, 17, "cavity", 0.05, 0.1, "mrt", 20),
}


def _slab_fields(case):
    from paper_1801_03863_gb300 import workloads as wl
    nx, ny, bc = SLAB_CASES[case][:3]
    if bc == "periodic":
        return wl.taylor_green(nx, u0=0.05, ny=ny)
    return _cavity_fields(nx, ny)


def _cavity_fields(nx, ny):
    rng = np.random.default_rng(5)
    rho = 1.0 + 1e-3 * rng.uniform(-1, 1, (ny, nx))
    ux = 0.01 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.01 * rng.uniform(-1, 1, (ny, nx))
    return rho, ux, uy


def _slab_run(case, rank, world, dist):
    import oracle
    from paper_1801_03863_gb300.slab import SlabExchange, slab_step
    nx, ny, bc, nu, u_lid, coll, steps = SLAB_CASES[case]
    ex = SlabExchange(nx, ny, world, rank, periodic=(bc == "periodic"), dist=dist)
    y0, y1 = ex.rows
    rho, ux, uy = _slab_fields(case)
    sim = oracle.Sim(oracle.D2Q9, nx, y1 - y0, oracle.tau_from_nu(nu),
                     {"periodic": oracle.BC_PERIODIC, "cavity": oracle.BC_CAVITY}[bc],
                     collision={"minxent4": oracle.MINXENT4, "mrt": oracle.MRT}[coll],
                     u_lid=u_lid)
    sim.set_slab(y0, ny)
    sim.init(rho[y0:y1], ux[y0:y1], uy[y0:y1])
    slab_step(sim, ex, steps)
    return (y0, y1), sim.get_f(), sim.counters()


def _slab_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "OMP_NUM_THREADS": "1"})
    import torch.distributed as dist

    import bench
    d = bench.Dist()
    out = {case: _slab_run(case, rank, world, dist) for case in SLAB_CASES}
    d.barrier()
    q.put((rank, out))
    d.close()


def test_slab_rows_cover_the_lattice():
    from paper_1801_03863_gb300.slab import slab_rows
    for ny in (3, 17, 64, 101):
        for world in range(1, min(ny, 8) + 1):
            rows = slab_rows(ny, world)
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            h = [b - a for a, b in rows]
            assert min(h) >= 1 and max(h) - min(h) <= 1
    with pytest.raises(ValueError):
        slab_rows(2, 3)


def test_one_rank_slab_equals_whole_lattice():
    """world = 1: the exchange closes the periodic ring on itself and the
    cavity's faces are closed, so slab_step is the plain step."""
    import oracle
    for case, (nx, ny, bc, nu, u_lid, coll, steps) in SLAB_CASES.items():
        (y0, y1), f, c = _slab_run(case, 0, 1, None)
        assert (y0, y1) == (0, ny)
        sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(nu),
                         {"periodic": oracle.BC_PERIODIC, "cavity": oracle.BC_CAVITY}[bc],
                         collision={"minxent4": oracle.MINXENT4, "mrt": oracle.MRT}[coll],
                         u_lid=u_lid)
        sim.init(*_slab_fields(case))
        sim.step(steps)
        assert np.array_equal(f, sim.get_f()), case


@pytest.mark.parametrize("world", [2, 4])
def test_slab_ranks_equal_one_lattice_bitwise(world):
    import oracle
    res = _spawn(world, _slab_main)
    for case, (nx, ny, bc, nu, u_lid, coll, steps) in SLAB_CASES.items():
        sim = oracle.Sim(oracle.D2Q9, nx, ny, oracle.tau_from_nu(nu),
                         {"periodic": oracle.BC_PERIODIC, "cavity": oracle.BC_CAVITY}[bc],
                         collision={"minxent4": oracle.MINXENT4, "mrt": oracle.MRT}[coll],
                         u_lid=u_lid)
        sim.init(*_slab_fields(case))
        sim.step(steps)
        want = sim.get_f()
        got = np.concatenate([out[case][1] for _, out in res], axis=1)
        assert [out[case][0] for _, out in res][0][0] == 0
        assert np.array_equal(got, want), case
        # status counters add up across the slabs
        tot = sum(out[case][2]["newton_skipped"] for _, out in res)
        assert tot == sim.counters()["newton_skipped"]
