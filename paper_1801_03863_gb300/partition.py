"""Sharding of an ensemble across ranks (one process per GPU).

Ensemble members are independent lattices, so a multi-GPU run needs no
exchange on the data path: each rank advances its own share.  Shares are
balanced by lattice-update cost with the longest-processing-time greedy rule
(largest member first, onto the least-loaded rank), which is deterministic,
so every rank computes the same assignment without communicating.
"""
from __future__ import annotations

from typing import Sequence


def partition(costs: Sequence[float], nranks: int) -> list[list[int]]:
    """Split member indices into nranks lists of near-equal total cost.

    Ties are broken by member index and rank index, so the result depends only
    on (costs, nranks).  Each list is returned in ascending member order.
    """
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * nranks
    share: list[list[int]] = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda k: (load[k], k))
        share[r].append(i)
        load[r] += float(costs[i])
    return [sorted(s) for s in share]


def imbalance(costs: Sequence[float], shares: list[list[int]]) -> float:
    """max rank load / mean rank load (1.0 = perfect balance)."""
    loads = [sum(float(costs[i]) for i in s) for s in shares]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0


def gather_totals(local_totals, member_ids: Sequence[int], count: int, dist=None):
    """All ranks' per-member conservation totals as one (count, 3) FP64 table.

    local_totals: this rank's (len(member_ids), 3) totals (sum rho, sum rho u_x,
    sum rho u_y), row j for global member member_ids[j].  Every rank fills its
    own rows of a zero table and the tables are summed across ranks (one
    all-reduce): each row has exactly one nonzero contribution, and x + 0 is
    exact, so the result is bitwise what a single rank would report.
    dist: torch.distributed (initialised) or None for one rank.
    """
    import numpy as np
    import torch

    table = np.zeros((count, 3), dtype=np.float64)
    loc = np.asarray(local_totals, dtype=np.float64).reshape(len(member_ids), 3)
    table[list(member_ids)] = loc
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return table
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.from_numpy(table).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()
