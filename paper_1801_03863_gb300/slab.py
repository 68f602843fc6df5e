"""Row-slab decomposition of one D2Q9 lattice across ranks (one process per GPU).

A lattice of nx x ny nodes too large for one device is split into contiguous
row slabs, one per rank (``slab_rows``).  A time step of Eq. (2) collides
every node locally, then streams each population one node along its
velocity v_a.  The only values that cross a slab edge are the ones streamed
across it: through the top face the three populations with v_y = +1 of the
slab's last row, through the bottom face the three with v_y = -1 of its
first row.  In the column order of the moment matrix T (Eq. Tmatrix) these
are planes 2, 5, 6 (up) and 4, 7, 8 (down).  So a step needs one exchange
between collision and streaming: per face, one row of three planes (3 nx
values) to the neighbouring rank and one from it -- a pair of point-to-point
transfers per face, no collective.  A periodic lattice closes the ring (rank
0's lower neighbour is the last rank); a cavity's first and last slabs keep
their wall and lid rows and exchange nothing across those faces.

``SlabExchange`` does the exchange over torch.distributed (gloo on the CPU,
NCCL between GPUs); ``slab_step`` runs one step of a slab through any
backend with the two halves of the step (``collide``, ``post_row``,
``stream``).  The result equals the single-lattice run bit for bit: the
collision is node-local and the streaming reads the same post-collision
values, whichever rank computed them.
"""
from __future__ import annotations

import numpy as np

Q = 9
UP = (2, 5, 6)     # v_y = +1: leave a slab through its top face
DOWN = (4, 7, 8)   # v_y = -1: leave through its bottom face
TAG_UP, TAG_DOWN = 1, 2  # message tags, so two transfers to one neighbour never mix


def slab_rows(ny: int, world: int) -> list[tuple[int, int]]:
    """Contiguous row ranges [y0, y1) of near-equal height, one per rank."""
    if world < 1 or ny < world:
        raise ValueError("need at least one row per rank")
    base, extra = divmod(ny, world)
    out, y = [], 0
    for r in range(world):
        h = base + (1 if r < extra else 0)
        out.append((y, y + h))
        y += h
    return out


class SlabExchange:
    """Edge-row exchange of one rank's slab.

    exchange(first, last) takes the slab's first and last post-collision rows
    ([9, nx] float64) and returns (lo, hi): the post-collision row below the
    slab with the three up-going planes from the lower neighbour, and the row
    above it with the three down-going planes from the upper neighbour (the
    other planes are NaN: streaming never reads them).  At a closed face (a
    non-periodic lattice's first or last slab) the entry is None and the
    backend applies its own boundary rule there.
    """

    def __init__(self, nx: int, ny: int, world: int, rank: int, periodic: bool, dist=None):
        self.nx, self.ny, self.world, self.rank = nx, ny, world, rank
        self.periodic = periodic
        self.rows = slab_rows(ny, world)[rank]
        self.dist = dist
        below, above = rank - 1, rank + 1
        if periodic:
            below %= world
            above %= world
        self.below = below if 0 <= below < world else None
        self.above = above if 0 <= above < world else None

    def _halo(self, row: np.ndarray, planes) -> np.ndarray:
        out = np.full((Q, self.nx), np.nan)
        out[list(planes)] = row[list(planes)]
        return out

    def exchange(self, first: np.ndarray, last: np.ndarray):
        up = np.ascontiguousarray(last[list(UP)])      # to the rank above
        down = np.ascontiguousarray(first[list(DOWN)])  # to the rank below
        if self.world == 1:
            lo = self._halo(last, UP) if self.below is not None else None
            hi = self._halo(first, DOWN) if self.above is not None else None
            return lo, hi
        import torch
        ops, recv = [], {}
        if self.below is not None:
            recv["lo"] = torch.empty((3, self.nx), dtype=torch.float64)
            ops.append(self.dist.P2POp(self.dist.irecv, recv["lo"], self.below, tag=TAG_UP))
        if self.above is not None:
            recv["hi"] = torch.empty((3, self.nx), dtype=torch.float64)
            ops.append(self.dist.P2POp(self.dist.irecv, recv["hi"], self.above, tag=TAG_DOWN))
        if self.above is not None:
            ops.append(self.dist.P2POp(self.dist.isend, torch.from_numpy(up), self.above,
                                       tag=TAG_UP))
        if self.below is not None:
            ops.append(self.dist.P2POp(self.dist.isend, torch.from_numpy(down), self.below,
                                       tag=TAG_DOWN))
        for w in self.dist.batch_isend_irecv(ops):
            w.wait()
        lo = hi = None
        if "lo" in recv:
            lo = np.full((Q, self.nx), np.nan)
            lo[list(UP)] = recv["lo"].numpy()
        if "hi" in recv:
            hi = np.full((Q, self.nx), np.nan)
            hi[list(DOWN)] = recv["hi"].numpy()
        return lo, hi


def slab_step(backend, ex: SlabExchange, steps: int = 1) -> None:
    """Advance one rank's slab by `steps` time steps of Eq. (2): collide,
    exchange the edge rows, stream.  backend: collide(), post_row(y) ->
    [9, nx], stream(lo, hi) on the slab's local rows."""
    h = ex.rows[1] - ex.rows[0]
    for _ in range(steps):
        backend.collide()
        lo, hi = ex.exchange(backend.post_row(0), backend.post_row(h - 1))
        backend.stream(lo, hi)
