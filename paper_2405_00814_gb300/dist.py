"""Multi-process host logic (one process per GPU).

* Independent scenes (a batch of designs or uneven scenes) shard across ranks
  with no data-path collective: ``shard_scenes`` balances cells greedily.
* Whole-job throughput is the units all ranks processed over the slowest rank's
  time (``job_throughput``).
* A single grid larger than one GPU splits into y-slabs; every step needs one
  row of Ez from the +y neighbour before layer 1 and one row of Hx from the -y
  neighbour before layer 2 (the H update reads Ez(j+1), the E update reads
  Hx(j-1); Sec. III-B eqs. (7)-(9)).  ``SlabExchange`` does that exchange with
  point-to-point messages into the receiver's own buffers.  Each box in this
  build has one GPU, so the slab path is exercised on CPU ranks.
"""
from __future__ import annotations

import numpy as np


def shard_scenes(cells, world: int):
    """Greedy longest-processing-time assignment of scenes (given their cell
    counts) to `world` ranks; returns a list of index lists, one per rank."""
    order = sorted(range(len(cells)), key=lambda k: (-int(cells[k]), k))
    load = [0] * world
    out = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += int(cells[k])
    return [sorted(x) for x in out]


def job_throughput(units_local: float, seconds_local: float, group=None):
    """(sum of units over ranks) / (max of seconds over ranks)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return units_local / seconds_local
    u = torch.tensor([float(units_local)], dtype=torch.float64)
    s = torch.tensor([float(seconds_local)], dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(s, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()) / float(s.item())


def slab_rows(ny: int, rank: int, world: int):
    """Owned rows [j0, j1) of a rank in a y-slab decomposition."""
    base, extra = divmod(ny, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


class SlabExchange:
    """Halo exchange of a y-slab decomposition for host (numpy) arrays.

    A rank's local arrays cover global rows [j0 - g0, j1 + g1) where g0 = 1 unless
    the rank holds row 0 and g1 = 1 unless it holds the last row: one ghost row
    on each interior side.  ``ez_up`` fills the top ghost row of Ez from the +y
    neighbour's first owned row; ``h_down`` fills the bottom ghost row of Hx
    (and Hy) from the -y neighbour's last owned row."""

    def __init__(self, ny, rank, world, group=None):
        self.rank, self.world, self.group = rank, world, group
        self.j0, self.j1 = slab_rows(ny, rank, world)
        self.g0 = 0 if rank == 0 else 1
        self.g1 = 0 if rank == world - 1 else 1

    @property
    def local_rows(self):
        return self.j1 - self.j0 + self.g0 + self.g1

    def owned(self, a):
        return a[self.g0:self.g0 + (self.j1 - self.j0)]

    def _swap(self, send_row, recv_row, to, frm, tag):
        import torch
        import torch.distributed as dist
        reqs = []
        if to is not None:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(send_row)), to, group=self.group, tag=tag))
        if frm is not None:
            buf = torch.empty(recv_row.shape, dtype=torch.float64)
            dist.recv(buf, frm, group=self.group, tag=tag)
            recv_row[...] = buf.numpy()
        for r in reqs:
            r.wait()

    def ez_up(self, ez):
        """Ez ghost above <- first owned row of rank+1."""
        up = self.rank + 1 if self.rank + 1 < self.world else None
        dn = self.rank - 1 if self.rank > 0 else None
        send = ez[self.g0] if dn is not None else None
        recv = ez[-1] if up is not None else np.empty(ez.shape[1])
        self._swap(send, recv, dn, up, tag=1)

    def h_down(self, *hs):
        """H ghost below <- last owned row of rank-1 (for each array given)."""
        up = self.rank + 1 if self.rank + 1 < self.world else None
        dn = self.rank - 1 if self.rank > 0 else None
        for k, h in enumerate(hs):
            send = h[self.g0 + (self.j1 - self.j0) - 1] if up is not None else None
            recv = h[0] if dn is not None else np.empty(h.shape[1])
            self._swap(send, recv, up, dn, tag=2 + k)
