"""Multi-process host logic (one process per GPU).

* Independent scenes (a batch of designs or uneven scenes) shard across ranks
  with no data-path collective: ``shard_scenes`` balances cells greedily.
* Whole-job throughput is the units all ranks processed over the slowest rank's
  time (``job_throughput``).
* A single grid larger than one GPU splits into y-slabs (the domain
  decomposition of Sec. II); every step needs one row of Ez from the +y
  neighbour before layer 1 and one row of Hx from the -y neighbour before
  layer 2 (the H update reads Ez(j+1), the E update reads Hx(j-1); Sec. III-B
  eqs. (7)-(9)).  ``SlabExchange`` does that exchange per step for host
  arrays.  ``HaloExchange`` does it for slabs with ``ghost`` rows per cut,
  which advance up to ``ghost`` steps between exchanges (the library's slab
  contexts, fdtd_create_slab, with CUDA tensors over NCCL; host slabs with CPU
  tensors over gloo); ``exchange_local`` refreshes slabs held by one process
  (several slabs on one GPU).  Every exchange is point-to-point into the
  receiver's own memory: no peer loads.
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
            buf = torch.from_numpy(np.empty_like(recv_row))   # the row's own dtype (float32 or float64)
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


def exchange_local(slabs, bufs=None):
    """Refresh the ghost rows of slabs held by one process (ordered bottom to
    top, each holding the rows above the previous one's): at every cut the lower
    slab's top owned rows go to the upper slab's lower ghost rows and the upper
    slab's bottom owned rows to the lower slab's upper ghost rows, through
    buffers allocated once (CUDA tensors for the library's slabs, so each copy is
    a device-to-device copy into the receiver's own memory).  The exports of a
    cut read owned rows and the imports write ghost rows, so their order does
    not matter.  Returns the buffers for reuse."""
    import torch
    if bufs is None:
        bufs = []
        for a in slabs[:-1]:
            n = a.halo_count()
            dev = "cuda" if getattr(a, "on_device", True) else "cpu"
            bufs.append((torch.empty(n, dtype=torch.float32, device=dev),
                         torch.empty(n, dtype=torch.float32, device=dev)))
    for (a, b), (up, down) in zip(zip(slabs[:-1], slabs[1:]), bufs):
        a.halo_export(1, up)
        b.halo_export(0, down)
        b.halo_import(0, up)
        a.halo_import(1, down)
    return bufs


class HaloExchange:
    """Ghost-row exchange of a y-slab decomposition across ranks, for any slab
    with ``halo_count()``, ``halo_export(side, buf)`` and ``halo_import(side,
    buf)`` (side 0: the cut below the owned rows, 1: above).  Each exchange
    exports the owned rows next to every cut, sends them to the neighbour across
    it, receives that neighbour's rows and imports them into the ghost rows:
    point-to-point messages into the receiver's own buffers.  Tags tell the two
    directions apart (gloo; NCCL ignores tags but keeps the order of the one
    message per direction between a pair of ranks)."""

    def __init__(self, slab, rank, world, device="cpu", dtype=None, group=None):
        import torch
        self.slab, self.rank, self.world, self.group = slab, rank, world, group
        self.device = torch.device(device)
        n = slab.halo_count()
        dt = dtype or torch.float32
        self.nbr = {}
        if rank > 0:
            self.nbr[0] = rank - 1
        if rank + 1 < world:
            self.nbr[1] = rank + 1
        self.send = {s: torch.empty(n, dtype=dt, device=self.device) for s in self.nbr}
        self.recv = {s: torch.empty(n, dtype=dt, device=self.device) for s in self.nbr}

    def exchange(self):
        import torch
        import torch.distributed as dist
        for side in self.nbr:
            self.slab.halo_export(side, self.send[side])
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)   # the exports ran on the slab's stream
        reqs = []
        for side, peer in self.nbr.items():
            # tag 1: rows travelling up (sent across the upper cut), tag 2: down
            reqs.append(dist.isend(self.send[side], peer, group=self.group, tag=1 if side == 1 else 2))
            reqs.append(dist.irecv(self.recv[side], peer, group=self.group, tag=2 if side == 1 else 1))
        for r in reqs:
            r.wait()
        for side in self.nbr:
            self.slab.halo_import(side, self.recv[side])
