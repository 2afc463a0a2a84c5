"""Multi-process host logic on CPU ranks (gloo, world size 2): scene sharding,
whole-job throughput, and the y-slab halo exchange, which must reproduce the
single-rank oracle run exactly."""
import os
import socket

import numpy as np
import pytest

from paper_2405_00814_gb300 import dist as gd
from paper_2405_00814_gb300 import scenes


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run(fn, world, *args):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_entry, args=(fn, r, world, port, q, args)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for r in res:
        if isinstance(r, BaseException):
            raise r
    return sorted(res, key=lambda x: x[0])


def _entry(fn, rank, world, port, q, args):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        out = globals()[fn](rank, world, *args)
        dist.destroy_process_group()
        q.put((rank, out))
    except BaseException as e:  # report to the parent
        q.put(e)


def test_shard_scenes_partitions_and_balances():
    cells = [s.cells for s in scenes.batch_scenes()]
    for world in (2, 3, 8):
        sh = gd.shard_scenes(cells, world)
        flat = sorted(k for part in sh for k in part)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[k] for k in part) for part in sh]
        assert max(loads) - min(loads) <= max(cells)


def _throughput(rank, world):
    units = [100.0, 300.0][rank]
    secs = [2.0, 4.0][rank]
    return gd.job_throughput(units, secs)


def test_job_throughput_sums_units_over_max_time():
    res = _run("_throughput", 2)
    for _, v in res:
        assert v == pytest.approx(400.0 / 4.0)


def _slab_run(rank, world, nsteps):
    import oracle
    sc = scenes.cavity_ricker(n=64, nsteps=nsteps)
    ny, nx = sc.ny, sc.nx
    eps = 1.0 + 3.0 * scenes.random_fields(9, (ny, nx)) ** 2
    ex = gd.SlabExchange(ny, rank, world)
    lo, hi = ex.j0 - ex.g0, ex.j1 + ex.g1
    src = sc.source if ex.j0 <= sc.source.j < ex.j1 else None
    if src is not None:
        src = scenes.Source(src.i, src.j - lo, kind=src.kind, params=src.params)
    sim = oracle.TMz(nx=nx, ny=hi - lo, dx=sc.dx, dy=sc.dy, dt=sc.dt, eps_cell=eps[lo:hi], source=src,
                     nsteps_src=nsteps, with_source=src is not None)
    st = sim.state
    for n in range(nsteps):
        ex.ez_up(st["ez"])
        sim.layer_h()
        ex.h_down(st["hx"], st["hy"])
        sim.layer_e()
        if src is not None:
            st["ez"][src.j, src.i] += sim.src[n]
    return {k: ex.owned(st[k]).copy() for k in ("ez", "hx", "hy")}, (ex.j0, ex.j1)


def test_slab_halo_exchange_equals_single_rank():
    import oracle
    nsteps = 120
    res = _run("_slab_run", 2, nsteps)
    sc = scenes.cavity_ricker(n=64, nsteps=nsteps)
    eps = 1.0 + 3.0 * scenes.random_fields(9, (sc.ny, sc.nx)) ** 2
    ref = oracle.TMz(nx=sc.nx, ny=sc.ny, dx=sc.dx, dy=sc.dy, dt=sc.dt, eps_cell=eps, source=sc.source,
                     nsteps_src=nsteps)
    ref.run(nsteps)
    for _, (fields, (j0, j1)) in res:
        for k in ("ez", "hx", "hy"):
            assert np.array_equal(fields[k], ref.state[k][j0:j1]), k


class _OracleSlab:
    """A host slab for the exchange logic: the FP64 oracle over rows
    [j0 - ghost, j1 + ghost) of a CPML scene (ghost rows only where a
    neighbour is), the y-profile taken from the whole grid, any source cell that
    falls in its rows set in local coordinates.  It offers the halo calls of the
    library's slab contexts (packed [array][ghost][nx] rows in a CPU tensor)."""

    ARRAYS = ("ez", "hx", "hy", "pezx", "pezy", "phxy", "phyx")

    def __init__(self, sc, j0, j1, ghost, nsteps):
        import oracle
        self.g, self.nx = ghost, sc.nx
        self.glo = ghost if j0 > 0 else 0
        self.ghi = ghost if j1 < sc.ny else 0
        self.j0, self.j1 = j0, j1
        lo, hi = j0 - self.glo, j1 + self.ghi
        self.lo, self.ny = lo, hi - lo
        src = sc.source if lo < sc.source.j < hi else None
        if src is not None:
            src = scenes.Source(src.i, src.j - lo, kind=src.kind, params=src.params)
        eps = sc.eps_r[sc.mat].astype(np.float64)
        sig = sc.sigma[sc.mat].astype(np.float64)
        self.sim = oracle.TMz(nx=sc.nx, ny=self.ny, dx=sc.dx, dy=sc.dy, dt=sc.dt, npml=sc.npml,
                              eps_cell=eps[lo:hi], sigma_cell=sig[lo:hi], source=src, nsteps_src=nsteps,
                              with_source=src is not None)
        whole = oracle.cpml_axis(sc.ny, sc.npml, sc.dy, sc.dt)
        for k, v in whole.items():
            self.sim.py[k][:] = v[lo:hi]          # bound by pointer: written in place

    def halo_count(self):
        return len(self.ARRAYS) * self.g * self.nx

    def halo_export(self, side, buf):
        r0 = self.glo if side == 0 else self.ny - self.ghi - self.g
        rows = np.stack([self.sim.state[a][r0:r0 + self.g] for a in self.ARRAYS])
        buf.numpy()[:] = rows.ravel()

    def halo_import(self, side, buf):
        r0 = 0 if side == 0 else self.ny - self.ghi
        rows = buf.numpy().reshape(len(self.ARRAYS), self.g, self.nx)
        for k, a in enumerate(self.ARRAYS):
            self.sim.state[a][r0:r0 + self.g] = rows[k]

    def owned(self):
        return {k: self.sim.state[k][self.glo:self.ny - self.ghi].copy() for k in ("ez", "hx", "hy")}


def _halo_run(rank, world, cuts, ghost, nsteps):
    import torch
    sc = scenes.ellipse_scene(side=72, nsteps=nsteps, npml=8)
    rows = list(zip([0] + cuts, cuts + [sc.ny]))
    slab = _OracleSlab(sc, *rows[rank], ghost, nsteps)
    ex = gd.HaloExchange(slab, rank, world, dtype=torch.float64)
    done = 0
    while done < nsteps:
        n = min(ghost, nsteps - done)
        slab.sim.run(n)
        ex.exchange()
        done += n
    return slab.owned(), rows[rank]


@pytest.mark.parametrize("world,cuts,ghost", [(2, [36], 1), (2, [40], 4), (3, [5, 44], 3)])
def test_halo_exchange_of_ghost_depth_equals_single_rank(world, cuts, ghost):
    """Slabs that advance `ghost` steps between exchanges (the temporally
    blocked form of the GPU slab contexts) reproduce the single-rank run bit for
    bit; in the three-slab case the first cut lies inside the CPML, so the psi
    arrays travel with the fields."""
    import oracle
    nsteps = 97
    res = _run("_halo_run", world, cuts, ghost, nsteps)
    sc = scenes.ellipse_scene(side=72, nsteps=nsteps, npml=8)
    ref = oracle.TMz(sc, nsteps_src=nsteps)
    ref.run(nsteps)
    for _, (fields, (j0, j1)) in res:
        for k in ("ez", "hx", "hy"):
            assert np.array_equal(fields[k], ref.state[k][j0:j1]), (k, j0, j1)


def _f32_swap(rank, world):
    ex = gd.SlabExchange(16, rank, world)
    ez = np.full((ex.local_rows, 5), 10.0 * rank + 1, np.float32)
    hx = np.full((ex.local_rows, 5), 10.0 * rank + 2, np.float32)
    hy = np.full((ex.local_rows, 5), 10.0 * rank + 3, np.float32)
    ex.ez_up(ez)
    ex.h_down(hx, hy)
    if rank == 0:
        return ez[-1].copy(), None            # Ez ghost above, from rank 1
    return hx[0].copy(), hy[0].copy()         # H ghosts below, from rank 0


def test_slab_exchange_keeps_float32_rows():
    res = dict(_run("_f32_swap", 2))
    ez_ghost = res[0][0]
    hx_ghost, hy_ghost = res[1]
    assert ez_ghost.dtype == np.float32 and np.all(ez_ghost == 11.0)     # rank 1's first Ez row
    assert np.all(hx_ghost == 2.0) and np.all(hy_ghost == 3.0)          # rank 0's last H rows
