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
