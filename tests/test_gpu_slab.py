"""GPU: y-slab sub-domains of one grid (the domain decomposition of Sec. II)
advanced as separate contexts on one GPU, their ghost rows refreshed between
blocks of steps by device-to-device copies into each receiver's own buffers.
The owned rows must equal the single-context run of the same scene (and the
FP64 oracle)."""
import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import TOL_FIELD, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _whole(sc, nsteps, tblock, probe):
    from paper_2405_00814_gb300 import fdtd
    sim = fdtd.from_scene(sc, probes=False, monitors=False)
    sim.set_option("tblock", tblock)
    pid = sim.add_probe(*probe)
    sim.step(nsteps)
    out = {c: sim.get_field(c, (sc.ny, sc.nx)) for c in ("ez", "hx", "hy")}
    out["probe"] = sim.read_probe(pid, nsteps)
    sim.close()
    return out


def _slabs(sc, nsteps, tblock, cuts, kernel=0, probe=None):
    from paper_2405_00814_gb300 import dist as gd
    from paper_2405_00814_gb300 import fdtd
    g = tblock
    rows = list(zip([0] + cuts, cuts + [sc.ny]))
    slabs = [fdtd.Simulation.slab(sc, j0, j1, g) for j0, j1 in rows]
    pid = None
    for s, (j0, j1) in zip(slabs, rows):
        s.set_option("tblock", tblock)
        s.set_option("kernel", kernel)
        if probe is not None and j0 <= probe[1] < j1:
            pid = (s, s.add_probe(probe[0], probe[1] - s.slab_rows[2]))
    bufs = None
    done = 0
    while done < nsteps:
        n = min(g, nsteps - done)
        for s in slabs:
            s.step(n)
        bufs = gd.exchange_local(slabs, bufs)
        done += n
    out = {c: np.zeros((sc.ny, sc.nx), np.float32) for c in ("ez", "hx", "hy")}
    for s, (j0, j1) in zip(slabs, rows):
        off = s.slab_rows[2]
        for c in out:
            loc = s.get_field(c, (s.shape[1], sc.nx))
            out[c][j0:j1] = loc[j0 - off:j1 - off]
    if pid is not None:
        out["probe"] = pid[0].read_probe(pid[1], nsteps)
    for s in slabs:
        s.close()
    return out


@pytest.mark.parametrize("tblock,cuts,kernel", [
    (1, [100], 0),            # one step per exchange, one cut
    (4, [100], 0),            # four steps per exchange (the fused T = 4 wavefront)
    (4, [9, 150], 0),         # three slabs; the lower cut lies inside the 16-cell CPML
    (3, [77, 141], 1),        # unfused pair, three steps between exchanges
])
def test_slabs_equal_the_single_context_run(tblock, cuts, kernel):
    sc = scenes.ellipse_scene(side=232, nsteps=260, npml=16)
    nsteps = 258                          # not a multiple of the block: a short last block
    probe = (101, 181)
    ref = _whole(sc, nsteps, tblock, probe)
    got = _slabs(sc, nsteps, tblock, cuts, kernel=kernel, probe=probe)
    for c in ("ez", "hx", "hy"):
        e = rel_l2(got[c], ref[c])
        assert e <= 1e-6, (c, e)
    assert rel_l2(got["probe"], ref["probe"]) <= 1e-6
    orc = oracle_run(sc, nsteps)
    for c in ("ez", "hx", "hy"):
        assert rel_l2(got[c], orc[c]) <= TOL_FIELD, c


def test_slab_contract_errors():
    import torch
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=96, nsteps=10, npml=8)
    lo = fdtd.Simulation.slab(sc, 0, 48, 2)
    hi = fdtd.Simulation.slab(sc, 48, 96, 2)
    assert lo.slab_rows == (0, 48, 0) and hi.slab_rows == (48, 96, 46)
    assert lo.halo_count() == 7 * 2 * 96
    with pytest.raises(fdtd.FDTDError) as ei:
        lo.step(3)                                         # more steps than ghost rows
    assert ei.value.code == fdtd.EINVAL
    buf = torch.empty(lo.halo_count(), dtype=torch.float32, device="cuda")
    with pytest.raises(fdtd.FDTDError):
        lo.halo_export(0, buf)                             # no neighbour below the grid's first row
    with pytest.raises(ValueError):
        lo.halo_export(1, torch.empty(5, dtype=torch.float32, device="cuda"))
    for call in (lambda: lo.step_edgelist(1), lambda: lo.set_design(10, 10, np.ones((4, 4))),
                 lambda: lo.set_checkpointing(10)):
        with pytest.raises(fdtd.FDTDError):
            call()
    with pytest.raises(fdtd.FDTDError):
        fdtd.Simulation.slab(sc, 10, 11, 2)                # fewer owned rows than ghost rows
    lo.close()
    hi.close()
