"""GPU: the paper's split-field PML (Berenger, Sec. III-C) through the C ABI
(FDTD_SPLIT_PML) against the FP64 split-field oracle, its absorption, and the
inputs it refuses."""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import TOL_FIELD, rel_l2

pytestmark = pytest.mark.gpu
C0 = 299792458.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _gpu(sc, nsteps, probes, kernel=0, tblock=4, segment=24):
    from paper_2405_00814_gb300 import fdtd
    sim = fdtd.from_scene(sc, boundary="split", probes=False)
    sim.set_option("kernel", kernel)
    sim.set_option("tblock", tblock)
    sim.set_option("segment", segment)
    pids = [sim.add_probe(int(i), int(j)) for i, j in probes]
    sim.step(nsteps)
    out = {c: sim.get_field(c, (sc.ny, sc.nx)) for c in ("ez", "hx", "hy")}
    out["probes"] = np.stack([sim.read_probe(p, nsteps) for p in pids], 1) if pids else None
    sim.close()
    return out


@pytest.mark.parametrize("kernel,tblock,segment", [(1, 1, 64), (0, 4, 24), (0, 3, 16), (0, 2, 56), (0, 1, 8)])
@pytest.mark.parametrize("side,nsteps", [(200, 700), (131, 500)])
def test_split_pml_matches_oracle(oracle_mod, side, nsteps, kernel, tblock, segment):
    """Heterogeneous lossy interior, vacuum layer of 16 (12) cells, probes (one
    in the layer); the unfused pair and the temporally blocked split variant."""
    sc = scenes.ellipse_scene(side=side, nsteps=nsteps)
    probes = [(side // 2 + 7, side // 3), (side - sc.npml - 3, side // 2), (5, side - 4)]
    o = oracle_mod.TMzSplit(sc)
    ref = o.run(nsteps, samples=[(i, j, "ez") for i, j in probes])["samples"]
    g = _gpu(sc, nsteps, probes, kernel, tblock, segment)
    assert rel_l2(g["ez"], o.ez()) <= TOL_FIELD
    assert rel_l2(g["hx"], o.state["hx"]) <= TOL_FIELD
    assert rel_l2(g["hy"], o.state["hy"]) <= TOL_FIELD
    assert rel_l2(g["probes"], ref) <= TOL_FIELD


def test_split_pml_absorbs_on_the_gpu(oracle_mod):
    """A probe next to a 16-cell layer against an FP64 domain so large that no
    echo returns: the echo stays below -95 dB, as for the oracle."""
    f0 = 2.4e9
    dx = scenes._dx_for(2 * f0, 1.0, 20)
    dt = 0.99 * dx / (C0 * math.sqrt(2))
    nsteps = 900

    def scene(n, npml, off):
        s = scenes.Source(off + 30, off + 60, kind="gauss_mod", params=(f0,))
        return scenes.Scene2D(nx=n, ny=n, dx=dx, dy=dx, dt=dt, npml=npml, mat=np.zeros((n, n), np.uint8),
                              eps_r=np.array([1.0]), sigma=np.array([0.0]), nsteps=nsteps, source=s)

    small = _gpu(scene(120, 16, 0), nsteps, [(24, 60)])["probes"][:, 0]
    big = oracle_mod.TMz(scene(120 + 1800, 0, 900), nsteps_src=nsteps).run(
        nsteps, samples=[(924, 960, "ez")])["samples"][:, 0]
    refl = np.max(np.abs(small - big)) / np.max(np.abs(big))
    assert 20 * math.log10(refl) < -95.0


def test_split_pml_refusals():
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=128, nsteps=10)
    bad = scenes.ellipse_scene(side=128, nsteps=10)
    bad.mat = bad.mat.copy()
    bad.mat[3, 60] = 1                                    # a dielectric cell inside the layer
    with pytest.raises(fdtd.FDTDError):
        fdtd.Simulation(bad, boundary="split")
    sim = fdtd.from_scene(sc, boundary="split")
    with pytest.raises(fdtd.FDTDError):
        sim.set_design(4, 40, np.full((8, 8), 2.0))       # overlaps the layer
    with pytest.raises(fdtd.FDTDError):
        sim.set_checkpointing(10)
    sim.step(8)
    assert np.all(np.isfinite(sim.get_field("ez", (sc.ny, sc.nx))))
    sim.close()


def test_split_pml_literal_graph_matches_oracle(oracle_mod):
    """The 4-node graph of Sec. IV-B through fdtd_step_edgelist: fields and a
    probe against the FP64 split-field oracle."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=150, nsteps=400)
    probes = [(75, 40), (150 - sc.npml - 2, 75)]
    o = oracle_mod.TMzSplit(sc)
    ref = o.run(sc.nsteps, samples=[(i, j, "ez") for i, j in probes])["samples"]
    sim = fdtd.from_scene(sc, boundary="split", probes=False)
    pids = [sim.add_probe(i, j) for i, j in probes]
    sim.step_edgelist(sc.nsteps)
    assert rel_l2(sim.get_field("ez", (sc.ny, sc.nx)), o.ez()) <= TOL_FIELD
    assert rel_l2(sim.get_field("hx", (sc.ny, sc.nx)), o.state["hx"]) <= TOL_FIELD
    assert rel_l2(np.stack([sim.read_probe(p, sc.nsteps) for p in pids], 1), ref) <= TOL_FIELD
    sim.close()


def test_split_pml_exported_graph_is_the_oracle_graph(oracle_mod):
    """Same nodes, same edges in the same order, weights equal to FP32 rounding."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=64, nsteps=10, npml=8)
    o = oracle_mod.TMzSplit(sc)
    sim = fdtd.from_scene(sc, boundary="split")
    for layer in (1, 2):
        n, src, dst, w = sim.export_graph(layer)
        r, c, wo = o.graph_layer(layer)
        assert n == 4 * sc.nx * sc.ny
        dst_o = np.repeat(np.arange(n), np.diff(r))
        assert np.array_equal(dst, dst_o)
        assert np.array_equal(src, c)
        assert np.max(np.abs(w - wo) / np.maximum(np.abs(wo), 1e-30)) <= 2e-6
    sim.close()


@pytest.mark.parametrize("tblock,segment", [(4, 24), (3, 40)])
def test_split_pml_fused_design_and_line_source_in_layer(oracle_mod, tblock, segment):
    """The temporally blocked split variant with a design rectangle (its own
    coefficients) and a line source that starts inside the x-layer."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=170, nsteps=600)
    rng = np.random.default_rng(8)
    sc.design = (40, 50, 33, 21)
    sc.design_eps = 1 + 7 * rng.random((21, 33))
    sc.source = scenes.Source(9, 60, kind="gauss_mod", params=(2.4e9,), length=20)
    probes = [(9, 70), (60, 60), (150, 160)]
    o = oracle_mod.TMzSplit(sc)
    ref = o.run(sc.nsteps, samples=[(i, j, "ez") for i, j in probes])["samples"]
    sim = fdtd.from_scene(sc, boundary="split", probes=False)
    sim.set_option("tblock", tblock)
    sim.set_option("segment", segment)
    pids = [sim.add_probe(i, j) for i, j in probes]
    sim.step(sc.nsteps)
    assert rel_l2(sim.get_field("ez", (sc.ny, sc.nx)), o.ez()) <= TOL_FIELD
    assert rel_l2(sim.get_field("hy", (sc.ny, sc.nx)), o.state["hy"]) <= TOL_FIELD
    assert rel_l2(np.stack([sim.read_probe(p, sc.nsteps) for p in pids], 1), ref) <= TOL_FIELD
    sim.close()


def test_split_pml_autotune_and_graph(oracle_mod):
    """The autotuner's pick (no persistent kernel for a split layer) and CUDA-graph
    replay of the fused split solve."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=160, nsteps=400)
    o = oracle_mod.TMzSplit(sc)
    o.run(sc.nsteps)
    sim = fdtd.from_scene(sc, boundary="split")
    tune = sim.autotune(trial_steps=8)
    assert tune["options"]["kernel"] == 0
    sim.set_option("graph", 1)
    for _ in range(2):
        sim.reset()
        sim.step(sc.nsteps)
    assert rel_l2(sim.get_field("ez", (sc.ny, sc.nx)), o.ez()) <= TOL_FIELD
    sim.close()
