"""GPU: fdtd_set_materials -- a new geometry in an existing context (the map
uploaded into the padded layout, PEC walls re-marked, coefficient table, design
band and edge-list weights refreshed) steps bit for bit like a context created
from that geometry, on the blocked, graph-replayed and edge-list paths."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pair(side=300, nsteps=200):
    a = scenes.ellipse_scene(side=side, nsteps=nsteps, seed_id=2)
    b0 = scenes.ellipse_scene(side=side, nsteps=nsteps, seed_id=9)
    b = dataclasses.replace(a, mat=b0.mat, eps_r=b0.eps_r, sigma=b0.sigma)
    assert not np.array_equal(a.mat, b.mat)
    return a, b


def _fields(sim, sc):
    out = {c: sim.get_field(c, (sc.ny, sc.nx)) for c in ("ez", "hx", "hy")}
    out["probes"] = np.stack([sim.read_probe(p, sc.nsteps) for p in sim.probe_ids], 1)
    return out


def _same(x, y):
    for k in x:
        assert np.array_equal(x[k], y[k]), k


@pytest.mark.parametrize("graph", [False, True])
def test_switch_equals_fresh_context(graph):
    from paper_2405_00814_gb300 import fdtd
    a, b = _pair()
    ref = fdtd.from_scene(b)
    ref.set_option("tblock", 4)
    ref.set_option("segment", 24)
    ref.step(b.nsteps)
    want = _fields(ref, b)
    ref.close()
    sim = fdtd.from_scene(a)
    sim.set_option("tblock", 4)
    sim.set_option("segment", 24)
    sim.set_option("graph", int(graph))
    sim.step(a.nsteps)                      # a solve of the first geometry (records the graph)
    sim.reset()
    sim.set_materials(b.mat, b.eps_r, b.sigma)
    sim.step(b.nsteps)                      # replayed from the graph when graph = 1
    _same(_fields(sim, b), want)
    sim.close()


def test_switch_with_design_and_edge_list():
    from paper_2405_00814_gb300 import fdtd
    a, b = _pair(side=200, nsteps=120)
    rng = np.random.default_rng(4)
    eps_d = 1 + 8 * rng.random((30, 41))
    res = []
    for first in (b, a):
        sim = fdtd.from_scene(first)
        sim.set_design(70, 60, eps_d)
        sim.step_edgelist(5)                # builds the edge-list weights of the first geometry
        sim.reset()
        if first is a:
            sim.set_materials(b.mat, b.eps_r, b.sigma)
        sim.step(b.nsteps)
        f1 = _fields(sim, b)
        sim.reset()
        sim.step_edgelist(b.nsteps)
        f2 = _fields(sim, b)
        sim.close()
        res.append((f1, f2))
    _same(res[1][0], res[0][0])
    _same(res[1][1], res[0][1])


def test_unlisted_index_acts_as_pec():
    """A cell whose index is >= n_mat gets zero coefficients: its Ez stays 0."""
    from paper_2405_00814_gb300 import fdtd
    a, _ = _pair(side=128, nsteps=150)
    mat = a.mat.copy()
    mat[70, 60] = 200
    sim = fdtd.from_scene(a)
    sim.set_materials(mat, a.eps_r, a.sigma)
    sim.step(a.nsteps)
    ez = sim.get_field("ez", (a.ny, a.nx))
    assert ez[70, 60] == 0.0
    assert np.max(np.abs(ez)) > 0
    sim.close()


def test_set_materials_refusals():
    from paper_2405_00814_gb300 import fdtd
    a, b = _pair(side=96, nsteps=10)
    sim = fdtd.from_scene(a)
    with pytest.raises(fdtd.FDTDError):
        sim.set_materials(b.mat, np.array([]), np.array([]))
    with pytest.raises(fdtd.FDTDError):
        sim.set_materials(b.mat, np.array([1.0, -2.0]), np.array([0.0, 0.0]))
    sim.close()
    sp = fdtd.from_scene(a, boundary="split")
    bad = a.mat.copy()
    bad[2, 40] = 1                           # inside the split-field layer
    with pytest.raises(fdtd.FDTDError):
        sp.set_materials(bad, a.eps_r, a.sigma)
    sp.set_materials(a.mat, a.eps_r, a.sigma)
    sp.close()
    n = 8
    s3 = scenes.Scene3D(nx=n, ny=n, nz=n, dx=1e-3, dy=1e-3, dz=1e-3, dt=1e-12 / math.sqrt(3), npml=0,
                        mat=np.zeros((n, n, n), np.uint8), eps_r=np.array([1.0]), sigma=np.array([0.0]), nsteps=1)
    sim3 = fdtd.from_scene(s3, source=False)
    with pytest.raises(fdtd.FDTDError):
        sim3.set_materials(np.zeros((n * n, n), np.uint8), np.array([1.0]), np.array([0.0]))
    sim3.close()


def test_set_materials_in_a_batch_touches_only_the_selected_scene():
    from paper_2405_00814_gb300 import fdtd
    a, b = _pair(side=160, nsteps=150)
    c = scenes.ellipse_scene(side=200, nsteps=150, seed_id=4)
    ref = fdtd.Simulation.batch([b, c])
    for k, s in enumerate((b, c)):
        ref.select(k)
        ref.set_scene_source(s.source)
    ref.step(150)
    want = []
    for k, s in enumerate((b, c)):
        ref.select(k)
        want.append(ref.get_field("ez", (s.ny, s.nx)))
    ref.close()
    sim = fdtd.Simulation.batch([a, c])
    for k, s in enumerate((a, c)):
        sim.select(k)
        sim.set_scene_source(s.source)
    sim.select(0)
    sim.set_materials(b.mat, b.eps_r, b.sigma)
    sim.step(150)
    for k, s in enumerate((b, c)):
        sim.select(k)
        assert np.array_equal(sim.get_field("ez", (s.ny, s.nx)), want[k]), k
    sim.close()


def test_buffers_of_the_wrong_size_are_refused():
    """The binding checks every buffer the library reads or writes against the
    selected scene's size before the call (a short buffer would be overrun)."""
    import torch
    from paper_2405_00814_gb300 import fdtd
    a, _ = _pair(side=64, nsteps=10)
    c = scenes.ellipse_scene(side=80, nsteps=10, seed_id=4)
    sim = fdtd.Simulation.batch([a, c])
    with pytest.raises(ValueError):
        sim.get_field("ez", (64, 63))
    with pytest.raises(ValueError):
        sim.get_field("ez", out=torch.empty(64 * 64 - 1, device="cuda"))
    with pytest.raises(ValueError):
        sim.set_field("hx", np.zeros((64, 65), np.float32))
    with pytest.raises(ValueError):
        sim.set_materials(np.zeros((80, 80), np.uint8), a.eps_r, a.sigma)
    sim.select(1)
    assert sim.get_field("ez", (80, 80)).shape == (80, 80)
    with pytest.raises(ValueError):
        sim.get_field("ez", (64, 64))
    sim.close()
