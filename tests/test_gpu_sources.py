"""GPU: the paper's other sources and its photonic-crystal example (Sec. V-A,
V-B) -- sinusoidal and line sources, through the temporally blocked, unfused
and literal-graph paths -- against the FP64 oracle."""
import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import TOL_FIELD, assert_fields_close, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(sc, nsteps, path, **opts):
    from paper_2405_00814_gb300 import fdtd
    sim = fdtd.from_scene(sc)
    for k, v in opts.items():
        sim.set_option(k, v)
    if path == "edgelist":
        sim.step_edgelist(nsteps)
    else:
        sim.step(nsteps)
    out = {c: sim.get_field(c, (sc.ny, sc.nx)) for c in ("ez", "hx", "hy")}
    out["probes"] = np.stack([sim.read_probe(p, nsteps) for p in sim.probe_ids], 1)
    out["te_ey"] = sim.get_field_te("ey", (sc.ny, sc.nx))
    sim.close()
    return out


def test_photonic_crystal_waveguide():
    """The photonic-crystal example: 75 THz pulse launched by a line source
    across the eps_r = 12 waveguide, two groups of three air holes; fields and
    the two probe waveforms (the sampled waveform of the example) match the
    oracle."""
    sc = scenes.phc_waveguide()
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    g = _run(sc, sc.nsteps, "fused")
    assert_fields_close(g, o)
    assert rel_l2(g["probes"], o["probes"]) <= TOL_FIELD
    assert np.array_equal(g["te_ey"], -g["ez"])
    # the pulse reached the far probe
    assert np.max(np.abs(o["probes"][:, 1])) > 1e-3 * np.max(np.abs(o["probes"][:, 0]))


@pytest.mark.parametrize("path,opts", [("fused", {"tblock": 4, "segment": 16}), ("fused", {"tblock": 3, "segment": 24}),
                                       ("unfused", {"kernel": 1}), ("edgelist", {})])
def test_sine_line_source_paths(path, opts):
    """A continuous sinusoid on a 25-cell line crossing several row segments,
    heterogeneous lossy medium with a CPML, on every stepping path."""
    sc = scenes.ellipse_scene(side=180, nsteps=400)
    sc.source = scenes.Source(60, 70, kind="sine", params=(8e9,), length=25)
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    g = _run(sc, sc.nsteps, path, **opts)
    assert_fields_close(g, o)
    assert rel_l2(g["probes"], o["probes"]) <= TOL_FIELD


def test_te_graph_export_steps_te_fields():
    """The library's exported graph under the TE naming (export_graph(te=True))
    advances TE node values built from get_field_te as the GPU step does."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=64, nsteps=1, npml=0)
    rng = np.random.default_rng(3)
    sim = fdtd.from_scene(sc, source=False, probes=False, monitors=False)
    ez = rng.standard_normal((sc.ny, sc.nx)).astype(np.float32)
    ez[0, :] = 0.0
    ez[:, 0] = 0.0
    sim.set_field("ez", ez)
    sim.set_field("hx", rng.standard_normal((sc.ny, sc.nx)).astype(np.float32))
    sim.set_field("hy", rng.standard_normal((sc.ny, sc.nx)).astype(np.float32))
    shp = (sc.ny, sc.nx)
    te = {c: sim.get_field_te(c, shp).astype(np.float64) for c in ("ey", "hx", "hz")}
    n, src, dst, w1 = sim.export_graph(1, te=True)
    _, src2, dst2, w2 = sim.export_graph(2, te=True)
    nx = sc.nx
    h = np.zeros(n)
    for j in range(sc.ny):
        b = 3 * j * nx
        h[b:b + nx] = te["hx"][j]                       # u = i + 3 k nx
        h[b + nx:b + 3 * nx:2] = te["hz"][j]            # q = 2 i + nx (3 k + 1)
        h[b + nx + 1:b + 3 * nx:2] = te["ey"][j]        # t = 2 i + 1 + nx (3 k + 1)
    h1 = np.zeros(n)
    np.add.at(h1, dst, w1 * h[src])
    h2 = np.zeros(n)
    np.add.at(h2, dst2, w2 * h1[src2])
    sim.step(1)
    for name, sl in (("ey", lambda b: slice(b + nx + 1, b + 3 * nx, 2)), ("hz", lambda b: slice(b + nx, b + 3 * nx, 2)),
                     ("hx", lambda b: slice(b, b + nx))):
        got = np.stack([h2[sl(3 * j * nx)] for j in range(sc.ny)])
        assert rel_l2(got, sim.get_field_te(name, shp)) <= 1e-5, name
    sim.close()
