"""GPU parity of the literal edge-list path (Prop. 1 graph, Prop. 2 layers)."""
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


def _edgelist_run(sc, n):
    from paper_2405_00814_gb300 import fdtd
    sim = fdtd.from_scene(sc)
    sim.step_edgelist(n)
    res = {c: sim.get_field(c, (sc.ny, sc.nx)) for c in ("ez", "hx", "hy")}
    res["probes"] = np.stack([sim.read_probe(p, n) for p in sim.probe_ids], 1) if sim.probe_ids else None
    if sim.mon_id is not None:
        res["dft"] = sim.read_dft(sim.mon_id)
    sim.close()
    return res


@pytest.mark.parametrize("side,npml", [(96, 0), (150, 12)])
def test_edgelist_matches_oracle(side, npml):
    sc = scenes.ellipse_scene(side=side, nsteps=500, npml=max(npml, 1)) if npml else scenes.cavity_ricker(n=side, nsteps=500)
    o = oracle_run(sc, 500, probes=sc.probes)
    g = _edgelist_run(sc, 500)
    assert_fields_close(g, o)
    assert rel_l2(g["probes"], o["probes"]) <= TOL_FIELD


def test_edgelist_with_design_and_dft():
    sc = scenes.adjoint_scenes(side=128, n_designs=1, nsteps=700, npml=10, design=24)[0]
    o = oracle_run(sc, 700, monitors=sc.monitors, freqs=sc.freqs)
    g = _edgelist_run(sc, 700)
    assert_fields_close(g, o)
    assert np.max(np.abs(g["dft"] - o["dft"])) <= 1e-4 * np.max(np.abs(o["dft"]))


def test_exported_graph_is_the_oracle_graph():
    """The library's explicit graph has exactly the oracle's Prop. 1 edge set,
    and weights equal to FP32 rounding."""
    import oracle
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=40, nsteps=10, npml=6)
    sim = fdtd.from_scene(sc)
    ref = oracle.TMz(sc)
    for layer in (1, 2):
        nn, src, dst, w = sim.export_graph(layer)
        rowptr, col, wr = ref.graph_layer(layer)
        assert nn == len(rowptr) - 1
        assert len(src) == len(col)
        dst_ref = np.repeat(np.arange(nn), np.diff(rowptr))
        a = np.lexsort((src, dst))
        b = np.lexsort((col, dst_ref))
        assert np.array_equal(dst[a], dst_ref[b]) and np.array_equal(src[a], col[b])
        scale = np.maximum(np.abs(wr[b]), 1e-30)
        big = np.abs(wr[b]) > 1e-6 * np.max(np.abs(wr))
        assert np.max(np.abs(w[a] - wr[b])[big] / scale[big]) < 2e-6
    sim.close()
