"""GPU vs FP64 oracle, one check per benchmark configuration (at sizes the
oracle finishes in seconds), each measured error printed as a `PARITY` line so
that a run with -s states the error of every result: fields and probes (rel L2
at the last step), running DFTs (max |dF| / max |F|, and per monitor value
against max(|F|, 1e-2 max |F|); compensated FP32), the eps_r gradient
(per-cell error against the FP64 adjoint)."""
import json
import os

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import TOL_FIELD, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu
TOL_DFT = 1e-4
TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def r2(x, ref):
    """Coefficient of determination of x against ref (the agreement statistic the
    paper quotes over its validation scenes, Sec. V-A)."""
    x = np.asarray(x, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    return 1.0 - float(np.sum((x - ref) ** 2)) / float(np.sum((ref - ref.mean()) ** 2))


def _report(config, result, err, tol, r2v=None):
    line = {"config": config, "result": result, "error": float(err), "tol": tol}
    if r2v is not None:
        line["r2"] = r2v
    print("PARITY " + json.dumps(line))
    path = os.environ.get("PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")
    assert err <= tol, line


def _dft_err(g, o):
    return float(np.max(np.abs(g - o)) / np.max(np.abs(o)))


# per monitor value: |dF| / max(|F|, floor), floor = 1e-2 max |F| over the
# monitor (as the gradient's per-cell measure), so that values near a zero of
# the spectrum are measured against the monitor's scale
DFT_FLOOR = 1e-2


def _dft_err_per_value(g, o):
    o = np.asarray(o)
    den = np.maximum(np.abs(o), DFT_FLOOR * np.max(np.abs(o)))
    return float(np.max(np.abs(np.asarray(g) - o) / den))


# a component whose norm is a share s < 0.1 of its vector field's is bounded by
# its own norm at TOL_FIELD * 0.1 / s: an absolute error of at most 1e-5 of the
# vector field's norm, ten times tighter than the bound of the field itself
MINOR_SHARE = 0.1


def _minor_tol(share):
    return TOL_FIELD * MINOR_SHARE / share


def test_cavity_128():
    sc = scenes.cavity_ricker()
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    g = gpu_run(sc, sc.nsteps, tblock=4, segment=32)
    for c in ("ez", "hx", "hy"):
        _report("cavity128_pec_ricker_500", c, rel_l2(g[c], o[c]), TOL_FIELD, r2(g[c], o[c]))
    _report("cavity128_pec_ricker_500", "probes", rel_l2(g["probes"], o["probes"]), TOL_FIELD,
            r2(g["probes"], o["probes"]))


def test_heterogeneous_cpml_with_dft():
    sc = scenes.ellipse_scene(side=512, nsteps=1200)
    rng = np.random.default_rng(12)
    mons = np.stack([rng.integers(20, 492, 6), rng.integers(20, 492, 6)], 1).astype(np.int32)
    sc.monitors, sc.freqs = mons, np.array([1.2e9, 2.4e9, 3.6e9])
    o = oracle_run(sc, sc.nsteps, probes=sc.probes, monitors=mons, freqs=sc.freqs)
    g = gpu_run(sc, sc.nsteps, tblock=4, segment=56, warps=4)
    name = "ellipses512_cpml16_gaussmod_1200"
    for c in ("ez", "hx", "hy"):
        _report(name, c, rel_l2(g[c], o[c]), TOL_FIELD, r2(g[c], o[c]))
    _report(name, "probes", rel_l2(g["probes"], o["probes"]), TOL_FIELD, r2(g["probes"], o["probes"]))
    _report(name, "dft", _dft_err(g["dft"], o["dft"]), TOL_DFT)
    _report(name, "dft (per value)", _dft_err_per_value(g["dft"], o["dft"]), TOL_DFT)


def test_3d_boxes_plane_dft():
    import oracle
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.box_scene(side=64, nsteps=240, npml=8, n_boxes=12)
    sc.dft_plane_k = 44
    n = sc.nsteps
    osim = oracle.Yee3D(sc, nsteps_src=n)
    osim.run(n, plane_k=sc.dft_plane_k, freqs=sc.freqs)
    sim = fdtd.from_scene(sc)
    mid = sim.add_dft_plane(sc.dft_plane_k, ("ex", "ey", "ez"), sc.freqs)
    sim.step(n)
    name = "boxes64^3_cpml8_dipole_240"
    # every component against the norm of its vector field (E or H); a major
    # component (norm >= 0.1 of its field's) also against its own norm at the
    # field tolerance; a minor one against its own norm at _minor_tol(share):
    # its FP32 rounding error scales with the whole field, not with its share.
    vec = {c: float(np.sqrt(sum(np.linalg.norm(osim.state[q]) ** 2 for q in grp)))
           for grp in (("ex", "ey", "ez"), ("hx", "hy", "hz")) for c in grp}
    for c in ("ex", "ey", "ez", "hx", "hy", "hz"):
        got = sim.get_field(c, (sc.nz, sc.ny, sc.nx))
        share = float(np.linalg.norm(osim.state[c])) / vec[c]
        _report(name, c + " (vs its vector field)", rel_l2(got, osim.state[c], floor=vec[c]), TOL_FIELD,
                r2(got, osim.state[c]))
        own = rel_l2(got, osim.state[c])
        if share >= MINOR_SHARE:
            _report(name, c, own, TOL_FIELD)
        else:
            _report(name, f"{c} (minor: {share:.2%} of its field, own norm)", own, _minor_tol(share))
    F, Fo = sim.read_dft(mid), osim.plane[0] + 1j * osim.plane[1]
    _report(name, "dft_plane", _dft_err(F, Fo), TOL_DFT)
    for q, c in enumerate(("ex", "ey", "ez")):
        _report(name, f"dft_plane {c} (per value)", _dft_err_per_value(F[q], Fo[q]), TOL_DFT)
    sim.close()


def test_batch_persistent_graph():
    from paper_2405_00814_gb300 import fdtd
    scs = scenes.batch_scenes(n_scenes=5, nsteps=400, side_lo=200, side_hi=420)
    sim = fdtd.Simulation.batch(scs)
    for k, s in enumerate(scs):
        sim.select(k)
        sim.set_scene_source(s.source)
    sim.set_option("kernel", 2)
    sim.set_option("tblock", 4)
    sim.set_option("segment", 32)
    sim.set_option("graph", 1)
    sim.step(400)
    worst = 0.0
    for k, s in enumerate(scs):
        o = oracle_run(s, s.nsteps)
        sim.select(k)
        for c in ("ez", "hx", "hy"):
            worst = max(worst, rel_l2(sim.get_field(c, (s.ny, s.nx)), o[c]))
    sim.close()
    _report("batch5_sides200-420_persistent_graph_400", "fields (worst scene and component)", worst, TOL_FIELD)


def test_adjoint_gradient():
    import oracle
    from paper_2405_00814_gb300 import autograd
    scs = scenes.adjoint_scenes(side=128, n_designs=2, nsteps=900, npml=10, design=32, n_monitors=4)
    batch = autograd.DesignBatch(scs, ckpt_every=100)
    F = batch.forward(np.stack([s.design_eps for s in scs]))
    g = batch.gradient(2.0 * F)
    batch.close()
    fe, ge = 0.0, 0.0
    for k, sc in enumerate(scs):
        _, fre, fim, gref = oracle.TMz(sc, nsteps_src=sc.nsteps).adjoint_grad(sc.nsteps, 100, sc.monitors, sc.freqs,
                                                                              sc.design)
        fe = max(fe, _dft_err(F[k], fre + 1j * fim))
        den = np.maximum(np.abs(gref), 1e-2 * np.max(np.abs(gref)))
        ge = max(ge, float(np.max(np.abs(g[k] - gref) / den)))
    _report("adjoint128_x2designs_900_ckpt100", "dft", fe, TOL_DFT)
    _report("adjoint128_x2designs_900_ckpt100", "grad_eps_r (per cell)", ge, TOL_GRAD)
