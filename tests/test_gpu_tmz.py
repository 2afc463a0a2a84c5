"""GPU parity of the 2D TMz path (C ABI -> sm_103a kernels) against the FP64
oracle, element by element on the same seeded inputs."""
import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import TOL_FIELD, assert_fields_close, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("kernel,tblock", [(1, 1), (0, 1), (0, 2), (0, 3), (0, 4)])
def test_cavity_ricker_128_full_500_steps(kernel, tblock):
    sc = scenes.cavity_ricker()
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    g = gpu_run(sc, sc.nsteps, kernel=kernel, tblock=tblock, segment=32)
    assert_fields_close(g, o)
    e = rel_l2(g["probes"], o["probes"])
    assert e <= TOL_FIELD, e


@pytest.mark.parametrize("side,segment,warps,tblock", [(256, 128, 2, 4), (250, 40, 1, 3), (250, 8, 4, 4),
                                                        (131, 16, 3, 2)])
def test_heterogeneous_cpml_ragged(side, segment, warps, tblock):
    sc = scenes.ellipse_scene(side=side, nsteps=700)
    if side == 131:   # non-square
        sc.mat = np.ascontiguousarray(sc.mat[:97, :])
        sc.ny = 97
        sc.source.j = 48
        sc.probes = sc.probes[sc.probes[:, 1] < 97]
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    g = gpu_run(sc, sc.nsteps, tblock=tblock, segment=segment, warps=warps)
    assert_fields_close(g, o)
    assert rel_l2(g["probes"], o["probes"]) <= TOL_FIELD


@pytest.mark.parametrize("segment,taper,warps", [(24, 30, 4), (40, 45, 2), (16, 10, 3)])
def test_tapered_interior_list(segment, taper, warps):
    """Half-height tail segments, the interior CTAs run tallest first.  The
    fields match the oracle within TOL and the uniform run to rounding (other
    segment bounds move a few rows between the interior and the general kernel,
    whose FMA contraction may differ)."""
    sc = scenes.ellipse_scene(side=512, nsteps=300)
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    a = gpu_run(sc, sc.nsteps, tblock=4, segment=segment, warps=warps)
    b = gpu_run(sc, sc.nsteps, tblock=4, segment=segment, warps=warps, options={"taper": taper})
    for c in ("ez", "hx", "hy"):
        assert rel_l2(b[c], a[c]) < 1e-5, c
    assert rel_l2(b["probes"], a["probes"]) < 1e-5
    assert_fields_close(b, o)
    assert rel_l2(b["probes"], o["probes"]) <= TOL_FIELD


@pytest.mark.parametrize("warps_b,tblock,segment", [(1, 4, 24), (4, 4, 40), (8, 3, 16), (8, 4, 48)])
def test_cpml_cta_width(warps_b, tblock, segment):
    """The CPML kernels' CTAs of 1 to 8 warps (FDTD_OPT_WARPS_B): the CPML,
    narrow x-slab and lite lists padded to other widths; oracle within TOL and
    the 2-warp run to rounding."""
    sc = scenes.ellipse_scene(side=384, nsteps=400)
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    a = gpu_run(sc, sc.nsteps, tblock=tblock, segment=segment, warps=4)
    b = gpu_run(sc, sc.nsteps, tblock=tblock, segment=segment, warps=4, options={"warps_b": warps_b})
    for c in ("ez", "hx", "hy"):
        assert rel_l2(b[c], a[c]) < 1e-5, c
    assert_fields_close(b, o)
    assert rel_l2(b["probes"], o["probes"]) <= TOL_FIELD


def test_tapered_batch_of_uneven_scenes():
    """The tallest-first order moves whole CTAs between scenes of a batch."""
    from paper_2405_00814_gb300 import fdtd
    scs = scenes.batch_scenes(n_scenes=3, nsteps=400, side_lo=96, side_hi=300)
    sim = fdtd.Simulation.batch(scs)
    for k, s in enumerate(scs):
        sim.select(k)
        sim.set_scene_source(s.source)
    sim.set_option("segment", 24)
    sim.set_option("warps", 4)
    sim.set_option("taper", 40)
    sim.set_option("warps_b", 8)
    assert sim.get_option("taper") == 40 and sim.get_option("warps_b") == 8
    sim.step(400)
    for k, s in enumerate(scs):
        o = oracle_run(s, 400)
        sim.select(k)
        g = {c: sim.get_field(c, (s.ny, s.nx)) for c in ("ez", "hx", "hy")}
        assert_fields_close(g, o)
    sim.close()


@pytest.mark.parametrize("tblock,segment,warps,side", [(4, 68, 8, 512), (3, 24, 4, 384), (2, 16, 2, 250),
                                                        (1, 40, 3, 200)])
def test_bulk_row_copies(tblock, segment, warps, side):
    """FDTD_OPT_BULK: the interior kernel's rows by cp.async.bulk into
    mbarrier-tracked stages.  Same arithmetic on the same values, so the fields
    and probes equal the cp.async run bit for bit; the oracle within TOL."""
    sc = scenes.ellipse_scene(side=side, nsteps=400)
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    a = gpu_run(sc, sc.nsteps, tblock=tblock, segment=segment, warps=warps)
    b = gpu_run(sc, sc.nsteps, tblock=tblock, segment=segment, warps=warps, options={"bulk": 1, "warps_b": 8})
    c = gpu_run(sc, sc.nsteps, tblock=tblock, segment=segment, warps=warps, options={"warps_b": 8})
    for f in ("ez", "hx", "hy"):
        assert np.array_equal(b[f], c[f]), f
    assert np.array_equal(b["probes"], c["probes"])
    assert_fields_close(b, o)
    assert rel_l2(b["probes"], o["probes"]) <= TOL_FIELD
    for f in ("ez", "hx", "hy"):
        assert rel_l2(b[f], a[f]) < 1e-5, f


def test_bulk_row_copies_rectangular_cells_and_graph():
    """Bulk row copies with the float4 table (dx != dy), replayed from a CUDA
    graph after a reset."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=300, nsteps=360)
    sc.dy = 1.25 * sc.dx
    sc.dt = 0.99 / (299792458.0 * np.sqrt(1.0 / sc.dx ** 2 + 1.0 / sc.dy ** 2))
    o = oracle_run(sc, sc.nsteps)
    sim = fdtd.from_scene(sc, probes=False, monitors=False)
    for k, v in {"kernel": 0, "tblock": 4, "segment": 32, "warps": 4, "bulk": 1, "graph": 1}.items():
        sim.set_option(k, v)
    assert sim.get_option("bulk") == 1
    sim.step(sc.nsteps)
    sim.reset()
    sim.step(sc.nsteps)
    sim.sync()
    g = {f: sim.get_field(f, (sc.ny, sc.nx)) for f in ("ez", "hx", "hy")}
    sim.close()
    assert_fields_close(g, o)


def test_rectangular_cells():
    """dx != dy: the interior kernel keeps the full (Ca, Cb/dx, Cb/dy) table
    (square cells stage (Ca, Cb/dx) only); both against the oracle."""
    sc = scenes.ellipse_scene(side=320, nsteps=500)
    sq = gpu_run(sc, sc.nsteps, tblock=4, segment=32, warps=4)
    assert_fields_close(sq, oracle_run(sc, sc.nsteps))
    sc.dy = 1.25 * sc.dx
    sc.dt = 0.99 / (299792458.0 * np.sqrt(1.0 / sc.dx ** 2 + 1.0 / sc.dy ** 2))
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    g = gpu_run(sc, sc.nsteps, tblock=4, segment=32, warps=4)
    assert_fields_close(g, o)
    assert rel_l2(g["probes"], o["probes"]) <= TOL_FIELD


def test_unfused_and_fused_agree_to_rounding():
    sc = scenes.ellipse_scene(side=200, nsteps=500)
    a = gpu_run(sc, sc.nsteps, kernel=1)
    b = gpu_run(sc, sc.nsteps, kernel=0, tblock=4)
    for c in ("ez", "hx", "hy"):
        assert rel_l2(b[c], a[c]) < 1e-5


def test_dft_monitor_parity():
    sc = scenes.adjoint_scenes(side=160, n_designs=1, nsteps=900, npml=12, design=32)[0]
    o = oracle_run(sc, sc.nsteps, monitors=sc.monitors, freqs=sc.freqs)
    g = gpu_run(sc, sc.nsteps, tblock=4, segment=32)
    assert_fields_close(g, o)
    rel = np.abs(g["dft"] - o["dft"]) / np.max(np.abs(o["dft"]))
    assert np.max(rel) <= 1e-4, rel


def test_full_size_4096_light_cone():
    """The 4096^2 heterogeneous CPML workload in the benchmark's launch
    configuration, 600 steps: every field value equals the oracle run on the
    crop that holds the source's dependency cone, and is exactly zero outside."""
    sc = scenes.ellipse_scene()
    n = 600
    g = gpu_run(sc, n, tblock=4, segment=128, warps=2, probes=False)
    si, sj = sc.source.i, sc.source.j
    h = n + 2
    i0, j0 = si - h, sj - h
    crop = scenes.Scene2D(nx=2 * h + 1, ny=2 * h + 1, dx=sc.dx, dy=sc.dy, dt=sc.dt, npml=0,
                          mat=np.ascontiguousarray(sc.mat[j0:j0 + 2 * h + 1, i0:i0 + 2 * h + 1]),
                          eps_r=sc.eps_r, sigma=sc.sigma, nsteps=n,
                          source=scenes.Source(h, h, kind=sc.source.kind, params=sc.source.params))
    o = oracle_run(crop, n)
    for c in ("ez", "hx", "hy"):
        sub = g[c][j0:j0 + 2 * h + 1, i0:i0 + 2 * h + 1]
        assert rel_l2(sub, o[c]) <= TOL_FIELD, c
        outside = g[c].copy()
        outside[j0:j0 + 2 * h + 1, i0:i0 + 2 * h + 1] = 0
        assert np.count_nonzero(outside) == 0, c


def test_batch_of_uneven_scenes():
    from paper_2405_00814_gb300 import fdtd
    scs = scenes.batch_scenes(n_scenes=3, nsteps=400, side_lo=96, side_hi=300)
    sim = fdtd.Simulation.batch(scs)
    for k, s in enumerate(scs):
        sim.select(k)
        sim.set_scene_source(s.source)
    sim.step(400)
    for k, s in enumerate(scs):
        o = oracle_run(s, 400)
        sim.select(k)
        g = {c: sim.get_field(c, (s.ny, s.nx)) for c in ("ez", "hx", "hy")}
        assert_fields_close(g, o)
    sim.close()


def test_state_roundtrip_and_reset():
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=160, nsteps=300)
    sim = fdtd.from_scene(sc)
    sim.step(150)
    st = sim.save_state()
    sim.step(150)
    a = sim.get_field("ez", (sc.ny, sc.nx))
    pa = sim.read_probe(sim.probe_ids[0], 300)
    sim.load_state(st)
    assert sim.time_step == 150
    sim.step(150)
    b = sim.get_field("ez", (sc.ny, sc.nx))
    assert np.array_equal(a, b)
    assert np.array_equal(pa, sim.read_probe(sim.probe_ids[0], 300))
    sim.reset()
    assert sim.time_step == 0
    assert not np.any(sim.get_field("ez", (sc.ny, sc.nx)))
    sim.close()


def test_determinism_bitwise():
    sc = scenes.ellipse_scene(side=300, nsteps=240)
    a = gpu_run(sc, 240)
    b = gpu_run(sc, 240)
    for c in ("ez", "hx", "hy"):
        assert np.array_equal(a[c], b[c])


def test_set_field_mode_evolution():
    """A discrete cavity mode loaded through set_field evolves as cos(w_d n dt)."""
    import math
    from paper_2405_00814_gb300 import fdtd
    n = 96
    sc = scenes.cavity_ricker(n=n)
    sc.source = None
    c0 = 299792458.0
    mu0 = 4e-7 * math.pi
    i = np.arange(n)[None, :]
    j = np.arange(n)[:, None]
    phi = np.sin(3 * math.pi * i / n) * np.sin(2 * math.pi * j / n)
    pad = np.zeros((n + 1, n + 1))
    pad[:n, :n] = phi
    hy = -(sc.dt / (2 * mu0)) * (pad[:n, 1:] - pad[:n, :n]) / sc.dx
    hx = (sc.dt / (2 * mu0)) * (pad[1:, :n] - pad[:n, :n]) / sc.dy
    sim = fdtd.Simulation(sc)
    sim.set_field("ez", phi)
    sim.set_field("hx", hx)
    sim.set_field("hy", hy)
    sim.step(400)
    s2 = (c0 * sc.dt) ** 2 * (math.sin(3 * math.pi / (2 * n)) ** 2 / sc.dx ** 2 + math.sin(2 * math.pi / (2 * n)) ** 2 / sc.dy ** 2)
    w = 2 * math.asin(math.sqrt(s2)) / sc.dt
    ez = sim.get_field("ez", (n, n))
    assert rel_l2(ez, math.cos(w * 400 * sc.dt) * phi) < 1e-4
    sim.close()


def test_invalid_inputs_rejected():
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.cavity_ricker(n=32)
    with pytest.raises(fdtd.FDTDError) as ei:
        bad = scenes.cavity_ricker(n=32)
        bad.dt *= 1.02
        fdtd.Simulation(bad)
    assert ei.value.code == fdtd.EUNSTABLE
    sim = fdtd.Simulation(sc)
    with pytest.raises(fdtd.FDTDError):
        sim.set_source("ricker", 0, 5, param=1e10)          # on the PEC wall
    with pytest.raises(fdtd.FDTDError):
        sim.add_probe(40, 3)
    with pytest.raises(fdtd.FDTDError):
        sim.set_option("tblock", 9)
    for bad_taper in (-1, 61):
        with pytest.raises(fdtd.FDTDError):
            sim.set_option("taper", bad_taper)
    for bad_wb in (0, 9):
        with pytest.raises(fdtd.FDTDError):
            sim.set_option("warps_b", bad_wb)
    with pytest.raises(fdtd.FDTDError):
        sim.set_option("bulk", 2)
    sim.step(3)
    with pytest.raises(fdtd.FDTDError):
        sim.add_probe(3, 3)                                   # after stepping
    sim.close()
    bad = scenes.cavity_ricker(n=32)
    bad.mat = bad.mat.copy()
    bad.mat[5, 5] = 7                                         # index >= n_mat
    with pytest.raises(fdtd.FDTDError):
        fdtd.Simulation(bad)
