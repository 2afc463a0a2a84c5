"""GPU parity of the 3D Yee path (C ABI -> sm_103a kernels) against the FP64
oracle and the closed-form discrete cavity mode."""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import TOL_FIELD, rel_l2

pytestmark = pytest.mark.gpu
C0 = 299792458.0
MU0 = 4e-7 * math.pi
COMPS = ("ex", "ey", "ez", "hx", "hy", "hz")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle3(sc, n, samples=None, plane=False):
    import oracle
    sim = oracle.Yee3D(sc, nsteps_src=max(n, sc.nsteps))
    out = sim.run(n, samples=samples, plane_k=sc.dft_plane_k if plane else -1, freqs=sc.freqs if plane else None)
    res = {c: sim.state[c] for c in COMPS}
    res["samples"] = out.get("samples")
    if plane:
        res["plane"] = sim.plane[0] + 1j * sim.plane[1]
    return res


@pytest.mark.parametrize("tblock", [1, 2])
def test_3d_cavity_mode_closed_form(tblock):
    from paper_2405_00814_gb300 import fdtd
    nx, ny, nz = 24, 20, 16
    d = (1e-3, 1.1e-3, 0.9e-3)
    dt = 0.95 / (C0 * math.sqrt(sum(1 / x ** 2 for x in d)))
    sc = scenes.Scene3D(nx=nx, ny=ny, nz=nz, dx=d[0], dy=d[1], dz=d[2], dt=dt, npml=0,
                        mat=np.zeros((nz, ny, nx), np.uint8), eps_r=np.array([1.0]), sigma=np.array([0.0]),
                        nsteps=200)
    m, n, p = 1, 2, 1
    kt = np.array([2 / d[0] * math.sin(m * math.pi / (2 * nx)), 2 / d[1] * math.sin(n * math.pi / (2 * ny)),
                   2 / d[2] * math.sin(p * math.pi / (2 * nz))])
    a = np.cross(kt, np.array([0.3, -0.7, 1.1]))
    kx, ky, kz = m * math.pi / (nx * d[0]), n * math.pi / (ny * d[1]), p * math.pi / (nz * d[2])
    i = np.arange(nx)[None, None, :].astype(float)
    j = np.arange(ny)[None, :, None].astype(float)
    k = np.arange(nz)[:, None, None].astype(float)
    ex = a[0] * np.cos(kx * (i + .5) * d[0]) * np.sin(ky * j * d[1]) * np.sin(kz * k * d[2])
    ey = a[1] * np.sin(kx * i * d[0]) * np.cos(ky * (j + .5) * d[1]) * np.sin(kz * k * d[2])
    ez = a[2] * np.sin(kx * i * d[0]) * np.sin(ky * j * d[1]) * np.cos(kz * (k + .5) * d[2])

    def fwd(v, axis):
        pad = np.concatenate([v, np.zeros_like(np.take(v, [0], axis=axis))], axis=axis)
        return np.diff(pad, axis=axis)
    f = dt / (2 * MU0)
    hx = f * (fwd(ez, 1) / d[1] - fwd(ey, 0) / d[2])
    hy = f * (fwd(ex, 0) / d[2] - fwd(ez, 2) / d[0])
    hz = f * (fwd(ey, 2) / d[0] - fwd(ex, 1) / d[1])
    sim = fdtd.Simulation(sc)
    sim.set_option("tblock", tblock)
    for name, v in (("ex", ex), ("ey", ey), ("ez", ez), ("hx", hx), ("hy", hy), ("hz", hz)):
        sim.set_field(name, v)
    sim.step(200)
    w = 2 * math.asin(math.sqrt((C0 * dt / 2) ** 2 * float(np.sum(kt ** 2)))) / dt
    cw = math.cos(w * 200 * dt)
    for name, ref in (("ex", ex), ("ey", ey), ("ez", ez)):
        got = sim.get_field(name, (nz, ny, nx))
        assert rel_l2(got, cw * ref) < 1e-4, name
    sim.close()


@pytest.mark.parametrize("kernel,segz,side,tblock,n", [
    (0, 64, 40, 1, 150), (0, 7, 40, 1, 150), (1, 64, 40, 1, 150), (0, 5, 37, 1, 150),
    # the two-step kernel: segments of 1 .. 64 planes, a ragged last tile row,
    # an odd step count (the last step runs the one-step kernel)
    (0, 64, 40, 2, 150), (0, 7, 40, 2, 150), (0, 1, 37, 2, 150), (0, 2, 37, 2, 150), (0, 5, 37, 2, 151)])
def test_3d_boxes_cpml_probes_plane_dft(kernel, segz, side, tblock, n):
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.box_scene(side=side, nsteps=n, npml=6, n_boxes=10)
    sc.source = scenes.Source(20, 20, 20, component="ez", kind="ricker", params=(40e9,))
    sc.dft_plane_k = 28
    sc.freqs = np.array([10e9, 20e9, 30e9])
    probes = [(12, 14, 22, "ez"), (25, 9, 30, "hx"), (30, 30, 10, "ey")]
    o = _oracle3(sc, n, samples=probes, plane=True)
    sim = fdtd.from_scene(sc)
    sim.set_option("kernel", kernel)
    sim.set_option("segment", segz)
    sim.set_option("tblock", tblock)
    pids = [sim.add_probe(i, j, k, c) for i, j, k, c in probes]
    mid = sim.add_dft_plane(sc.dft_plane_k, ("ex", "ey", "ez"), sc.freqs)
    sim.step(n)
    for c in COMPS:
        assert rel_l2(sim.get_field(c, (sc.nz, sc.ny, sc.nx)), o[c]) <= TOL_FIELD, c
    got = np.stack([sim.read_probe(p, n) for p in pids], 1)
    for q in range(len(probes)):
        assert rel_l2(got[:, q], o["samples"][:, q]) <= TOL_FIELD, probes[q]
    dft = sim.read_dft(mid)
    assert np.max(np.abs(dft - o["plane"])) <= 1e-4 * np.max(np.abs(o["plane"]))
    sim.close()


def _random_state3(nx, ny, nz, seed):
    """Random E and H over the whole grid; the tangential E on the PEC walls
    (Ex at j|k = 0, Ey at i|k = 0, Ez at i|j = 0) is zero."""
    rng = np.random.default_rng(seed)
    st = {c: rng.standard_normal((nz, ny, nx)) * (1.0 if c[0] == "e" else 2.6e-3) for c in COMPS}
    st["ex"][:, 0, :] = 0
    st["ex"][0, :, :] = 0
    st["ey"][:, :, 0] = 0
    st["ey"][0, :, :] = 0
    st["ez"][:, :, 0] = 0
    st["ez"][:, 0, :] = 0
    return st


@pytest.mark.parametrize("tblock,segz,n,npml,shape", [
    (2, 4, 41, 5, (250, 23, 19)), (2, 19, 40, 5, (250, 23, 19)), (2, 3, 23, 0, (250, 23, 19)),
    (1, 4, 41, 5, (250, 23, 19)),
    # tiles clear of the CPML (the build without it, on the second stream) beside tiles in its reach
    (2, 8, 30, 4, (370, 40, 40)),
    # automatic segments: thin segments at the z-slabs, the planes between clear of them
    (2, 0, 31, 4, (370, 40, 40))])
def test_3d_rectangular_three_x_tiles(tblock, segz, n, npml, shape):
    """A 250 x 23 x 19 grid (three 120-cell x-tiles of the two-step kernel, the
    last one 10 cells wide; or 370 x 40 x 40, where some tiles are clear of the
    CPML), a CPML (or PEC walls), a lossy and two dielectric materials, random
    initial E and H everywhere plus a source on a tile seam, probes of all six
    components on both sides of the seams and a plane DFT: fields, probe
    records and the DFT equal the oracle."""
    import oracle
    from paper_2405_00814_gb300 import fdtd
    nx, ny, nz = shape
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[3:15, 4:20, 100:140] = 1
    mat[6:12, 2:9, 200:247] = 2
    mat[8:17, 10:21, 30:70] = 3
    dx = 1e-3
    dt = 0.99 / (C0 * math.sqrt(3.0) / dx)
    sc = scenes.Scene3D(nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dx, dt=dt, npml=npml, mat=mat,
                        eps_r=np.array([1.0, 4.0, 2.5, 6.0]), sigma=np.array([0.0, 0.0, 0.02, 0.0]), nsteps=n,
                        source=scenes.Source(120, 11, 9, component="ey", kind="ricker", params=(60e9,)))
    freqs = np.array([20e9, 45e9])
    probes = [(119, 11, 9, "ez"), (120, 12, 9, "hx"), (239, 11, 8, "hy"), (240, 11, 10, "ex"),
              (118, 9, 11, "hz"), (120, 11, 9, "ey"), (0, 0, 0, "hz"), (249, 22, 18, "hx")]
    st = _random_state3(nx, ny, nz, 11)
    osim = oracle.Yee3D(sc, nsteps_src=n)
    osim.set_state(**st)
    out = osim.run(n, samples=probes, plane_k=9, freqs=freqs)
    plane = osim.plane[0] + 1j * osim.plane[1]
    sim = fdtd.from_scene(sc)
    sim.set_option("segment", segz)
    sim.set_option("tblock", tblock)
    for c in COMPS:
        sim.set_field(c, st[c].astype(np.float32))
    pids = [sim.add_probe(i, j, k, c) for i, j, k, c in probes]
    mid = sim.add_dft_plane(9, ("ex", "ey", "ez"), freqs)
    sim.step(n)
    for c in COMPS:
        assert rel_l2(sim.get_field(c, (nz, ny, nx)), osim.state[c]) <= TOL_FIELD, c
    got = np.stack([sim.read_probe(p, n) for p in pids], 1)
    for q in range(len(probes)):
        assert rel_l2(got[:, q], out["samples"][:, q]) <= TOL_FIELD, probes[q]
    dft = sim.read_dft(mid)
    assert np.max(np.abs(dft - plane)) <= 1e-4 * np.max(np.abs(plane))
    sim.close()


def test_3d_two_step_equals_one_step():
    """The two-step kernel and the one-step kernel give the same fields on the
    40^3 box scene (both FP32; only the rounding of the same sums differs).
    Hz, which the z-directed dipole leaves near zero, is measured against the
    norm of the whole H field."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.box_scene(side=40, nsteps=60, npml=6, n_boxes=10)
    out = []
    for tb in (1, 2):
        sim = fdtd.from_scene(sc)
        sim.set_option("tblock", tb)
        sim.step(60)
        out.append({c: sim.get_field(c, (sc.nz, sc.ny, sc.nx)) for c in COMPS})
        sim.close()
    norm = {k: math.sqrt(sum(float(np.sum(out[0][c].astype(np.float64) ** 2)) for c in COMPS if c[0] == k))
            for k in "eh"}
    for c in COMPS:
        floor = norm[c[0]] if float(np.linalg.norm(out[0][c])) < 1e-2 * norm[c[0]] else 0.0
        assert rel_l2(out[1][c], out[0][c], floor=floor) <= 1e-5, c


@pytest.mark.parametrize("kernel,tblock", [(0, 1), (1, 1), (0, 2)])
def test_3d_full_size_512_light_cone(kernel, tblock):
    """The 512^3 box workload (10-cell CPML, 64 boxes, Gaussian Ez dipole) as the
    benchmark runs it, 110 steps: every field equals the oracle on the crop that
    holds the dipole's dependency cone and is exactly zero outside it."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.box_scene()
    n = 110
    sim = fdtd.from_scene(sc)
    sim.set_option("kernel", kernel)
    sim.set_option("tblock", tblock)
    sim.step(n)
    si, sj, sk = sc.source.i, sc.source.j, sc.source.k
    h = n + 2
    sl = (slice(sk - h, sk + h + 1), slice(sj - h, sj + h + 1), slice(si - h, si + h + 1))
    crop = scenes.Scene3D(nx=2 * h + 1, ny=2 * h + 1, nz=2 * h + 1, dx=sc.dx, dy=sc.dy, dz=sc.dz, dt=sc.dt, npml=0,
                          mat=np.ascontiguousarray(sc.mat[sl]), eps_r=sc.eps_r, sigma=sc.sigma, nsteps=sc.nsteps,
                          source=scenes.Source(h, h, h, component="ez", kind=sc.source.kind, params=sc.source.params))
    o = _oracle3(crop, n)
    # a component the dipole's symmetry leaves (near) zero in the cone -- its
    # reference norm below 1e-3 of its vector field's -- is measured against the
    # vector field's norm; every other component against its own norm
    norm_e = math.sqrt(sum(float(np.sum(o[c] ** 2)) for c in ("ex", "ey", "ez")))
    norm_h = math.sqrt(sum(float(np.sum(o[c] ** 2)) for c in ("hx", "hy", "hz")))
    for c in COMPS:
        g = sim.get_field(c, (sc.nz, sc.ny, sc.nx))
        kind = norm_e if c[0] == "e" else norm_h
        floor = kind if float(np.linalg.norm(o[c])) < 1e-3 * kind else 0.0
        assert rel_l2(g[sl], o[c], floor=floor) <= TOL_FIELD, c
        g[sl] = 0
        assert np.count_nonzero(g) == 0, c
        del g
    sim.close()


def test_3d_options():
    """3D contexts default to the two-step kernel with automatic segments;
    FDTD_OPT_TBLOCK takes 1 or 2 there, FDTD_OPT_SEGMENT 0 (automatic) or >= 1."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.box_scene(side=24, nsteps=8, npml=4, n_boxes=3)
    sim = fdtd.from_scene(sc)
    assert sim.get_option("tblock") == 2
    assert sim.get_option("segment") == 0
    for bad in (0, 3, 4):
        with pytest.raises(fdtd.FDTDError) as ei:
            sim.set_option("tblock", bad)
        assert ei.value.code == fdtd.EINVAL
    with pytest.raises(fdtd.FDTDError):
        sim.set_option("segment", -1)
    sim.set_option("segment", 5)
    sim.step(3)                       # a pair, then a one-step launch
    sim.set_option("segment", 0)
    sim.set_option("tblock", 1)
    sim.step(2)
    sim.sync()
    assert sim.time_step == 5
    sim.close()


def test_3d_thick_cpml_falls_back_to_one_step():
    """A 62-cell CPML on a 128^3 grid puts every lane of a tile in the x-slab,
    more auxiliary slots than the two-step kernel's shared memory holds; the
    steps run the one-step kernel and still equal the oracle."""
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.box_scene(side=128, nsteps=20, npml=62, n_boxes=4)
    sc.source = scenes.Source(64, 64, 64, component="ez", kind="ricker", params=(60e9,))
    o = _oracle3(sc, 20)
    sim = fdtd.from_scene(sc)
    assert sim.get_option("tblock") == 2
    sim.step(20)
    for c in COMPS:
        assert rel_l2(sim.get_field(c, (sc.nz, sc.ny, sc.nx)), o[c]) <= TOL_FIELD, c
    sim.close()


@pytest.mark.parametrize("n_planes", [2, 5])
def test_3d_two_step_several_monitors(n_planes):
    """Plane monitors on both sides of a z-segment boundary (the two-step kernel
    copies each plane's E after the first step; more than four planes send every
    step through the one-step kernel) and a cell monitor whose first-step
    samples the kernel records: each plane DFT equals the oracle's, and the cell
    DFT equals the direct FP64 sum dt Σ_n E^n e^{-i 2π f (n+1) dt} over the
    oracle's samples, over an odd number of steps."""
    import oracle
    from paper_2405_00814_gb300 import fdtd
    n = 61
    sc = scenes.box_scene(side=40, nsteps=n, npml=6, n_boxes=10)
    sc.source = scenes.Source(20, 20, 20, component="ez", kind="ricker", params=(40e9,))
    freqs = np.array([15e9, 35e9])
    planes = [5, 23, 24, 28, 31][:n_planes]
    cells = np.array([(12, 14, 22), (25, 9, 30), (30, 30, 10)], np.int32)
    sim = fdtd.from_scene(sc)
    sim.set_option("segment", 24)
    mids = [sim.add_dft_plane(k, ("ex", "ey", "ez"), freqs) for k in planes]
    cmid = sim.add_dft_monitor(cells, freqs)
    sim.step(n)
    for k, mid in zip(planes, mids):
        osim = oracle.Yee3D(sc, nsteps_src=n)
        osim.run(n, plane_k=k, freqs=freqs)
        ref = osim.plane[0] + 1j * osim.plane[1]
        got = sim.read_dft(mid)
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref)), k
    osim = oracle.Yee3D(sc, nsteps_src=n)
    out = osim.run(n, samples=[(int(i), int(j), int(k), "ez") for i, j, k in cells])
    e = out["samples"]                                   # [n, cells]
    ph = np.exp(-2j * np.pi * np.outer(np.arange(1, n + 1) * sc.dt, freqs))   # [n, f]
    ref = sc.dt * np.einsum("nc,nf->cf", e, ph)
    got = sim.read_dft(cmid)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    sim.close()
