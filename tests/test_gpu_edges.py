"""GPU edge cases against the FP64 oracle: the smallest grids, grids thinner
than a warp strip or a segment, widths just past a strip boundary, a strongly
lossy medium (Ca < 0 in eq. (7)), steps split across calls, zero steps, and 3D
grids of a few cells."""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import TOL_FIELD, assert_fields_close, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu
C0 = 299792458.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _scene(nx, ny, npml, seed, nsteps=200, sigma_lossy=0.05):
    """Three materials scattered cell by cell (vacuum inside the CPML), a Ricker
    source near the centre and two probes; dx = dy = 1 mm, 0.99 of Courant."""
    rng = np.random.default_rng(seed)
    mat = np.minimum((rng.random((ny, nx)) * 3).astype(np.uint8), 2)
    if npml:
        mat[:npml, :] = 0
        mat[-npml:, :] = 0
        mat[:, :npml] = 0
        mat[:, -npml:] = 0
    dx = 1e-3
    dt = 0.99 / (C0 * math.sqrt(2.0 / dx ** 2))
    si, sj = max(1, nx // 2), max(1, ny // 2)
    probes = np.array([[max(1, nx // 3), max(1, ny // 3)], [max(1, nx - 2), max(1, ny - 2)]], np.int32)
    return scenes.Scene2D(nx=nx, ny=ny, dx=dx, dy=dx, dt=dt, npml=npml, mat=mat,
                          eps_r=np.array([1.0, 4.0, 9.5]), sigma=np.array([0.0, 0.02, sigma_lossy]),
                          nsteps=nsteps, source=scenes.Source(si, sj, kind="ricker", params=(30e9,)),
                          probes=probes, name=f"edge{nx}x{ny}")


@pytest.mark.parametrize("nx,ny,npml,tblock,segment", [
    (4, 4, 0, 4, 8),        # smallest grid: one strip of mostly pad lanes, segment taller than the grid
    (5, 7, 0, 3, 8),
    (121, 9, 0, 4, 64),     # the second strip owns one column
    (300, 5, 0, 2, 16),     # thinner than T rows of warm-up
    (13, 250, 0, 4, 8),     # one strip, many segments
    (64, 48, 6, 4, 24),     # CPML on a small grid: every strip touches a slab
    (241, 120, 8, 1, 16),   # T = 1, widths one past two strips
])
def test_small_and_ragged_grids(nx, ny, npml, tblock, segment):
    sc = _scene(nx, ny, npml, seed=nx * 1000 + ny)
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    g = gpu_run(sc, sc.nsteps, tblock=tblock, segment=segment, warps=2)
    assert_fields_close(g, o)
    assert rel_l2(g["probes"], o["probes"]) <= TOL_FIELD


def test_strongly_lossy_medium_negative_ca():
    """sigma = 400 S/m in eps_r = 9.5: sigma dt / (2 eps) > 1, so Ca < 0 (eq. (7))."""
    sc = _scene(96, 80, 0, seed=7, nsteps=300, sigma_lossy=400.0)
    eps = 9.5 / (4e-7 * math.pi * C0 ** 2)
    assert 400.0 * sc.dt / (2 * eps) > 1.0
    o = oracle_run(sc, sc.nsteps, probes=sc.probes)
    g = gpu_run(sc, sc.nsteps, tblock=4, segment=16, warps=4)
    assert_fields_close(g, o)


def test_steps_split_across_calls_are_bitwise_equal():
    """A T-step block never depends on how the steps were split across calls:
    1 + 2 + 5 + 3 steps give the same bits as 11 at once."""
    from paper_2405_00814_gb300 import fdtd
    sc = _scene(200, 150, 10, seed=3, nsteps=11)
    out = []
    for parts in ((11,), (1, 2, 5, 3)):
        sim = fdtd.from_scene(sc)
        sim.set_option("tblock", 4)
        sim.set_option("segment", 16)
        for p in parts:
            sim.step(p)
        out.append({c: sim.get_field(c, (sc.ny, sc.nx)) for c in ("ez", "hx", "hy")})
        sim.close()
    for c in ("ez", "hx", "hy"):
        assert np.array_equal(out[0][c], out[1][c]), c


def test_zero_steps_is_a_no_op():
    from paper_2405_00814_gb300 import fdtd
    sc = _scene(40, 30, 0, seed=5)
    sim = fdtd.from_scene(sc)
    l0 = sim.launch_count
    sim.step(0)
    assert sim.launch_count == l0
    assert sim.time_step == 0
    assert not np.any(sim.get_field("ez", (sc.ny, sc.nx)))
    sim.close()


@pytest.mark.parametrize("kernel,tblock", [(0, 1), (1, 1), (0, 2)])
@pytest.mark.parametrize("n", [4, 9])
def test_3d_tiny_grids(kernel, tblock, n):
    """3D grids of a few cells (every tile mostly pad), random materials."""
    from paper_2405_00814_gb300 import fdtd
    import oracle
    rng = np.random.default_rng(100 + n)
    mat = np.minimum((rng.random((n, n, n)) * 3).astype(np.uint8), 2)
    d = 1e-3
    dt = 0.99 / (C0 * math.sqrt(3.0 / d ** 2))
    c = n // 2
    sc = scenes.Scene3D(nx=n, ny=n, nz=n, dx=d, dy=d, dz=d, dt=dt, npml=0, mat=mat,
                        eps_r=np.array([1.0, 3.0, 6.0]), sigma=np.array([0.0, 0.01, 0.1]), nsteps=60,
                        source=scenes.Source(c, c, c, component="ez", kind="ricker", params=(40e9,)))
    osim = oracle.Yee3D(sc, nsteps_src=sc.nsteps)
    osim.run(sc.nsteps)
    sim = fdtd.from_scene(sc)
    sim.set_option("kernel", kernel)
    sim.set_option("tblock", tblock)
    sim.set_option("segment", 3)
    sim.step(sc.nsteps)
    for comp in ("ex", "ey", "ez", "hx", "hy", "hz"):
        assert rel_l2(sim.get_field(comp, (n, n, n)), osim.state[comp]) <= TOL_FIELD, comp
    sim.close()
