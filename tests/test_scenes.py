"""The seeded input recipes the benchmark and the parity tests use (the
paper's datasets are not available, Sec. V-A): each generator is
deterministic and produces the sizes, value ranges and structure stated for
it (vacuum absorbing layers, index ranges, source and monitor positions)."""
import math

import numpy as np

from paper_2405_00814_gb300 import scenes

C0 = 299792458.0


def _layer_is_vacuum(mat, npml):
    return (not mat[:npml].any() and not mat[-npml:].any() and not mat[:, :npml].any()
            and not mat[:, -npml:].any())


def test_benchmark_scene_recipe_and_determinism():
    a = scenes.ellipse_scene()
    b = scenes.ellipse_scene()
    assert np.array_equal(a.mat, b.mat) and np.array_equal(a.eps_r, b.eps_r)
    assert (a.nx, a.ny, a.npml, a.nsteps) == (4096, 4096, 16, 4000)
    assert a.mat.dtype == np.uint8 and a.mat.max() <= 200 and len(a.eps_r) == 201
    assert a.eps_r[0] == 1.0 and a.sigma[0] == 0.0
    assert np.all((a.eps_r[1:] >= 1.0) & (a.eps_r[1:] <= 12.0))
    assert np.all((a.sigma[1:] >= 0.0) & (a.sigma[1:] <= 0.05))
    assert _layer_is_vacuum(a.mat, a.npml)
    # dx: 20 points per the shortest wavelength at f_max = 2 f0 in eps_r = 12; dt at 0.99 of Courant
    f0 = a.source.params[0]
    assert f0 == 2.4e9 and a.source.kind == "gauss_mod" and (a.source.i, a.source.j) == (2048, 2048)
    assert math.isclose(a.dx, C0 / (2 * f0 * math.sqrt(12.0)) / 20, rel_tol=1e-12)
    assert math.isclose(a.dt, 0.99 * a.dx / (C0 * math.sqrt(2.0)), rel_tol=1e-12)
    # the ellipses fill a sizeable share of the interior
    assert 0.1 < np.count_nonzero(a.mat) / a.mat.size < 0.95


def test_batch_scenes_recipe():
    scs = scenes.batch_scenes()
    assert len(scs) == 64
    sides = np.array([s.nx for s in scs])
    assert np.all((sides >= 256) & (sides <= 2048)) and np.all([s.nx == s.ny for s in scs])
    assert len(set(sides.tolist())) > 32                      # log-uniform, mostly distinct
    for s in scs:
        assert s.npml == 12 and _layer_is_vacuum(s.mat, 12) and s.nsteps == 2000
        assert 12 <= s.source.i < s.nx - 12 and 12 <= s.source.j < s.ny - 12
    assert len({(s.source.i, s.source.j) for s in scs}) > 60   # own source positions


def test_adjoint_scenes_recipe():
    scs = scenes.adjoint_scenes()
    assert len(scs) == 8
    i0, j0, w, h = scs[0].design
    assert (w, h) == (256, 256) and (i0, j0) == (384, 384)
    for s in scs:
        assert s.design == scs[0].design and s.design_eps.shape == (256, 256)
        assert np.all((s.design_eps >= 1.0) & (s.design_eps <= 12.0))
        assert len(s.monitors) == 8 and len({tuple(m) for m in s.monitors}) == 8
        assert np.all((s.monitors >= 17) & (s.monitors <= 1024 - 18))
        assert list(s.freqs) == [5e9] and s.nsteps == 3000 and s.npml == 16
    assert not np.array_equal(scs[0].design_eps, scs[1].design_eps)   # 8 different designs


def test_box_scene_recipe():
    s = scenes.box_scene()
    assert (s.nx, s.ny, s.nz, s.npml) == (512, 512, 512, 10)
    assert len(s.eps_r) == 65 and np.all((s.eps_r[1:] >= 1.0) & (s.eps_r[1:] <= 9.0)) and not s.sigma.any()
    m = s.mat
    assert not (m[:10].any() or m[-10:].any() or m[:, :10].any() or m[:, -10:].any() or m[:, :, :10].any()
                or m[:, :, -10:].any())
    assert s.dft_plane_k == 384 and list(s.freqs) == [2.5e9, 5.0e9, 7.5e9]
    assert s.source.component == "ez" and (s.source.i, s.source.j, s.source.k) == (256, 256, 256)
    assert math.isclose(s.dx, C0 / (10e9 * 3.0) / 15, rel_tol=1e-12)


def test_photonic_crystal_geometry():
    s = scenes.phc_waveguide()
    assert (s.nx, s.ny) == (416, 173) and list(s.eps_r) == [1.0, 12.0]
    um = 1e-6
    jc = int(round(2.5 * um / s.dx))
    # guide cells on the axis away from the holes, air at the six hole centres
    assert s.mat[jc, int(round(2.0 * um / s.dx))] == 1       # left of the first hole (3.3 +- 0.36 um)
    for k in range(3):
        for sgn in (-1, 1):
            xh = 6.0 * um + sgn * (0.7 + k) * um
            assert s.mat[jc, int(round(xh / s.dx))] == 0
    # the guide is 1.2 um wide: the row 0.5 um off-axis is inside, 0.7 um outside
    i = int(round(2.0 * um / s.dx))
    assert s.mat[jc + int(0.5 * um / s.dx), i] == 1 and s.mat[jc + int(0.7 * um / s.dx) + 1, i] == 0
    assert s.source.length > 1 and s.source.kind == "gauss_mod" and s.source.params[0] == 75e12
    assert _layer_is_vacuum(s.mat, s.npml)
