"""Pins of the split-field PML oracle (Berenger; the paper's own absorbing
boundary, Sec. III-C, eqs. (10)-(13), and its 4-node graph, Sec. IV-B).

* Without a layer the split recurrence is the plain Yee recurrence: Ezx + Ezy
  evolves exactly as Ez (the split only separates the two halves of curl H).
* The 4-node literal graph applied as two sparse layers equals the stencil.
* A graded layer absorbs: a probe next to it matches a domain so large that no
  echo returns in the window, to within a bound about 15 dB above the level the
  grading reaches.  A wrong axis on a conductivity, a missing magnetic loss or a
  mismatched sigma* raises the echo far above the bound.
"""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes

C0 = 299792458.0


def _state_close(a, b, tol):
    for k in ("hx", "hy"):
        assert np.max(np.abs(a[k] - b[k])) <= tol * max(np.max(np.abs(b[k])), 1e-300), k


def test_split_without_layer_is_the_plain_recurrence(oracle_mod):
    sc = scenes.ellipse_scene(side=96, nsteps=300)
    sc.npml = 0
    plain = oracle_mod.TMz(sc, nsteps_src=sc.nsteps)
    plain.run(sc.nsteps)
    split = oracle_mod.TMzSplit(sc)
    split.run(sc.nsteps)
    ez = split.ez()
    assert np.max(np.abs(ez - plain.state["ez"])) <= 1e-12 * np.max(np.abs(plain.state["ez"]))
    _state_close(split.state, plain.state, 1e-12)


@pytest.mark.parametrize("nx,ny,npml", [(7, 5, 2), (12, 9, 3), (16, 16, 4)])
def test_split_graph_equals_stencil(oracle_mod, nx, ny, npml):
    rng = np.random.default_rng(nx * 100 + ny)
    dx = 1e-3
    dt = 0.9 * dx / (C0 * math.sqrt(2))
    sc = scenes.Scene2D(nx=nx, ny=ny, dx=dx, dy=dx, dt=dt, npml=npml, mat=np.zeros((ny, nx), np.uint8),
                        eps_r=np.array([1.0]), sigma=np.array([0.0]), nsteps=1)
    eps = 1.0 + 5.0 * rng.random((ny, nx))
    sig = 0.1 * rng.random((ny, nx))
    sim = oracle_mod.TMzSplit(sc, eps_cell=eps, sigma_cell=sig)
    sim.set_state(**{k: rng.standard_normal((ny, nx)) for k in ("ezx", "ezy", "hx", "hy")})
    h0 = sim.to_nodes()
    r1, c1, w1 = sim.graph_layer(1)
    r2, c2, w2 = sim.graph_layer(2)
    assert len(h0) == 4 * nx * ny
    # the numbering is a bijection onto [0, 4 nx ny)
    idx = sorted(sim.node_index(k, i, j) for k in ("u", "q", "tx", "tz") for j in range(ny) for i in range(nx))
    assert idx == list(range(4 * nx * ny))
    h1 = oracle_mod.TMz.csr_mv(r1, c1, w1, h0)
    sim.layer_h()
    ref1 = sim.to_nodes()
    assert np.max(np.abs(h1 - ref1)) <= 1e-13 * np.max(np.abs(ref1))
    h2 = oracle_mod.TMz.csr_mv(r2, c2, w2, h1)
    sim.layer_e()
    ref2 = sim.to_nodes()
    assert np.max(np.abs(h2 - ref2)) <= 1e-13 * np.max(np.abs(ref2))


@pytest.mark.parametrize("npml,bound_db", [(8, -78.0), (16, -95.0)])
def test_split_pml_reflection_bound(oracle_mod, npml, bound_db):
    f0 = 2.4e9
    dx = scenes._dx_for(2 * f0, 1.0, 20)
    dt = 0.99 * dx / (C0 * math.sqrt(2))
    nsteps = 900

    def scene(n, npml_, off):
        s = scenes.Source(off + 30, off + 60, kind="gauss_mod", params=(f0,))
        return scenes.Scene2D(nx=n, ny=n, dx=dx, dy=dx, dt=dt, npml=npml_, mat=np.zeros((n, n), np.uint8),
                              eps_r=np.array([1.0]), sigma=np.array([0.0]), nsteps=nsteps, source=s)

    small = oracle_mod.TMzSplit(scene(120, npml, 0)).run(nsteps, samples=[(24, 60, "ez")])["samples"][:, 0]
    big = oracle_mod.TMz(scene(120 + 1800, 0, 900), nsteps_src=nsteps).run(
        nsteps, samples=[(924, 960, "ez")])["samples"][:, 0]
    refl = np.max(np.abs(small - big)) / np.max(np.abs(big))
    assert 20 * math.log10(refl) < bound_db


def test_split_profile_grading(oracle_mod):
    """sigma(rho) = sigma_max (rho/d)^3 with sigma_max = 0.8 (m+1)/(eta0 delta):
    zero inside, the E node on the wall at depth d, H nodes half a cell in."""
    n, npml, d = 40, 8, 1e-3
    sE, sH = oracle_mod.split_axis(n, npml, d, 3.0)
    eta0 = math.sqrt(4e-7 * math.pi / (1.0 / (4e-7 * math.pi * C0 ** 2)))
    smax = 0.8 * 4 / (eta0 * d)
    assert np.all(sE[npml:n - npml + 1] == 0.0)
    assert math.isclose(sE[0], smax, rel_tol=1e-14)
    assert math.isclose(sE[3], smax * (5 / 8) ** 3, rel_tol=1e-14)
    assert math.isclose(sH[0], smax * (7.5 / 8) ** 3, rel_tol=1e-14)
    assert math.isclose(sH[n - 1], smax * (7.5 / 8) ** 3, rel_tol=1e-14)


def test_split_line_source_is_the_sum_of_point_sources(oracle_mod):
    """Linearity of the split recurrence: a line source over cells (i, j0 .. j1-1)
    gives the sum of the point-source runs, also where the line enters the layer."""
    sc = scenes.ellipse_scene(side=72, nsteps=140, npml=8)
    i, j0, j1 = 5, 30, 36          # i = 5 lies inside the 8-cell layer
    sc.source = scenes.Source(i, j0, kind="gauss_mod", params=(20e9,), length=j1 - j0)
    line = oracle_mod.TMzSplit(sc)
    line.run(sc.nsteps)
    total = {k: np.zeros((sc.ny, sc.nx)) for k in ("ezx", "ezy", "hx", "hy")}
    for j in range(j0, j1):
        sc.source = scenes.Source(i, j, kind="gauss_mod", params=(20e9,))
        pt = oracle_mod.TMzSplit(sc)
        pt.run(sc.nsteps)
        for k in total:
            total[k] += pt.state[k]
    for k in total:
        assert np.max(np.abs(line.state[k] - total[k])) <= 1e-12 * max(np.max(np.abs(total[k])), 1e-300), k
