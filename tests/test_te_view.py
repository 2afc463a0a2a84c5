"""The paper's TE naming (Sec. III-B, Prop. 1) as a view of the library's TMz
graph: with S = diag(te_node_signs), S W S applied to S h reproduces the step,
and its interior edge weights carry the signs and magnitudes of the TE update
equations (7)-(9) written out directly (no GPU: the graph is the oracle's)."""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from paper_2405_00814_gb300.fdtd import te_node_signs

C0 = 299792458.0
MU0 = 4e-7 * math.pi
EPS0 = 1.0 / (MU0 * C0 ** 2)


def _flip(r, c, w, sg):
    dst = np.repeat(np.arange(len(r) - 1), np.diff(r))
    return w * sg[c] * sg[dst]


@pytest.mark.parametrize("split", [False, True])
def test_te_graph_reproduces_the_step(oracle_mod, split):
    sc = scenes.ellipse_scene(side=40, nsteps=1, npml=6)
    sim = oracle_mod.TMzSplit(sc) if split else oracle_mod.TMz(sc, nsteps_src=1)
    rng = np.random.default_rng(11)
    names = ("ezx", "ezy", "hx", "hy") if split else ("ez", "hx", "hy")
    sim.set_state(**{k: rng.standard_normal((sc.ny, sc.nx)) for k in names})
    h0 = sim.to_nodes()
    n = len(h0)
    sg = te_node_signs(sc.nx, sc.ny, n, split).astype(np.float64)
    r1, c1, w1 = sim.graph_layer(1)
    r2, c2, w2 = sim.graph_layer(2)
    te1 = oracle_mod.TMz.csr_mv(r1, c1, _flip(r1, c1, w1, sg), sg * h0)
    te2 = oracle_mod.TMz.csr_mv(r2, c2, _flip(r2, c2, w2, sg), te1)
    sim.layer_h()
    sim.layer_e()
    ref = sg * sim.to_nodes()
    assert np.max(np.abs(te2 - ref)) <= 1e-13 * np.max(np.abs(ref))
    # the electric nodes hold Ey = -Ez, the magnetic ones Hx and Hz = Hy
    kinds = ("tx", "tz") if split else ("t",)
    for kind in kinds + ("u", "q"):
        i, j = 17, 23
        v = sg[sim.node_index(kind, i, j)]
        assert v == (-1.0 if kind.startswith("t") else 1.0)


def test_te_interior_weights_are_the_te_equations(oracle_mod):
    """At a lossy dielectric interior cell: the Hx node gets +Db from the Ey node
    one k up and -Db from its own, the Hz node -Db from the Ey node one i up
    (eqs. (8), (9)); the Ey node gets A-/A+ from itself, +Cb/dz from the Hx
    node above, -Cb/dx from the Hz node to the right (eq. (7))."""
    nx = ny = 12
    dx, dz = 1e-3, 1.3e-3
    dt = 0.9 / (C0 * math.sqrt(1 / dx ** 2 + 1 / dz ** 2))
    mat = np.zeros((ny, nx), np.uint8)
    mat[5, 6] = 1
    eps_r, sigma = 4.5, 0.3
    sc = scenes.Scene2D(nx=nx, ny=ny, dx=dx, dy=dz, dt=dt, npml=0, mat=mat,
                        eps_r=np.array([1.0, eps_r]), sigma=np.array([0.0, sigma]), nsteps=1)
    sim = oracle_mod.TMz(sc, nsteps_src=1)
    n = sim.graph_nodes()
    sg = te_node_signs(nx, ny, n).astype(np.float64)
    W = {}
    for layer in (1, 2):
        r, c, w = sim.graph_layer(layer)
        dst = np.repeat(np.arange(n), np.diff(r))
        for d, s_, v in zip(dst, c, _flip(r, c, w, sg)):
            W[(layer, int(d), int(s_))] = v
    i, k = 6, 5
    t = sim.node_index
    db_z, db_x = dt / (MU0 * dz), dt / (MU0 * dx)
    eps = eps_r * EPS0
    ap, am = 1 + sigma * dt / (2 * eps), 1 - sigma * dt / (2 * eps)
    cb = dt / (ap * eps)
    close = lambda a, b: math.isclose(a, b, rel_tol=1e-13)
    # layer 1: Hx(i, k) and Hz(i, k) from the Ey nodes (forward differences in the library's staggering)
    assert close(W[(1, t("u", i, k), t("t", i, k + 1))], db_z)
    assert close(W[(1, t("u", i, k), t("t", i, k))], -db_z)
    assert close(W[(1, t("q", i, k), t("t", i + 1, k))], -db_x)
    assert close(W[(1, t("q", i, k), t("t", i, k))], db_x)
    # layer 2: Ey(i, k) from itself and the four H nodes around it
    assert close(W[(2, t("t", i, k), t("t", i, k))], am / ap)
    assert close(W[(2, t("t", i, k), t("u", i, k))], cb / dz)
    assert close(W[(2, t("t", i, k), t("u", i, k - 1))], -cb / dz)
    assert close(W[(2, t("t", i, k), t("q", i, k))], -cb / dx)
    assert close(W[(2, t("t", i, k), t("q", i - 1, k))], cb / dx)
