"""Pins of the FP64 reverse-mode (adjoint) oracle.

(i) dot-product identity <A x, y> = <x, A^T y> for one leapfrog step with CPML
and lossy media; (ii) the stencil-form adjoint equals the literal graph's
transposed layers applied in reverse order (Prop. 2 read backwards); (iii) the
checkpointed gradient dL/deps_r equals central finite differences of the
forward loss.
"""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes

C0 = 299792458.0
NAMES = ("ez", "hx", "hy", "pezx", "pezy", "phxy", "phyx")


def _masked_random(sim, seed):
    rng = np.random.default_rng(seed)
    st = {k: rng.standard_normal((sim.ny, sim.nx)) for k in NAMES}
    px, py = sim.px, sim.py
    st["pezx"] *= ((px["bE"] != 0) | (px["cE"] != 0))[None, :]
    st["pezy"] *= ((py["bE"] != 0) | (py["cE"] != 0))[:, None]
    st["phyx"] *= ((px["bH"] != 0) | (px["cH"] != 0))[None, :]
    st["phxy"] *= ((py["bH"] != 0) | (py["cH"] != 0))[:, None]
    for k in ("ez", "pezx", "pezy"):
        st[k][0, :] = 0
        st[k][:, 0] = 0
    return st


def _sim(oracle_mod, nx=23, ny=19, npml=4, seed=1):
    rng = np.random.default_rng(seed)
    dx, dy = 1e-3, 1.2e-3
    dt = 0.99 / (C0 * math.sqrt(1 / dx ** 2 + 1 / dy ** 2))
    return oracle_mod.TMz(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, npml=npml,
                          eps_cell=1 + 11 * rng.random((ny, nx)), sigma_cell=0.05 * rng.random((ny, nx)))


@pytest.mark.parametrize("npml", [0, 4])
def test_adjoint_dot_product(oracle_mod, npml):
    sim = _sim(oracle_mod, npml=npml)
    x = _masked_random(sim, 2)
    y = _masked_random(sim, 3)
    sim.set_state(**x)
    sim.run(1)
    ax = {k: sim.state[k].copy() for k in NAMES}
    aty = {k: y[k].copy() for k in NAMES}
    sim.adjoint_step(aty)
    lhs = sum(float(np.sum(ax[k] * y[k])) for k in NAMES)
    rhs = sum(float(np.sum(x[k] * aty[k])) for k in NAMES)
    scale = math.sqrt(sum(float(np.sum(ax[k] ** 2)) for k in NAMES) * sum(float(np.sum(y[k] ** 2)) for k in NAMES))
    assert abs(lhs - rhs) <= 1e-13 * scale


def test_adjoint_equals_graph_transpose(oracle_mod):
    sim = _sim(oracle_mod, nx=26, ny=21, npml=5, seed=4)
    y = _masked_random(sim, 5)
    sim.set_state(**y)
    hy = sim.to_nodes()
    W1, W2 = sim.graph_layer(1), sim.graph_layer(2)
    g = sim.csr_mtv(*W1, sim.csr_mtv(*W2, hy))
    a = {k: y[k].copy() for k in NAMES}
    sim.adjoint_step(a)
    sim.set_state(**a)
    ref = sim.to_nodes()
    assert np.max(np.abs(g - ref)) <= 1e-13 * np.max(np.abs(ref))


def _fd_problem(oracle_mod, lossy):
    nx = ny = 48
    dx = 1e-3
    dt = 0.99 * dx / (C0 * math.sqrt(2))
    design = (16, 14, 12, 12)
    eps_d = scenes.smoothed_noise_design(99, 12, 12, smooth=2.0)
    eps = np.ones((ny, nx))
    sig = np.zeros((ny, nx))
    eps[14:26, 16:28] = eps_d
    if lossy:
        sig[14:26, 16:28] = 0.03
    src = scenes.Source(9, 24, kind="ricker", params=(10e9,))
    mons = np.array([[38, 10], [40, 30]], np.int32)
    freqs = np.array([8e9, 11e9])
    return dict(nx=nx, ny=ny, dx=dx, dy=dx, dt=dt, npml=6, eps=eps, sig=sig, src=src, mons=mons,
                freqs=freqs, design=design)


def _loss(oracle_mod, pb, eps, nsteps):
    sim = oracle_mod.TMz(nx=pb["nx"], ny=pb["ny"], dx=pb["dx"], dy=pb["dy"], dt=pb["dt"], npml=pb["npml"],
                         eps_cell=eps, sigma_cell=pb["sig"], source=pb["src"], nsteps_src=nsteps)
    sim.run(nsteps, dft_cells=pb["mons"], freqs=pb["freqs"])
    re, im = sim.dft
    return float(np.sum(re ** 2 + im ** 2))


@pytest.mark.parametrize("lossy", [False, True])
def test_adjoint_gradient_matches_central_fd(oracle_mod, lossy):
    pb = _fd_problem(oracle_mod, lossy)
    nsteps = 260
    sim = oracle_mod.TMz(nx=pb["nx"], ny=pb["ny"], dx=pb["dx"], dy=pb["dy"], dt=pb["dt"], npml=pb["npml"],
                         eps_cell=pb["eps"], sigma_cell=pb["sig"], source=pb["src"], nsteps_src=nsteps)
    loss, fre, fim, grad = sim.adjoint_grad(nsteps, 37, pb["mons"], pb["freqs"], pb["design"])
    assert abs(loss - _loss(oracle_mod, pb, pb["eps"], nsteps)) <= 1e-12 * loss
    i0, j0, w, h = pb["design"]
    h_fd = 1e-4
    gmax = np.max(np.abs(grad))
    for (dj, di) in [(0, 0), (3, 7), (6, 5), (11, 11), (9, 2), (5, 10)]:
        ep = pb["eps"].copy()
        ep[j0 + dj, i0 + di] += h_fd
        em = pb["eps"].copy()
        em[j0 + dj, i0 + di] -= h_fd
        fd = (_loss(oracle_mod, pb, ep, nsteps) - _loss(oracle_mod, pb, em, nsteps)) / (2 * h_fd)
        assert abs(grad[dj, di] - fd) <= 1e-6 * max(abs(fd), 1e-2 * gmax), (dj, di, grad[dj, di], fd)
