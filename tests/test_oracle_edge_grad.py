"""Pins of the edge-weight reverse mode of the FP64 oracle (the paper's layers
as learnable message passing, Sec. IV-A: dL/dw for every edge of both layers).

(i) The graph forward with the source and the running DFT reproduces the
stencil run (fields and F).  (ii) dL/dw equals central finite differences of
the forward loss for edges of every kind: the 11 interior classes, CPML
auxiliary edges, pass-through edges.  (iii) Chained through eq. (7)
(dCa/deps_r, dCb/deps_r), the 5 electric classes give the eps_r gradient of the
stencil adjoint, itself pinned by finite differences in eps_r.
"""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes

C0 = 299792458.0
EPS0 = 1.0 / (4e-7 * math.pi * C0 ** 2)


def _problem(oracle_mod, lossy=True, nsteps=120):
    nx, ny = 30, 26
    dx, dy = 1e-3, 1.1e-3
    dt = 0.99 / (C0 * math.sqrt(1 / dx ** 2 + 1 / dy ** 2))
    rng = np.random.default_rng(7)
    eps = 1 + 6 * rng.random((ny, nx))
    sig = (0.04 * rng.random((ny, nx))) if lossy else np.zeros((ny, nx))
    eps[:5, :] = eps[-5:, :] = 1.0
    eps[:, :5] = eps[:, -5:] = 1.0
    sig[:5, :] = sig[-5:, :] = 0.0
    sig[:, :5] = sig[:, -5:] = 0.0
    src = scenes.Source(8, 12, kind="gauss_mod", params=(40e9,), length=3)
    sim = oracle_mod.TMz(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, npml=4, eps_cell=eps, sigma_cell=sig,
                         source=src, nsteps_src=nsteps)
    mons = np.array([[20, 18], [22, 9], [14, 20]], np.int32)
    freqs = np.array([30e9, 45e9])
    return sim, mons, freqs, eps, sig, src


def test_graph_forward_is_the_stencil_run(oracle_mod):
    sim, mons, freqs, *_ = _problem(oracle_mod)
    h, F, _ = sim.graph_forward(120, monitors=mons, freqs=freqs)
    sim.run(120, dft_cells=mons, freqs=freqs)
    ref = sim.to_nodes()
    assert np.max(np.abs(h - ref)) <= 1e-12 * np.max(np.abs(ref))
    Fs = sim.dft[0] + 1j * sim.dft[1]
    assert np.max(np.abs(F - Fs)) <= 1e-12 * np.max(np.abs(Fs))


def _loss(sim, layers, mons, freqs, a, b, nsteps):
    _, F, _ = sim.graph_forward(nsteps, layers, mons, freqs)
    return float(np.sum(a * F.real + b * F.imag))


def test_edge_gradient_matches_central_fd(oracle_mod):
    nsteps = 120
    sim, mons, freqs, *_ = _problem(oracle_mod, nsteps=nsteps)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((len(mons), len(freqs))) * 1e9
    b = rng.standard_normal((len(mons), len(freqs))) * 1e9
    g1, g2, _ = sim.graph_edge_grad(nsteps, mons, freqs, a, b)
    W = {1: sim.graph_layer(1), 2: sim.graph_layer(2)}
    G = {1: g1, 2: g2}
    nn = sim.graph_nodes()
    base = 3 * sim.nx * sim.ny
    picks = []
    # interior classes at two cells, plus CPML auxiliary and pass-through rows
    for (i, j) in ((15, 13), (11, 17)):
        for layer, kd, ks, di, dj in sim.EDGE_CLASSES:
            picks.append((layer, sim.node_index(kd, i, j), sim.node_index(ks, i + di, j + dj)))
    for layer in (1, 2):
        r, c, _ = W[layer]
        for d in (base + 3, nn - 2, sim.node_index("t", 2, 20), sim.node_index("u", 27, 3)):
            for e in range(r[d], r[d + 1]):
                picks.append((layer, d, int(c[e])))
    gmax = max(np.max(np.abs(g1)), np.max(np.abs(g2)))
    checked = 0
    for layer, d, sidx in picks:
        r, c, w = W[layer]
        row = np.arange(r[d], r[d + 1])
        e = int(row[c[row] == sidx][0])
        hd = 1e-6 * max(abs(w[e]), 1.0)
        wp, wm = w.copy(), w.copy()
        wp[e] += hd
        wm[e] -= hd
        lp = _loss(sim, (W[1], (r, c, wp)) if layer == 2 else ((r, c, wp), W[2]), mons, freqs, a, b, nsteps)
        lm = _loss(sim, (W[1], (r, c, wm)) if layer == 2 else ((r, c, wm), W[2]), mons, freqs, a, b, nsteps)
        fd = (lp - lm) / (2 * hd)
        assert abs(G[layer][e] - fd) <= 1e-6 * max(abs(fd), 1e-3 * gmax), (layer, d, sidx, G[layer][e], fd)
        checked += 1
    assert checked >= 22 + 8


@pytest.mark.parametrize("lossy", [False, True])
def test_electric_classes_chain_to_the_eps_gradient(oracle_mod, lossy):
    """sum over the 5 electric classes of dL/dw * dw/deps_r, with D = eps0 eps_r +
    sigma dt/2, dCa/deps_r = eps0 sigma dt / D^2 and dCb/deps_r = -eps0 dt / D^2,
    equals the stencil adjoint's dL/deps_r for L = sum |F|^2 (dL/dF = 2 F)."""
    nsteps = 150
    sim, mons, freqs, eps, sig, src = _problem(oracle_mod, lossy, nsteps)
    design = (10, 8, 9, 7)
    loss, fre, fim, geps = sim.adjoint_grad(nsteps, 40, mons, freqs, design)
    sim2 = oracle_mod.TMz(nx=sim.nx, ny=sim.ny, dx=sim.dx, dy=sim.dy, dt=sim.dt, npml=4, eps_cell=eps,
                          sigma_cell=sig, source=src, nsteps_src=nsteps)
    g1, g2, F = sim2.graph_edge_grad(nsteps, mons, freqs, 2 * fre, 2 * fim)
    assert np.max(np.abs(F - (fre + 1j * fim))) <= 1e-12 * np.max(np.abs(F))
    gc = sim2.edge_class_grad(g1, g2, design)
    i0, j0, w, h = design
    e = eps[j0:j0 + h, i0:i0 + w] * EPS0
    s = sig[j0:j0 + h, i0:i0 + w]
    D = e + s * sim.dt / 2
    dca = EPS0 * s * sim.dt / D ** 2
    dcb = -EPS0 * sim.dt / D ** 2
    chain = gc[0] * dca + (gc[1] - gc[2]) * dcb / sim.dx + (-gc[3] + gc[4]) * dcb / sim.dy
    assert np.max(np.abs(chain - geps)) <= 1e-9 * np.max(np.abs(geps))
    # the magnetic classes do not depend on eps_r but are not zero
    assert np.max(np.abs(gc[5:])) > 0
