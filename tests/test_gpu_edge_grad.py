"""GPU edge-weight gradients (fdtd_edge_grad: dL/dw of the 11 weights every
design cell owns, Sec. IV-A's layers taken as learnable) against the FP64
oracle's reverse mode over the literal graph, their chain to the eps_r
gradient, and the inputs the mode refuses."""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3
C0 = 299792458.0
EPS0 = 1.0 / (4e-7 * math.pi * C0 ** 2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _grad_err(g, ref):
    den = np.maximum(np.abs(ref), 1e-2 * np.max(np.abs(ref)))
    return float(np.max(np.abs(g - ref) / den))


def _gpu(sc, ckpt, dLdF, *, tblock=4, segment=16, mode=2, sig_d=None, kernel=0):
    from paper_2405_00814_gb300 import fdtd
    i0, j0, w, h = sc.design
    sim = fdtd.Simulation.batch([sc])
    sim.select(0)
    sim.set_scene_source(sc.source)
    sim.set_design(i0, j0, sc.design_eps, sig_d)
    mid = sim.add_dft_monitor(sc.monitors, sc.freqs)
    sim.set_option("kernel", kernel)
    sim.set_option("tblock", tblock)
    sim.set_option("segment", segment)
    sim.set_option("adj_store", mode)
    sim.set_checkpointing(ckpt)
    sim.step(sc.nsteps)
    F = sim.read_dft(mid)
    g = sim.edge_grad([dLdF], [(h, w)])[0] if mode == 2 else sim.adjoint_grad([dLdF], (1, h, w))[0]
    sim.close()
    return F, g


@pytest.mark.parametrize("side,npml,design,at,nsteps,ckpt,tblock,segment,kernel", [
    (96, 8, 24, None, 600, 64, 4, 16, 0),          # centred design, last segment partial
    (150, 10, 37, (96, 30), 500, 100, 3, 24, 0),   # two strips: the design crosses the strip boundary at x = 120
    (96, 8, 24, None, 300, 50, 2, 8, 0),           # short tasks: the window spans several task rows
    (96, 8, 24, None, 300, 64, 1, 64, 1),          # unfused forward (window copied after each step)
    (120, 8, 30, (20, 50), 300, 64, 4, 32, 2),     # persistent forward; the design's tasks reach the CPML
])
def test_edge_grad_matches_oracle(side, npml, design, at, nsteps, ckpt, tblock, segment, kernel):
    import oracle
    sc = scenes.adjoint_scenes(side=side, n_designs=1, nsteps=nsteps, npml=npml, design=design, n_monitors=3)[0]
    if at is not None:
        sc.design = (at[0], at[1], design, design)
    rng = np.random.default_rng(side)
    dLdF = (rng.standard_normal((len(sc.monitors), len(sc.freqs))) +
            1j * rng.standard_normal((len(sc.monitors), len(sc.freqs)))) * 1e9
    F, g = _gpu(sc, ckpt, dLdF, tblock=tblock, segment=segment, kernel=kernel)
    osim = oracle.TMz(sc, nsteps_src=sc.nsteps)
    g1, g2, Fo = osim.graph_edge_grad(sc.nsteps, sc.monitors, sc.freqs, dLdF.real, dLdF.imag)
    ref = osim.edge_class_grad(g1, g2, sc.design)
    assert np.max(np.abs(F - Fo)) <= 1e-4 * np.max(np.abs(Fo))
    for k in range(11):
        assert _grad_err(g[k], ref[k]) <= TOL_GRAD, (k, _grad_err(g[k], ref[k]))


def test_edge_grad_chains_to_the_eps_gradient():
    """The 5 electric classes chained through eq. (7) give fdtd_adjoint_grad's
    dL/deps_r (history mode), on a lossy design."""
    sc = scenes.adjoint_scenes(side=96, n_designs=1, nsteps=500, npml=8, design=24, n_monitors=3)[0]
    i0, j0, w, h = sc.design
    sig_d = 0.05 * np.random.default_rng(5).random((h, w))
    F, _ = _gpu(sc, 50, np.zeros((3, 1)), mode=1, sig_d=sig_d)
    _, geps = _gpu(sc, 50, 2.0 * F, mode=1, sig_d=sig_d)
    F2, gc = _gpu(sc, 50, 2.0 * F, mode=2, sig_d=sig_d)
    assert np.max(np.abs(F2 - F)) <= 1e-5 * np.max(np.abs(F))
    e = sc.design_eps * EPS0
    D = e + sig_d * sc.dt / 2
    dca = EPS0 * sig_d * sc.dt / D ** 2
    dcb = -EPS0 * sc.dt / D ** 2
    chain = gc[0] * dca + (gc[1] - gc[2]) * dcb / sc.dx + (gc[4] - gc[3]) * dcb / sc.dy
    assert _grad_err(chain, geps) <= TOL_GRAD, _grad_err(chain, geps)


def _recorded(sc, mode, design=None, steps=40):
    from paper_2405_00814_gb300 import fdtd
    sim = fdtd.Simulation.batch([sc])
    sim.select(0)
    sim.set_scene_source(sc.source)
    i0, j0, w, h = sc.design if design is None else design
    sim.set_design(i0, j0, sc.design_eps if design is None else np.full((h, w), 2.0))
    sim.add_dft_monitor(sc.monitors, sc.freqs)
    sim.set_option("adj_store", mode)
    sim.set_checkpointing(20)
    if steps:
        sim.step(steps)
    return sim


def test_edge_grad_refusals():
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.adjoint_scenes(side=96, n_designs=1, nsteps=40, npml=8, design=24, n_monitors=3)[0]
    i0, j0, w, h = sc.design
    dLdF = np.ones((3, 1), np.complex64)
    sim = _recorded(sc, 1)                       # history mode: no edge gradients
    with pytest.raises(fdtd.FDTDError):
        sim.edge_grad([dLdF], [(h, w)])
    sim.close()
    sim = _recorded(sc, 2)                       # edge mode: no eps gradient
    with pytest.raises(fdtd.FDTDError):
        sim.adjoint_grad([dLdF], (1, h, w))
    sim.close()
    sim = _recorded(sc, 2, design=(8, 30, 10, 10), steps=0)   # the ring reaches the CPML
    with pytest.raises(fdtd.FDTDError):
        sim.step(5)
    sim.close()
    for mode in (1, 2):                          # the recorded rectangle cannot change size
        sim = _recorded(sc, mode, steps=10)
        with pytest.raises(fdtd.FDTDError):
            sim.set_design(i0, j0, np.full((h, w + 1), 2.0))
        sim.set_design(i0 + 1, j0, np.full((h, w), 2.0))
        sim.close()


def test_edge_grad_two_scenes_and_device_output():
    """A batch of two designs: each scene's [11, h, w] block equals the one its
    own single-scene context gives, on host and in a CUDA tensor."""
    import torch
    from paper_2405_00814_gb300 import fdtd
    scs = scenes.adjoint_scenes(side=96, n_designs=2, nsteps=300, npml=8, design=24, n_monitors=3)
    rng = np.random.default_rng(21)
    dLdF = [(rng.standard_normal((3, 1)) + 1j * rng.standard_normal((3, 1))) * 1e9 for _ in scs]
    singles = [_gpu(sc, 60, d)[1] for sc, d in zip(scs, dLdF)]
    sim = fdtd.Simulation.batch(scs)
    for k, sc in enumerate(scs):
        sim.select(k)
        sim.set_scene_source(sc.source)
        i0, j0, w, h = sc.design
        sim.set_design(i0, j0, sc.design_eps)
        sim.add_dft_monitor(sc.monitors, sc.freqs)
    sim.set_option("tblock", 4)
    sim.set_option("segment", 16)
    sim.set_option("adj_store", 2)
    sim.set_checkpointing(60)
    sim.step(scs[0].nsteps)
    shapes = [(sc.design[3], sc.design[2]) for sc in scs]
    g = sim.edge_grad(dLdF, shapes)
    for k in range(2):
        assert _grad_err(g[k], singles[k]) <= 1e-5, k
    sim.close()
    # the same run with the result written into a device tensor
    sim = fdtd.Simulation.batch(scs)
    for k, sc in enumerate(scs):
        sim.select(k)
        sim.set_scene_source(sc.source)
        i0, j0, w, h = sc.design
        sim.set_design(i0, j0, sc.design_eps)
        sim.add_dft_monitor(sc.monitors, sc.freqs)
    sim.set_option("tblock", 4)
    sim.set_option("segment", 16)
    sim.set_option("adj_store", 2)
    sim.set_checkpointing(60)
    sim.step(scs[0].nsteps)
    out = torch.empty(2 * 11 * 24 * 24, dtype=torch.float32, device="cuda")
    sim.edge_grad(dLdF, shapes, out=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(2, 11, 24, 24)
    assert np.array_equal(got, np.stack(g))
    sim.close()
