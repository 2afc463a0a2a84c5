"""GPU reverse mode (design history kept from the forward pass, or checkpointed
recompute, + fused adjoint kernels) against the FP64 oracle's adjoint and central
finite differences of the FP64 oracle."""
import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _grad_err(g, ref):
    """per cell |g - ref| / max(|ref|, 1e-2 max|ref|)"""
    den = np.maximum(np.abs(ref), 1e-2 * np.max(np.abs(ref)))
    return float(np.max(np.abs(g - ref) / den))


def _oracle_grad(sc, ckpt):
    import oracle
    sim = oracle.TMz(sc, nsteps_src=sc.nsteps)
    return sim.adjoint_grad(sc.nsteps, ckpt, sc.monitors, sc.freqs, sc.design)


def _oracle_loss(sc, eps_design):
    import oracle
    s2 = scenes.Scene2D(**{**sc.__dict__, "design_eps": eps_design})
    sim = oracle.TMz(s2, nsteps_src=sc.nsteps)
    sim.run(sc.nsteps, dft_cells=sc.monitors, freqs=sc.freqs)
    return float(np.sum(sim.dft[0] ** 2 + sim.dft[1] ** 2))


@pytest.mark.parametrize("store", [True, False])
@pytest.mark.parametrize("side,npml,design,nsteps,ckpt,tblock", [(128, 10, 32, 900, 100, 4), (96, 8, 24, 700, 37, 3)])
def test_adjoint_matches_oracle(side, npml, design, nsteps, ckpt, tblock, store):
    from paper_2405_00814_gb300 import autograd
    scs = scenes.adjoint_scenes(side=side, n_designs=2, nsteps=nsteps, npml=npml, design=design, n_monitors=4)
    batch = autograd.DesignBatch(scs, ckpt_every=ckpt, tblock=tblock, store=store)
    eps = np.stack([s.design_eps for s in scs])
    F = batch.forward(eps)
    g = batch.gradient(2.0 * F)
    for k, sc in enumerate(scs):
        loss, fre, fim, gref = _oracle_grad(sc, ckpt)
        Fref = fre + 1j * fim
        assert np.max(np.abs(F[k] - Fref)) <= 1e-4 * np.max(np.abs(Fref))
        assert _grad_err(g[k], gref) <= TOL_GRAD, _grad_err(g[k], gref)
    batch.close()


def test_adjoint_matches_central_fd():
    from paper_2405_00814_gb300 import autograd
    sc = scenes.adjoint_scenes(side=96, n_designs=1, nsteps=700, npml=8, design=24, n_monitors=4)[0]
    batch = autograd.DesignBatch([sc], ckpt_every=50)
    F = batch.forward(sc.design_eps[None])
    g = batch.gradient(2.0 * F)[0]
    cells = scenes.fd_cells(6, 24)
    h = 1e-4
    fd = []
    for dj, di in cells:
        ep = sc.design_eps.copy()
        ep[dj, di] += h
        em = sc.design_eps.copy()
        em[dj, di] -= h
        fd.append((_oracle_loss(sc, ep) - _oracle_loss(sc, em)) / (2 * h))
    fd = np.array(fd)
    got = np.array([g[dj, di] for dj, di in cells])
    gscale = np.max(np.abs(g))
    err = np.abs(got - fd) / np.maximum(np.abs(fd), 1e-2 * gscale)
    assert np.max(err) <= TOL_GRAD, (got, fd)
    batch.close()


@pytest.mark.parametrize("store", [True, False])
def test_adjoint_lossy_design_matches_oracle(store):
    """A design region with sigma > 0: dCa/deps_r no longer vanishes, and the
    gradient still follows from E^{n+1} - E^n."""
    from paper_2405_00814_gb300 import fdtd
    import oracle
    sc = scenes.adjoint_scenes(side=96, n_designs=1, nsteps=600, npml=8, design=24, n_monitors=3)[0]
    i0, j0, w, h = sc.design
    sig_d = 0.05 * np.random.default_rng(11).random((h, w))
    sim = fdtd.Simulation.batch([sc])
    sim.select(0)
    sim.set_scene_source(sc.source)
    sim.set_design(i0, j0, sc.design_eps, sig_d)
    mid = sim.add_dft_monitor(sc.monitors, sc.freqs)
    sim.set_option("adj_store", int(store))
    sim.set_checkpointing(60)
    sim.step(sc.nsteps)
    F = sim.read_dft(mid)
    g = sim.adjoint_grad([2.0 * F], (1, h, w))[0]
    sim.close()
    sig_cell = sc.sigma[sc.mat].astype(np.float64)
    sig_cell[j0:j0 + h, i0:i0 + w] = sig_d
    osim = oracle.TMz(sc, sigma_cell=sig_cell, nsteps_src=sc.nsteps)
    _, fre, fim, gref = osim.adjoint_grad(sc.nsteps, 60, sc.monitors, sc.freqs, sc.design)
    assert np.max(np.abs(F - (fre + 1j * fim))) <= 1e-4 * np.max(np.abs(fre + 1j * fim))
    assert _grad_err(g, gref) <= TOL_GRAD, _grad_err(g, gref)


def test_autograd_function_backward():
    import torch
    from paper_2405_00814_gb300 import autograd
    scs = scenes.adjoint_scenes(side=96, n_designs=2, nsteps=600, npml=8, design=24, n_monitors=3)
    batch = autograd.DesignBatch(scs, ckpt_every=100)
    Fn = autograd.dft_intensity_loss()
    eps = torch.tensor(np.stack([s.design_eps for s in scs]), device="cuda", requires_grad=True)
    loss = Fn.apply(eps, batch)
    loss.backward()
    ref = batch.gradient(2.0 * batch.forward(eps.detach().cpu().numpy()))
    assert eps.grad.shape == eps.shape
    assert rel_l2(eps.grad.cpu().numpy(), ref) < 1e-6
    batch.close()


@pytest.mark.slow
def test_adjoint_full_size_1024_design0():
    """The 1024^2 inverse-design workload as specified (8 designs, 3000 steps,
    checkpoints every 100): design 0's gradient against the FP64 oracle adjoint
    over the whole 256^2 region, and against FP64 central differences on 16
    seeded design cells."""
    from paper_2405_00814_gb300 import autograd
    scs = scenes.adjoint_scenes()
    batch = autograd.DesignBatch(scs, ckpt_every=100)
    eps = np.stack([s.design_eps for s in scs])
    F = batch.forward(eps)
    g = batch.gradient(2.0 * F)
    sc = scs[0]
    loss, fre, fim, gref = _oracle_grad(sc, 100)
    assert np.max(np.abs(F[0] - (fre + 1j * fim))) <= 1e-4 * np.max(np.abs(fre + 1j * fim))
    assert _grad_err(g[0], gref) <= TOL_GRAD
    cells = scenes.fd_cells(16, 256)
    h = 1e-4
    fd = np.array([(_oracle_loss(sc, sc.design_eps + h * _onehot(256, dj, di)) -
                    _oracle_loss(sc, sc.design_eps - h * _onehot(256, dj, di))) / (2 * h) for dj, di in cells])
    got = np.array([g[0][dj, di] for dj, di in cells])
    err = np.abs(got - fd) / np.maximum(np.abs(fd), 1e-2 * np.max(np.abs(g[0])))
    assert np.max(err) <= TOL_GRAD, (got, fd)
    batch.close()


def _onehot(n, dj, di):
    z = np.zeros((n, n))
    z[dj, di] = 1.0
    return z


def test_design_set_from_device_memory_equals_host_values():
    """fdtd_set_design with on_device: the coefficients formed by the kernel
    from a CUDA tensor give the same run as the host path, and an invalid value
    found on the device is refused and drops the rectangle."""
    import torch
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.adjoint_scenes(side=96, n_designs=1, nsteps=200, npml=8, design=24, n_monitors=3)[0]
    i0, j0, w, h = sc.design
    sig = np.full((h, w), 0.02)
    out = []
    for dev in (False, True):
        sim = fdtd.from_scene(sc)
        if dev:
            sim.set_design(i0, j0, torch.tensor(sc.design_eps, device="cuda"), torch.tensor(sig, device="cuda"))
        else:
            sim.set_design(i0, j0, sc.design_eps, sig)
        sim.step(200)
        out.append({c: sim.get_field(c, (sc.ny, sc.nx)) for c in ("ez", "hx", "hy")})
        if dev:
            bad = torch.tensor(sc.design_eps, device="cuda")
            bad[3, 4] = 0.0
            with pytest.raises(fdtd.FDTDError) as ei:
                sim.set_design(i0, j0, bad)
            assert ei.value.code == fdtd.EINVAL
        sim.close()
    for c in ("ez", "hx", "hy"):
        assert rel_l2(out[1][c], out[0][c]) <= 1e-7, c
