"""Pins of the FP64 3D Yee oracle: closed-form discrete cavity modes (3-term
numerical dispersion), exact discrete energy, and the 3D Courant limit."""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes

MU0 = 4e-7 * math.pi
C0 = 299792458.0


def _grid(nx, ny, nz):
    i = np.arange(nx)[None, None, :].astype(float)
    j = np.arange(ny)[None, :, None].astype(float)
    k = np.arange(nz)[:, None, None].astype(float)
    return i, j, k


def _mode3(nx, ny, nz, m, n, p, d, amp):
    """Standing discrete mode of the PEC box: each E component sampled at its Yee
    position, amplitudes amp orthogonal to the discrete wave vector."""
    dx, dy, dz = d
    kx, ky, kz = m * math.pi / (nx * dx), n * math.pi / (ny * dy), p * math.pi / (nz * dz)
    i, j, k = _grid(nx, ny, nz)
    ex = amp[0] * np.cos(kx * (i + 0.5) * dx) * np.sin(ky * j * dy) * np.sin(kz * k * dz)
    ey = amp[1] * np.sin(kx * i * dx) * np.cos(ky * (j + 0.5) * dy) * np.sin(kz * k * dz)
    ez = amp[2] * np.sin(kx * i * dx) * np.sin(ky * j * dy) * np.cos(kz * (k + 0.5) * dz)
    return ex, ey, ez


def _curl_e(ex, ey, ez, d):
    """curl E as the H update uses it (forward differences, ghost zeros)."""
    dx, dy, dz = d

    def fwd(a, axis):
        pad = np.concatenate([a, np.zeros_like(np.take(a, [0], axis=axis))], axis=axis)
        return np.diff(pad, axis=axis)
    cx = fwd(ez, 1) / dy - fwd(ey, 0) / dz
    cy = fwd(ex, 0) / dz - fwd(ez, 2) / dx
    cz = fwd(ey, 2) / dx - fwd(ex, 1) / dy
    return cx, cy, cz


@pytest.mark.parametrize("mnp,amp", [((1, 1, 0), None), ((1, 2, 1), None), ((2, 1, 3), None)])
def test_cavity_mode_3d(oracle_mod, mnp, amp):
    nx, ny, nz = 14, 12, 10
    d = (1e-3, 1.2e-3, 0.9e-3)
    dt = 0.95 / (C0 * math.sqrt(sum(1 / x ** 2 for x in d)))
    m, n, p = mnp
    kt = np.array([2 / d[0] * math.sin(m * math.pi / (2 * nx)), 2 / d[1] * math.sin(n * math.pi / (2 * ny)),
                   2 / d[2] * math.sin(p * math.pi / (2 * nz))])
    # amplitude orthogonal to the discrete wave vector (divergence-free mode)
    a = np.cross(kt, np.array([0.3, -0.7, 1.1])) if p != 0 else np.array([0.0, 0.0, 1.0])
    sim = oracle_mod.Yee3D(nx=nx, ny=ny, nz=nz, dx=d[0], dy=d[1], dz=d[2], dt=dt)
    ex, ey, ez = _mode3(nx, ny, nz, m, n, p, d, a)
    cx, cy, cz = _curl_e(ex, ey, ez, d)
    f = dt / (2 * MU0)
    sim.set_state(ex=ex, ey=ey, ez=ez, hx=f * cx, hy=f * cy, hz=f * cz)
    s2 = (C0 * dt / 2) ** 2 * float(np.sum(kt ** 2))
    w = 2 * math.asin(math.sqrt(s2)) / dt
    scale = max(np.max(np.abs(ex)), np.max(np.abs(ey)), np.max(np.abs(ez)))
    for _ in range(3):
        sim.run(40)
        c = math.cos(w * sim.n * dt)
        for name, ref in (("ex", ex), ("ey", ey), ("ez", ez)):
            assert np.max(np.abs(sim.state[name] - c * ref)) < 1e-11 * scale, name


def _random_e(nx, ny, nz, seed):
    ex = scenes.random_fields(seed, (nz, ny, nx))
    ey = scenes.random_fields(seed + 1, (nz, ny, nx))
    ez = scenes.random_fields(seed + 2, (nz, ny, nx))
    ex[:, 0, :] = 0; ex[0, :, :] = 0
    ey[:, :, 0] = 0; ey[0, :, :] = 0
    ez[:, :, 0] = 0; ez[:, 0, :] = 0
    return ex, ey, ez


def test_energy_exactly_conserved_3d(oracle_mod):
    nx, ny, nz = 12, 10, 9
    d = (1e-3, 0.9e-3, 1.1e-3)
    dt = 0.99 / (C0 * math.sqrt(sum(1 / x ** 2 for x in d)))
    eps = 1 + 8 * np.random.default_rng(1).random((nz, ny, nx))
    sim = oracle_mod.Yee3D(nx=nx, ny=ny, nz=nz, dx=d[0], dy=d[1], dz=d[2], dt=dt, eps_cell=eps)
    ex, ey, ez = _random_e(nx, ny, nz, 20)
    sim.set_state(ex=ex, ey=ey, ez=ez, hx=scenes.random_fields(30, (nz, ny, nx), 1e-3),
                  hy=scenes.random_fields(31, (nz, ny, nx), 1e-3), hz=scenes.random_fields(32, (nz, ny, nx), 1e-3))
    w = []
    for _ in range(120):
        # W^n needs E^n with H^{n+1/2} and H^{n-1/2}: keep E^n and H^{n-1/2},
        # step once, evaluate with E^n put back, then restore E^{n+1}
        h_prev = [sim.state[k].copy() for k in ("hx", "hy", "hz")]
        e_n = {k: sim.state[k].copy() for k in ("ex", "ey", "ez")}
        sim.run(1)
        e_next = {k: sim.state[k].copy() for k in ("ex", "ey", "ez")}
        sim.set_state(**e_n)
        w.append(sim.energy(*h_prev))
        sim.set_state(**e_next)
    w = np.array(w)
    assert np.max(np.abs(w - w[0])) / abs(w[0]) < 1e-12


@pytest.mark.parametrize("S,blows", [(1.01, True), (0.99, False)])
def test_courant_limit_3d(oracle_mod, S, blows):
    n = 16
    dx = 1e-3
    dt = S / (C0 * math.sqrt(3) / dx)
    sim = oracle_mod.Yee3D(nx=n, ny=n, nz=n, dx=dx, dy=dx, dz=dx, dt=dt)
    ex, ey, ez = _random_e(n, n, n, 40)
    sim.set_state(ex=ex, ey=ey, ez=ez)
    sim.run(400)
    amp = max(np.max(np.abs(sim.state[k])) for k in ("ex", "ey", "ez"))
    assert (amp > 1e6) if blows else (amp < 10.0)


def test_3d_reduces_to_2d_tmz(oracle_mod):
    """A z-invariant Ez-only field with no z-PML evolves exactly like 2D TMz."""
    nx, ny, nz = 20, 16, 4
    dx, dy, dz = 1e-3, 1e-3, 1e-3
    dt = 0.99 / (C0 * math.sqrt(1 / dx ** 2 + 1 / dy ** 2 + 1 / dz ** 2))
    eps2 = 1 + 5 * np.random.default_rng(8).random((ny, nx))
    s3 = oracle_mod.Yee3D(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, dt=dt,
                          eps_cell=np.broadcast_to(eps2, (nz, ny, nx)).copy())
    s2 = oracle_mod.TMz(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, eps_cell=eps2)
    ez = scenes.random_fields(3, (ny, nx))
    ez[0, :] = 0
    ez[:, 0] = 0
    s3.set_state(ez=np.broadcast_to(ez, (nz, ny, nx)).copy())
    s2.set_state(ez=ez)
    s3.run(30)
    s2.run(30)
    for k in range(nz):
        assert np.max(np.abs(s3.state["ez"][k] - s2.state["ez"])) < 1e-14 * np.max(np.abs(s2.state["ez"]))
        assert np.max(np.abs(s3.state["hy"][k] - s2.state["hy"])) < 1e-14 * np.max(np.abs(s2.state["hy"]))


@pytest.mark.parametrize("comp", ["ez", "ex"])
def test_cpml_reflection_bound_3d(oracle_mod, comp):
    """The 3D psi recursions: a probe near a Ricker dipole inside a CPML box
    against an enlarged PEC box whose echoes cannot reach it in the window.  A
    z-directed and an x-directed dipole between them excite all six components."""
    dx = 1e-3
    dt = 0.99 * dx / (C0 * math.sqrt(3))
    nsteps = 130
    fp = 15e9

    def run(n, npml, off):
        src = scenes.Source(off + 16, off + 15, off + 17, component=comp, kind="ricker", params=(fp,))
        sim = oracle_mod.Yee3D(nx=n, ny=n, nz=n, dx=dx, dy=dx, dz=dx, dt=dt, npml=npml, source=src,
                               nsteps_src=nsteps)
        out = sim.run(nsteps, samples=[(off + 12, off + 13, off + 20, c) for c in ("ex", "ey", "ez", "hx", "hy", "hz")])
        return out["samples"]

    small = run(32, 8, 0)
    big = run(32 + 2 * 80, 0, 80)
    amp = np.max(np.abs(big), axis=0)
    for c in range(6):
        kind_max = np.max(amp[:3]) if c < 3 else np.max(amp[3:])
        if amp[c] < 1e-6 * kind_max:
            continue  # zero by the dipole's symmetry, up to rounding
        refl = np.max(np.abs(small[:, c] - big[:, c])) / amp[c]
        assert 20 * math.log10(refl) < -70.0, c  # this grading reaches -81 .. -104 dB


def test_plane_dft_equals_direct_sum_3d(oracle_mod):
    """The running DFT of a plane (Sec. I: frequency responses from sampled
    waveforms): F(f) = sum_{n>=1} E^n exp(-i 2 pi f n dt) dt over every cell of
    the plane and every E component, against a direct FP64 sum of the stored
    samples.  The run is split in two calls, so the step count carried between
    calls enters the phase as well."""
    sc = scenes.box_scene(side=20, nsteps=90, npml=4, n_boxes=3)
    sc.source = scenes.Source(9, 8, 10, component="ez", kind="ricker", params=(20e9,))
    kp = 11
    freqs = np.array([2.5e9, 6.0e9, 9.5e9])
    comps = ("ex", "ey", "ez")
    sim = oracle_mod.Yee3D(sc)
    samples = [(i, j, kp, c) for c in comps for j in range(sc.ny) for i in range(sc.nx)]
    a = sim.run(50, samples=samples, plane_k=kp, plane_comps=comps, freqs=freqs)["samples"]
    b = sim.run(40, samples=samples, plane_k=kp, plane_comps=comps, freqs=freqs)["samples"]
    series = np.concatenate([a, b])                       # row q holds E^{q+1}
    t = (np.arange(series.shape[0]) + 1) * sc.dt
    direct = (series.T @ np.exp(-2j * math.pi * freqs[None, :] * t[:, None])) * sc.dt
    direct = direct.reshape(len(comps), sc.ny, sc.nx, len(freqs)).transpose(0, 3, 1, 2)
    re, im = sim.plane
    scale = np.max(np.abs(direct))
    assert scale > 0
    assert np.max(np.abs(re - direct.real)) <= 1e-12 * scale
    assert np.max(np.abs(im - direct.imag)) <= 1e-12 * scale
    # the plane is not trivially zero: the dipole reaches every component
    for c in range(3):
        assert np.max(np.abs(direct[c])) > 1e-3 * scale
