"""Pins of the FP64 2D oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
discrete cavity modes (Yee's numerical dispersion relation), the 2x2 leapfrog
recurrence of a lossy mode, the exactly conserved discrete energy, the Courant
limit, mirror symmetry, textbook source / DFT definitions, and the literal graph
of Prop. 1/2 evaluated as a sparse matrix product.
"""
import math

import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes

MU0 = 4e-7 * math.pi
C0 = 299792458.0
EPS0 = 1.0 / (MU0 * C0 * C0)


def _mode(nx, ny, m, n):
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    return np.sin(m * math.pi * i / nx) * np.sin(n * math.pi * j / ny)


def _mode_h_init(phi, dt, dx, dy):
    """H^{-1/2} = (dt / 2 mu0) K^T phi, the half-step-back field of a standing mode."""
    ny, nx = phi.shape
    pad = np.zeros((ny + 1, nx + 1))
    pad[:ny, :nx] = phi
    dphi_x = pad[:ny, 1:nx + 1] - pad[:ny, :nx]
    dphi_y = pad[1:ny + 1, :nx] - pad[:ny, :nx]
    hy = -(dt / (2 * MU0)) * dphi_x / dx
    hx = (dt / (2 * MU0)) * dphi_y / dy
    return hx, hy


def _omega_d(nx, ny, m, n, dx, dy, dt):
    s2 = (C0 * dt) ** 2 * (math.sin(m * math.pi / (2 * nx)) ** 2 / dx ** 2 +
                           math.sin(n * math.pi / (2 * ny)) ** 2 / dy ** 2)
    return 2.0 * math.asin(math.sqrt(s2)) / dt


@pytest.mark.parametrize("nx,ny,m,n", [(32, 24, 1, 1), (32, 24, 3, 2), (17, 29, 5, 7)])
def test_cavity_mode_closed_form(oracle_mod, nx, ny, m, n):
    dx, dy = 1e-3, 1.3e-3
    dt = 0.95 / (C0 * math.sqrt(1 / dx ** 2 + 1 / dy ** 2))
    sim = oracle_mod.TMz(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, npml=0)
    phi = _mode(nx, ny, m, n)
    hx, hy = _mode_h_init(phi, dt, dx, dy)
    sim.set_state(ez=phi, hx=hx, hy=hy)
    w = _omega_d(nx, ny, m, n, dx, dy, dt)
    for blk in range(4):
        sim.run(50)
        expect = math.cos(w * sim.n * dt) * phi
        assert np.max(np.abs(sim.state["ez"] - expect)) < 1e-11


def test_cavity_spectral_peak_matches_continuum(oracle_mod):
    """Config-1 cavity (a = b = 128 mm) rung by the centred Ricker: the lowest
    excited mode sits at the discrete TM11 frequency, which is within 0.1 % of the
    continuum (c/2) sqrt(2)/a = 1.656 GHz."""
    sc = scenes.cavity_ricker(nsteps=8000)
    sim = oracle_mod.TMz(sc)
    out = sim.run(8000, samples=[(40, 40, "ez")])
    sig = out["samples"][:, 0]
    sig = sig[200:]
    f_cont = 0.5 * C0 * math.sqrt(2) / 0.128
    fd = _omega_d(128, 128, 1, 1, sc.dx, sc.dy, sc.dt) / (2 * math.pi)
    assert abs(fd - f_cont) / f_cont < 1e-3
    freqs = np.linspace(1.3e9, 2.0e9, 1401)
    t = (np.arange(len(sig)) + 201) * sc.dt
    spec = np.abs(np.exp(-2j * math.pi * freqs[:, None] * t[None, :]) @ sig)
    f_peak = freqs[np.argmax(spec)]
    assert abs(f_peak - fd) / fd < 5e-3


def test_lossy_mode_matches_2x2_recurrence(oracle_mod):
    nx = ny = 16
    dx = dy = 1e-3
    dt = 0.9 / (C0 * math.sqrt(2) / dx)
    eps_r, sig = 4.0, 0.02
    sim = oracle_mod.TMz(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, eps_cell=np.full((ny, nx), eps_r),
                         sigma_cell=np.full((ny, nx), sig))
    m, n = 2, 1
    phi = _mode(nx, ny, m, n)
    sim.set_state(ez=phi)
    lam = 4 * math.sin(m * math.pi / (2 * nx)) ** 2 / dx ** 2 + 4 * math.sin(n * math.pi / (2 * ny)) ** 2 / dy ** 2
    eps = EPS0 * eps_r
    x = sig * dt / (2 * eps)
    ca, cb = (1 - x) / (1 + x), dt / (eps * (1 + x))
    M = np.array([[ca - cb * lam * dt / MU0, cb * lam], [-dt / MU0, 1.0]])
    v = np.array([1.0, 0.0])
    for k in range(300):
        sim.run(1)
        v = M @ v
        if k % 37 == 0 or k == 299:
            assert np.max(np.abs(sim.state["ez"] - v[0] * phi)) < 1e-12


def test_loss_coefficient_matches_exponential_decay(oracle_mod):
    """A uniform field with no curl decays by Ca per step; the semi-implicit
    averaging of eq. (7) matches exp(-sigma t / eps) to third order."""
    dt, eps_r, sig, n = 1e-12, 2.0, 0.5, 200
    ca, cb = oracle_mod.coeffs_e(np.array([eps_r]), np.array([sig]), dt)
    a = sig * dt / (EPS0 * eps_r)
    assert abs(ca[0] ** n - math.exp(-a * n)) < n * a ** 3 / 12 + 1e-15
    ca0, cb0 = oracle_mod.coeffs_e(np.array([eps_r]), np.array([0.0]), dt)
    assert ca0[0] == 1.0 and abs(cb0[0] - dt / (EPS0 * eps_r)) < 1e-15 * cb0[0]


def test_energy_exactly_conserved(oracle_mod):
    nx, ny = 40, 30
    dx, dy = 1e-3, 0.8e-3
    dt = 0.99 / (C0 * math.sqrt(1 / dx ** 2 + 1 / dy ** 2))
    eps = 1.0 + 8.0 * np.random.default_rng(3).random((ny, nx))
    sim = oracle_mod.TMz(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, eps_cell=eps)
    ez = scenes.random_fields(11, (ny, nx))
    ez[0, :] = 0
    ez[:, 0] = 0
    sim.set_state(ez=ez, hx=scenes.random_fields(12, (ny, nx), 1e-3), hy=scenes.random_fields(13, (ny, nx), 1e-3))
    w = []
    for _ in range(300):
        hx0, hy0 = sim.state["hx"].copy(), sim.state["hy"].copy()
        sim.layer_h()  # H^{n+1/2} from H^{n-1/2}
        w.append(sim.energy(hx0, hy0))
        sim.layer_e()
    w = np.array(w)
    assert np.max(np.abs(w - w[0])) / abs(w[0]) < 1e-12


@pytest.mark.parametrize("S,blows", [(1.01, True), (0.99, False)])
def test_courant_limit(oracle_mod, S, blows):
    nx = ny = 48
    dx = dy = 1e-3
    dt = S / (C0 * math.sqrt(2) / dx)
    sim = oracle_mod.TMz(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt)
    ez = scenes.random_fields(5, (ny, nx))
    ez[0, :] = 0
    ez[:, 0] = 0
    sim.set_state(ez=ez)
    sim.run(300)
    amp = np.max(np.abs(sim.state["ez"]))
    if blows:
        assert amp > 1e6
    else:
        assert amp < 10.0


def test_mirror_symmetry_config1(oracle_mod):
    sc = scenes.cavity_ricker(nsteps=300)
    sim = oracle_mod.TMz(sc)
    sim.run(300)
    ez = sim.state["ez"]
    n = sc.nx
    i = np.arange(1, n)
    scale = np.max(np.abs(ez))
    mir = ez[1:, :][:, i][:, ::-1]  # Ez(N - i, j) for i = 1..N-1
    assert np.max(np.abs(ez[1:, 1:] - mir)) <= 1e-13 * scale
    assert np.max(np.abs(ez - ez.T)) <= 1e-13 * scale
    hy = sim.state["hy"]
    # Hy at (i+1/2) is odd under x -> N - x: Hy(i) = -Hy(N-1-i)
    assert np.max(np.abs(hy[1:, :] + hy[1:, ::-1])) <= 1e-13 * np.max(np.abs(hy))


@pytest.mark.parametrize("nx,ny", [(4, 4), (7, 5), (17, 9), (33, 17)])
def test_prop1_index_maps_are_a_bijection(oracle_mod, nx, ny):
    sim = oracle_mod.TMz(nx=nx, ny=ny, dx=1e-3, dy=1e-3, dt=1e-12)
    idx = []
    for j in range(ny):
        for i in range(nx):
            for k in ("t", "u", "q"):
                idx.append(sim.node_index(k, i, j))
    assert sorted(idx) == list(range(3 * nx * ny))
    assert sim.graph_nodes() == 3 * nx * ny  # no CPML, no extra nodes


def _random_state(sim, seed):
    rng = np.random.default_rng(seed)
    st = {}
    for k in ("ez", "hx", "hy", "pezx", "pezy", "phxy", "phyx"):
        st[k] = rng.standard_normal((sim.ny, sim.nx))
    st["ez"][0, :] = 0
    st["ez"][:, 0] = 0
    # psi lives only where its profile is non-zero
    px, py = sim.px, sim.py
    st["pezx"] *= ((px["bE"] != 0) | (px["cE"] != 0))[None, :]
    st["pezy"] *= ((py["bE"] != 0) | (py["cE"] != 0))[:, None]
    st["phyx"] *= ((px["bH"] != 0) | (px["cH"] != 0))[None, :]
    st["phxy"] *= ((py["bH"] != 0) | (py["cH"] != 0))[:, None]
    st["pezx"][0, :] = st["pezx"][:, 0] = 0
    st["pezy"][0, :] = st["pezy"][:, 0] = 0
    return st


@pytest.mark.parametrize("nx,ny,npml,lossy", [(4, 4, 0, False), (17, 9, 0, True), (24, 20, 4, True),
                                              (31, 26, 6, False)])
def test_graph_form_equals_stencil(oracle_mod, nx, ny, npml, lossy):
    """Prop. 2: two message-passing layers over the Prop. 1 graph reproduce the
    stencil recurrence (identical up to FP64 summation order)."""
    rng = np.random.default_rng(nx * 100 + ny)
    eps = 1 + 11 * rng.random((ny, nx))
    sig = 0.05 * rng.random((ny, nx)) if lossy else np.zeros((ny, nx))
    dx, dy = 1e-3, 1.1e-3
    dt = 0.99 / (C0 * math.sqrt(1 / dx ** 2 + 1 / dy ** 2))
    sim = oracle_mod.TMz(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, npml=npml, eps_cell=eps, sigma_cell=sig)
    st = _random_state(sim, 7)
    sim.set_state(**st)
    h = sim.to_nodes()
    W1 = sim.graph_layer(1)
    W2 = sim.graph_layer(2)
    for _ in range(20):
        h = sim.csr_mv(*W1, h)
        h = sim.csr_mv(*W2, h)
    sim.run(20)
    ref = sim.to_nodes()
    assert np.max(np.abs(h - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_sources_match_closed_forms(oracle_mod):
    fp = 10e9
    t0 = 1.5 / fp
    # Ricker: peak 1 at t0, zeros at t0 +- 1/(sqrt(2) pi fp), minima -2 e^{-3/2} at t0 +- sqrt(1.5)/(pi fp)
    for t, v in [(t0, 1.0), (t0 + 1 / (math.sqrt(2) * math.pi * fp), 0.0),
                 (t0 - 1 / (math.sqrt(2) * math.pi * fp), 0.0),
                 (t0 + math.sqrt(1.5) / (math.pi * fp), -2 * math.exp(-1.5))]:
        n = 37
        s = oracle_mod.waveform("ricker", fp, t / (n + 1), n + 1)
        assert abs(s[n] - v) < 1e-12
    f0 = 2.4e9
    tg = 1 / f0
    for t, v in [(4 * tg, 0.0), (4 * tg + 0.25 / f0, math.exp(-(0.25) ** 2)),
                 (4 * tg - 0.25 / f0, -math.exp(-(0.25) ** 2))]:
        s = oracle_mod.waveform("gauss_mod", f0, t / 51, 51)
        assert abs(s[50] - v) < 1e-12
    s = oracle_mod.waveform("gauss", 1e10, 4e-10 / 40, 40)
    assert abs(s[39] - 1.0) < 1e-15


def test_running_dft_equals_direct_sum(oracle_mod):
    sc = scenes.cavity_ricker(nsteps=400)
    sim = oracle_mod.TMz(sc)
    cells = [(30, 70), (64, 64), (100, 12)]
    freqs = np.array([1.0e9, 3.3e9, 7.5e9])
    out = sim.run(400, samples=[(i, j, "ez") for i, j in cells], dft_cells=np.array(cells), freqs=freqs)
    t = (np.arange(400) + 1) * sc.dt
    direct = (out["samples"].T @ np.exp(-2j * math.pi * freqs[None, :] * t[:, None])) * sc.dt
    re, im = sim.dft
    assert np.max(np.abs(re - direct.real)) <= 1e-12 * np.max(np.abs(direct))
    assert np.max(np.abs(im - direct.imag)) <= 1e-12 * np.max(np.abs(direct))


@pytest.mark.parametrize("npml,bound_db", [(8, -75.0), (16, -95.0)])
def test_cpml_reflection_bound(oracle_mod, npml, bound_db):
    """CPML has no closed form: compare a probe against a domain so large that no
    boundary echo reaches the probe in the window.  The reflection must stay below
    a bound about 15 dB above the level this grading reaches (-90 / -110 dB);
    a wrong sign, scale or missing term in the profile or the psi recursion
    raises it far above that."""
    f0 = 2.4e9
    dx = scenes._dx_for(2 * f0, 1.0, 20)
    dt = 0.99 * dx / (C0 * math.sqrt(2))
    nsteps = 900
    src = scenes.Source(0, 0, kind="gauss_mod", params=(f0,))

    def run(n, npml, off):
        s = scenes.Source(off + 30, off + 60, kind="gauss_mod", params=(f0,))
        sim = oracle_mod.TMz(nx=n, ny=n, dx=dx, dy=dx, dt=dt, npml=npml, source=s, nsteps_src=nsteps)
        return sim.run(nsteps, samples=[(off + 24, off + 60, "ez")])["samples"][:, 0]

    small = run(120, npml, 0)
    big = run(120 + 2 * 900, 0, 900)
    refl = np.max(np.abs(small - big)) / np.max(np.abs(big))
    assert 20 * math.log10(refl) < bound_db
    del src


def test_sine_source_closed_form_and_period(oracle_mod):
    """The sinusoidal source (Sec. V-A) is s(t) = sin(2 pi f t) from t = 0: peaks
    +1 / -1 a quarter and three quarters into each period, zero at half periods,
    and periodic with 1/f."""
    f = 3e9
    for t, v in [(0.25 / f, 1.0), (0.75 / f, -1.0), (0.5 / f, 0.0), (7.25 / f, 1.0)]:
        n = 29
        s = oracle_mod.waveform("sine", f, t / (n + 1), n + 1)
        assert abs(s[n] - v) < 1e-12
    dt = 1 / (f * 40)           # exactly 40 steps per period
    s = oracle_mod.waveform("sine", f, dt, 200)
    assert np.max(np.abs(s[40:] - s[:-40])) < 1e-12


def test_line_source_is_the_sum_of_point_sources(oracle_mod):
    """The recurrence is linear, so a line source over cells (i, j0 .. j1-1) must
    give the sum of the runs of point sources at those cells (heterogeneous lossy
    medium with a CPML): a cell skipped, doubled or misplaced fails it."""
    sc = scenes.ellipse_scene(side=80, nsteps=150)
    i, j0, j1 = 23, 30, 37
    line = scenes.Source(i, j0, kind="gauss_mod", params=(20e9,), length=j1 - j0)
    sim = oracle_mod.TMz(sc, source=line, nsteps_src=sc.nsteps)
    sim.run(sc.nsteps)
    total = {k: np.zeros((sc.ny, sc.nx)) for k in ("ez", "hx", "hy")}
    for j in range(j0, j1):
        pt = oracle_mod.TMz(sc, source=scenes.Source(i, j, kind="gauss_mod", params=(20e9,)), nsteps_src=sc.nsteps)
        pt.run(sc.nsteps)
        for k in total:
            total[k] += pt.state[k]
    for k in total:
        assert np.max(np.abs(sim.state[k] - total[k])) <= 1e-12 * np.max(np.abs(total[k])), k


def _cpml_recover(b, c, dt):
    """Invert the one-step recursive-convolution coefficients of a CPML node
    with kappa = 1: b = exp(-(sigma + alpha) dt / eps0) gives sigma + alpha, and
    c = sigma (b - 1) / (sigma + alpha) then gives sigma; alpha is the rest."""
    eps0 = 1.0 / (MU0 * C0 ** 2)
    s_plus_a = -np.log(b) * eps0 / dt
    sigma = c * s_plus_a / (b - 1.0)
    return sigma, s_plus_a - sigma


def test_cpml_profile_values_at_fixed_depths(oracle_mod):
    """The absorber's profiles (Sec. III-C; Roden-Gedney CPML with the grading
    chosen for these workloads): polynomial sigma of order 3 up to
    sigma_max = 0.8 (m + 1) / (eta0 delta) at the PEC, kappa = 1, and alpha
    falling linearly from alpha_max = 0.05 S/m at the inner interface to 0 at the
    PEC.  E nodes sit at integer depths rho = npml - i, H nodes half a cell
    further in.  sigma and alpha are recovered from (b, c) at every node and
    compared with the profile written out at each depth, with hand values at
    rho = 1/2, 1, npml - 1/2 and npml; a reversed alpha ramp or a half-cell
    shift of the H nodes fails."""
    n, npml, d = 40, 8, 1e-3
    dt = 0.99 * d / (C0 * math.sqrt(2))
    eps0 = 1.0 / (MU0 * C0 ** 2)
    p = oracle_mod.cpml_axis(n, npml, d, dt)
    eta0 = math.sqrt(MU0 / eps0)
    smax, amax = 0.8 * 4 / (eta0 * d), 0.05
    assert np.all(p["kE"] == 1.0) and np.all(p["kH"] == 1.0)
    # outside the layer the node is a plain Yee node: b = c = 0 (psi stays zero)
    assert np.all(p["bE"][npml:n - npml + 1] == 0.0) and np.all(p["cE"][npml:n - npml + 1] == 0.0)
    assert np.all(p["bH"][npml:n - npml] == 0.0) and np.all(p["cH"][npml:n - npml] == 0.0)
    # depth of every node inside the layer, both faces
    nodes = [("E", i, npml - i) for i in range(npml)] + [("E", i, i - (n - npml)) for i in range(n - npml + 1, n)]
    nodes += [("H", i, npml - i - 0.5) for i in range(npml)] + \
             [("H", i, i + 0.5 - (n - npml)) for i in range(n - npml, n)]
    for kind, i, rho in nodes:
        b, c = p["b" + kind][i], p["c" + kind][i]
        sig, alp = _cpml_recover(b, c, dt)
        x = rho / npml
        assert math.isclose(sig, smax * x ** 3, rel_tol=1e-9), (kind, i, rho)
        assert math.isclose(alp, amax * (1.0 - x), rel_tol=1e-7, abs_tol=1e-9 * amax), (kind, i, rho)
    # hand values: rho = 1/2 (H node next to the interface, both faces)
    for i in (npml - 1, n - npml):
        sig, alp = _cpml_recover(p["bH"][i], p["cH"][i], dt)
        assert math.isclose(sig, smax / 4096.0, rel_tol=1e-9)          # (1/16)^3
        assert math.isclose(alp, amax * 15.0 / 16.0, rel_tol=1e-9)
    # rho = 1 (E node one cell in)
    sig, alp = _cpml_recover(p["bE"][npml - 1], p["cE"][npml - 1], dt)
    assert math.isclose(sig, smax / 512.0, rel_tol=1e-9) and math.isclose(alp, amax * 7.0 / 8.0, rel_tol=1e-9)
    # rho = npml - 1/2 (outermost H node, both faces)
    for i in (0, n - 1):
        sig, alp = _cpml_recover(p["bH"][i], p["cH"][i], dt)
        assert math.isclose(sig, smax * (15.0 / 16.0) ** 3, rel_tol=1e-9)
        assert math.isclose(alp, amax / 16.0, rel_tol=1e-6)
    # rho = npml: the E node on the PEC wall has alpha = 0, so c = b - 1 and
    # b = exp(-sigma_max dt / eps0)
    assert math.isclose(p["bE"][0], math.exp(-smax * dt / eps0), rel_tol=1e-13)
    assert math.isclose(p["cE"][0], p["bE"][0] - 1.0, rel_tol=1e-13)


def test_cpml_coefficients_integrate_the_kernel(oracle_mod):
    """c is the CPML's causal kernel -(sigma / eps0) exp(-(sigma + alpha) tau / eps0)
    (kappa = 1) integrated over one step, and b its decay over one step, so that
    psi^{n+1} = b psi^n + c dF is the exact recursive convolution for a
    piecewise-constant dF.  The integral is taken numerically (Gauss-Legendre),
    with sigma and alpha written out from the grading at each depth."""
    n, npml, d = 30, 6, 2e-3
    dt = 0.99 * d / (C0 * math.sqrt(2))
    eps0 = 1.0 / (MU0 * C0 ** 2)
    p = oracle_mod.cpml_axis(n, npml, d, dt)
    smax = 0.8 * 4 / (math.sqrt(MU0 / eps0) * d)
    xg, wg = np.polynomial.legendre.leggauss(40)
    tau = 0.5 * dt * (xg + 1.0)
    for kind, i, rho in [("E", i, npml - i) for i in range(npml)] + [("H", i, npml - i - 0.5) for i in range(npml)]:
        sig = smax * (rho / npml) ** 3
        alp = 0.05 * (1.0 - rho / npml)
        kern = -(sig / eps0) * np.exp(-(sig + alp) * tau / eps0)
        c_int = 0.5 * dt * float(np.dot(wg, kern))
        b_dec = math.exp(-(sig + alp) * dt / eps0)
        assert math.isclose(p["c" + kind][i], c_int, rel_tol=1e-12), (kind, i)
        assert math.isclose(p["b" + kind][i], b_dec, rel_tol=1e-13), (kind, i)
