"""Seeded synthetic scene generators (inputs only).

This module produces the *inputs* of an FDTD run: grid sizes, cell sizes and
time step, a uint8 material-index map with its material table (eps_r, sigma),
source positions, probe / monitor cells and continuous design regions.  It holds
none of the method's arithmetic (no update coefficients, no CPML profiles, no
waveforms): the CUDA library and the FP64 oracle each compute those from these
inputs on their own.

Workload shapes follow the paper's experiments (random dielectric shapes of
random permittivity and conductivity on a vacuum background, random source
positions, grid sides in the paper's 200-6400 range; Sec. V-A and V-C).  The
paper's own scenes are not available, so these seeded scenes stand in for them.

Random numbers come from numpy's PCG64 bit generator and only through
``Generator.random`` (53-bit uniform doubles), whose stream is fixed by the
published PCG64 definition; every other draw is derived from those doubles here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C0 = 299792458.0            # speed of light in vacuum, m/s (SI definition)
SEED_BASE = 240500814       # seed of workload k is SEED_BASE + k

# material index reserved by the CUDA library for PEC cells; scenes never use it
MAX_USER_MATERIALS = 255


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _u(rng, lo, hi, size=None):
    return lo + (hi - lo) * rng.random(size)


@dataclass
class Source:
    """A soft point source: the field component at a cell gets s(t) added after
    each E update.  kind is 'ricker', 'gauss_mod', 'gauss', 'sine' or 'sampled'."""
    i: int
    j: int
    k: int = 0
    component: str = "ez"
    kind: str = "ricker"
    params: tuple = ()            # ricker: (f_peak,); gauss_mod: (f0,); gauss: (f_max,); sine: (f,)
    samples: np.ndarray | None = None   # kind == 'sampled': s((n+1) dt) for n = 0..
    length: int = 1               # 2D line source: cells (i, j .. j + length - 1)


@dataclass
class Scene2D:
    """2D TMz scene: Ez, Hx, Hy on an nx x ny Yee grid (x fastest)."""
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    npml: int
    mat: np.ndarray               # uint8 [ny, nx]
    eps_r: np.ndarray             # float64 [n_mat]
    sigma: np.ndarray             # float64 [n_mat], S/m
    nsteps: int
    source: Source | None = None
    probes: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))  # (i, j)
    design: tuple | None = None   # (i0, j0, w, h) continuous eps_r region
    design_eps: np.ndarray | None = None   # float64 [h, w]
    monitors: np.ndarray | None = None     # (i, j) DFT monitor cells
    freqs: np.ndarray | None = None        # DFT frequencies, Hz
    name: str = ""

    @property
    def cells(self) -> int:
        return self.nx * self.ny


@dataclass
class Scene3D:
    """3D Yee scene: Ex, Ey, Ez, Hx, Hy, Hz on an nx x ny x nz grid."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    dt: float
    npml: int
    mat: np.ndarray               # uint8 [nz, ny, nx]
    eps_r: np.ndarray
    sigma: np.ndarray
    nsteps: int
    source: Source | None = None
    dft_plane_k: int = -1
    dft_components: tuple = ("ex", "ey", "ez")
    freqs: np.ndarray | None = None
    name: str = ""

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


# ----------------------------------------------------------------------------------
# geometry helpers (rasterisation on the Ez node positions, later shapes overwrite)
# ----------------------------------------------------------------------------------

def _raster_ellipses(mat, npml, centres, axes, angles, first_index):
    ny, nx = mat.shape
    lo_x, hi_x, lo_y, hi_y = npml, nx - npml, npml, ny - npml
    for e in range(len(centres)):
        cx, cy = centres[e]
        a, b = axes[e]
        th = angles[e]
        r = max(a, b)
        i0, i1 = max(lo_x, int(math.floor(cx - r))), min(hi_x, int(math.ceil(cx + r)) + 1)
        j0, j1 = max(lo_y, int(math.floor(cy - r))), min(hi_y, int(math.ceil(cy + r)) + 1)
        if i0 >= i1 or j0 >= j1:
            continue
        ii = np.arange(i0, i1, dtype=np.float64)[None, :] - cx
        jj = np.arange(j0, j1, dtype=np.float64)[:, None] - cy
        c, s = math.cos(th), math.sin(th)
        u = ii * c + jj * s
        v = -ii * s + jj * c
        inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        mat[j0:j1, i0:i1][inside] = first_index + e


def ellipse_medium(rng, side: int, npml: int, n_ellipses: int, axis_scale: float,
                   min_axis: float = 0.0):
    """200-ellipse medium of the heterogeneous 2D workload: centres uniform in the
    non-PML interior, semi-axes U[10, 300] * axis_scale cells, rotation U[0, pi),
    eps_r ~ U[1, 12], sigma ~ U[0, 0.05] S/m; index 0 is vacuum."""
    if n_ellipses > MAX_USER_MATERIALS - 1:
        raise ValueError("too many ellipses for a uint8 material map")
    mat = np.zeros((side, side), np.uint8)
    centres = np.stack([_u(rng, npml, side - npml, n_ellipses),
                        _u(rng, npml, side - npml, n_ellipses)], axis=1)
    axes = np.stack([_u(rng, 10.0, 300.0, n_ellipses), _u(rng, 10.0, 300.0, n_ellipses)], axis=1)
    axes = np.maximum(axes * axis_scale, min_axis)
    angles = _u(rng, 0.0, math.pi, n_ellipses)
    eps = np.concatenate([[1.0], _u(rng, 1.0, 12.0, n_ellipses)])
    sig = np.concatenate([[0.0], _u(rng, 0.0, 0.05, n_ellipses)])
    _raster_ellipses(mat, npml, centres, axes, angles, 1)
    return mat, eps, sig


def _dx_for(f_max: float, eps_max: float, ppw: int) -> float:
    return C0 / (f_max * math.sqrt(eps_max)) / ppw


def _dt_2d(dx: float, dy: float, courant: float = 0.99) -> float:
    return courant / (C0 * math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2))


def _dt_3d(dx: float, dy: float, dz: float, courant: float = 0.99) -> float:
    return courant / (C0 * math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2 + 1.0 / dz ** 2))


# ----------------------------------------------------------------------------------
# the five workloads (plus scaled-down variants used by the parity tests)
# ----------------------------------------------------------------------------------

def cavity_ricker(n: int = 128, nsteps: int = 500, n_probes: int = 4) -> Scene2D:
    """128 x 128 vacuum PEC cavity, dx = 1 mm, Ricker (10 GHz peak) soft source at
    the centre, Ez probed at seeded interior cells."""
    rng = _rng(SEED_BASE + 1)
    dx = 1e-3
    dt = _dt_2d(dx, dx)
    probes = set()
    while len(probes) < n_probes:
        i = 1 + int(rng.random() * (n - 1))
        j = 1 + int(rng.random() * (n - 1))
        probes.add((i, j))
    return Scene2D(nx=n, ny=n, dx=dx, dy=dx, dt=dt, npml=0,
                   mat=np.zeros((n, n), np.uint8), eps_r=np.array([1.0]), sigma=np.array([0.0]),
                   nsteps=nsteps,
                   source=Source(n // 2, n // 2, kind="ricker", params=(10e9,)),
                   probes=np.array(sorted(probes), np.int32), name=f"tmz{n}_pec_ricker")


def ellipse_scene(side: int = 4096, nsteps: int = 4000, npml: int = 16, seed_id: int = 2,
                  n_ellipses: int | None = None, n_probes: int = 4) -> Scene2D:
    """Heterogeneous 2D TMz workload: 200 random ellipses (scaled with side/4096 for
    smaller sides), 16-cell CPML, Gaussian-modulated 2.4 GHz soft source at the
    centre, dx = lambda_min / 20 with f_max = 4.8 GHz and eps_max = 12."""
    rng = _rng(SEED_BASE + seed_id)
    scale = side / 4096.0
    if n_ellipses is None:
        n_ellipses = 200 if side == 4096 else max(4, int(round(200 * scale * scale)))
    mat, eps, sig = ellipse_medium(rng, side, npml, n_ellipses, scale, min_axis=3.0 if side != 4096 else 0.0)
    f0 = 2.4e9
    dx = _dx_for(2 * f0, 12.0, 20)
    dt = _dt_2d(dx, dx)
    probes = []
    for _ in range(n_probes):
        probes.append((npml + int(rng.random() * (side - 2 * npml)),
                       npml + int(rng.random() * (side - 2 * npml))))
    return Scene2D(nx=side, ny=side, dx=dx, dy=dx, dt=dt, npml=npml, mat=mat, eps_r=eps,
                   sigma=sig, nsteps=nsteps,
                   source=Source(side // 2, side // 2, kind="gauss_mod", params=(f0,)),
                   probes=np.array(probes, np.int32), name=f"tmz{side}_ellipses_cpml{npml}")


def batch_scenes(n_scenes: int = 64, nsteps: int = 2000, npml: int = 12,
                 side_lo: int = 256, side_hi: int = 2048) -> list[Scene2D]:
    """Batched workload: 64 independent ellipse scenes with log-uniform sides in
    [256, 2048], 12-cell CPML, each with its own seeded source position."""
    rng = _rng(SEED_BASE + 4)
    f0 = 2.4e9
    dx = _dx_for(2 * f0, 12.0, 20)
    dt = _dt_2d(dx, dx)
    out = []
    for s in range(n_scenes):
        side = int(round(math.exp(_u(rng, math.log(side_lo), math.log(side_hi)))))
        scale = side / 4096.0
        n_ell = max(4, int(round(200 * scale * scale)))
        mat, eps, sig = ellipse_medium(rng, side, npml, n_ell, scale, min_axis=3.0)
        si = npml + int(rng.random() * (side - 2 * npml))
        sj = npml + int(rng.random() * (side - 2 * npml))
        out.append(Scene2D(nx=side, ny=side, dx=dx, dy=dx, dt=dt, npml=npml, mat=mat,
                           eps_r=eps, sigma=sig, nsteps=nsteps,
                           source=Source(si, sj, kind="gauss_mod", params=(f0,)),
                           name=f"batch{s}_{side}"))
    return out


def smoothed_noise_design(seed: int, h: int, w: int, smooth: float = 8.0) -> np.ndarray:
    """eps_r = 1 + 11 * minmax(Gaussian-smoothed U[0, 1] noise)."""
    from scipy.ndimage import gaussian_filter
    noise = _rng(seed).random((h, w))
    sm = gaussian_filter(noise, sigma=smooth)
    sm = (sm - sm.min()) / (sm.max() - sm.min())
    return 1.0 + 11.0 * sm


def adjoint_scenes(side: int = 1024, n_designs: int = 8, nsteps: int = 3000, npml: int = 16,
                   design: int = 256, n_monitors: int = 8) -> list[Scene2D]:
    """Inverse-design workload: 1024^2 vacuum + CPML 16, a centred 256^2 continuous
    design region, Gaussian-modulated 5 GHz source at (200, 512), loss
    sum |F(5 GHz)|^2 over 8 seeded monitor cells.  Smaller sides scale every
    position by side/1024."""
    seed = SEED_BASE + 5
    rng = _rng(seed)
    sc = side / 1024.0
    f0 = 5e9
    dx = _dx_for(2 * f0, 12.0, 20)
    dt = _dt_2d(dx, dx)
    i0 = (side - design) // 2
    mon = []
    while len(mon) < n_monitors:
        mi = int(round(_u(rng, 700, 990) * sc))
        mj = int(round(_u(rng, 40, 984) * sc))
        mi = min(max(mi, npml + 1), side - npml - 2)
        mj = min(max(mj, npml + 1), side - npml - 2)
        if (mi, mj) not in mon:
            mon.append((mi, mj))
    src = (int(round(200 * sc)), int(round(512 * sc)))
    out = []
    for b in range(n_designs):
        eps_d = smoothed_noise_design(seed + 1000 * b, design, design, smooth=8.0 * max(sc, 0.125))
        out.append(Scene2D(nx=side, ny=side, dx=dx, dy=dx, dt=dt, npml=npml,
                           mat=np.zeros((side, side), np.uint8), eps_r=np.array([1.0]),
                           sigma=np.array([0.0]), nsteps=nsteps,
                           source=Source(src[0], src[1], kind="gauss_mod", params=(f0,)),
                           design=(i0, i0, design, design), design_eps=eps_d,
                           monitors=np.array(mon, np.int32), freqs=np.array([f0]),
                           name=f"adjoint{side}_design{b}"))
    return out


def fd_cells(n: int, design: int, seed_id: int = 5) -> np.ndarray:
    """Seeded cells (dj, di) inside a design x design region for finite differences."""
    rng = _rng(SEED_BASE + seed_id + 77)
    cells = set()
    while len(cells) < n:
        cells.add((int(rng.random() * design), int(rng.random() * design)))
    return np.array(sorted(cells), np.int32)


def box_scene(side: int = 512, nsteps: int = 2000, npml: int = 10, n_boxes: int = 64,
              seed_id: int = 3) -> Scene3D:
    """3D workload: 64 dielectric boxes (edges U[8, 64] cells per axis, scaled by
    side/512, centres uniform in the interior, eps_r ~ U[1, 9], sigma = 0), z-directed
    Gaussian-pulse dipole at the centre (f_max = 10 GHz), dx = lambda_min / 15,
    DFT plane at z = 3/4 side for Ex, Ey, Ez at 2.5, 5.0 and 7.5 GHz."""
    rng = _rng(SEED_BASE + seed_id)
    sc = side / 512.0
    mat = np.zeros((side, side, side), np.uint8)
    eps = [1.0]
    for b in range(n_boxes):
        edges = [max(2, int(round(_u(rng, 8, 64) * sc))) for _ in range(3)]
        centre = [_u(rng, npml, side - npml) for _ in range(3)]
        lo = [max(npml, int(math.floor(centre[a] - edges[a] / 2))) for a in range(3)]
        hi = [min(side - npml, lo[a] + edges[a]) for a in range(3)]
        eps.append(_u(rng, 1.0, 9.0))
        if all(hi[a] > lo[a] for a in range(3)):
            mat[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = b + 1
    f_max = 10e9
    dx = _dx_for(f_max, 9.0, 15)
    dt = _dt_3d(dx, dx, dx)
    c = side // 2
    return Scene3D(nx=side, ny=side, nz=side, dx=dx, dy=dx, dz=dx, dt=dt, npml=npml, mat=mat,
                   eps_r=np.array(eps), sigma=np.zeros(len(eps)), nsteps=nsteps,
                   source=Source(c, c, c, component="ez", kind="gauss", params=(f_max,)),
                   dft_plane_k=(3 * side) // 4, freqs=np.array([2.5e9, 5.0e9, 7.5e9]),
                   name=f"yee{side}_boxes_cpml{npml}")


def phc_waveguide(nsteps: int = 3000, npml: int = 16, width_um: float = 1.2) -> Scene2D:
    """The photonic-crystal example (Sec. V-B): a dielectric waveguide (eps_r = 12)
    along x, periodic in one dimension by two groups of 3 round air holes of
    radius 0.36 um, 1 um apart within a group, the groups 1.4 um apart; a line
    source across the waveguide near its start driven by a 75 THz
    Gaussian-modulated pulse.  The paper gives no waveguide width (1.2 um here),
    domain size or probe position; dx is 20 points per the shortest wavelength
    (f_max = 150 THz in eps_r = 12) and dt 0.99 of the Courant limit.  Probes: on
    the axis in the gap between the groups and past the holes.  Deterministic:
    no random draws."""
    um = 1e-6
    f0 = 75e12
    dx = _dx_for(2 * f0, 12.0, 20)
    dt = _dt_2d(dx, dx)
    lx, ly = 12.0 * um, 5.0 * um
    nx, ny = int(round(lx / dx)), int(round(ly / dx))
    mat = np.zeros((ny, nx), np.uint8)
    x = np.arange(nx)[None, :] * dx
    y = np.arange(ny)[:, None] * dx
    xc, yc = lx / 2, ly / 2
    mat[np.broadcast_to(np.abs(y - yc) <= width_um * um / 2, (ny, nx))] = 1
    for k in range(3):
        for sgn in (-1.0, 1.0):
            hx = xc + sgn * (0.7 + k * 1.0) * um
            mat[(x - hx) ** 2 + (y - yc) ** 2 <= (0.36 * um) ** 2] = 0
    mat[:npml, :] = 0
    mat[-npml:, :] = 0
    mat[:, :npml] = 0
    mat[:, -npml:] = 0
    jc = int(round(yc / dx))
    half = int(width_um * um / 2 / dx)
    src = Source(int(round(1.0 * um / dx)), jc - half, kind="gauss_mod", params=(f0,), length=2 * half + 1)
    probes = np.array([[int(round(xc / dx)), jc], [int(round((lx - 1.0 * um) / dx)), jc]], np.int32)
    return Scene2D(nx=nx, ny=ny, dx=dx, dy=dx, dt=dt, npml=npml, mat=mat, eps_r=np.array([1.0, 12.0]),
                   sigma=np.array([0.0, 0.0]), nsteps=nsteps, source=src, probes=probes, name="phc_waveguide")


def free_space(side: int, nsteps: int = 1024, npml: int = 16) -> Scene2D:
    """Free-space timing workload of the paper's grid sweep (sides 250..6400,
    1024 steps), with a Gaussian-modulated 2.4 GHz source at the centre."""
    f0 = 2.4e9
    dx = _dx_for(2 * f0, 1.0, 20)
    dt = _dt_2d(dx, dx)
    return Scene2D(nx=side, ny=side, dx=dx, dy=dx, dt=dt, npml=npml,
                   mat=np.zeros((side, side), np.uint8), eps_r=np.array([1.0]),
                   sigma=np.array([0.0]), nsteps=nsteps,
                   source=Source(side // 2, side // 2, kind="gauss_mod", params=(f0,)),
                   name=f"free{side}")


def random_fields(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Seeded U[-scale, scale) field values (initial states for invariance tests)."""
    return scale * (2.0 * _rng(seed).random(shape) - 1.0)
