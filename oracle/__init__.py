"""FP64 CPU oracle (ctypes front end of oracle/liboracle.so).

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py may import this package.
It computes the discrete Yee leapfrog recurrence of arXiv 2405.00814 plainly in
double precision (Sec. III-B eqs. (7)-(9) rotated to TMz, Prop. 1/2 for the
literal graph form) and shares no code with the CUDA path; the two meet only at
the seeded inputs from ``paper_2405_00814_gb300.scenes``.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
tests/test_oracle_*.py (closed-form cavity modes, the 2x2 lossy-mode recurrence,
exact discrete energy, Courant blow-up, mirror symmetry, graph = stencil,
adjoint dot-product and finite differences; the edge-weight reverse mode by
finite differences in single weights and by its chain to the eps_r gradient).  The CPML profile choice itself has
no closed form; it is checked by a reflection bound against an enlarged domain.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_LIB = None

CPML_M = 3.0          # polynomial grading order
CPML_ALPHA_MAX = 0.05  # S/m, at the inner interface
CPML_KAPPA_MAX = 1.0

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        _LIB = C.CDLL(path)
        L = _LIB
        L.or_mu0.restype = C.c_double
        L.or_eps0.restype = C.c_double
        L.or_c0.restype = C.c_double
        L.or2_energy.restype = C.c_double
        L.or3_energy.restype = C.c_double
        L.or2_graph_nodes.restype = C.c_int64
        L.or2_graph_layer.restype = C.c_int64
        L.or2_node_index.restype = C.c_int64
        L.or_coeffs_e.argtypes = [C.c_int64, _dp, _dp, C.c_double, _dp, _dp]
        L.or_cpml_axis.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_double] + [_dp] * 6
        L.or_waveform.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int64, _dp]
    return _LIB


def mu0() -> float:
    return lib().or_mu0()


def eps0() -> float:
    return lib().or_eps0()


def c0() -> float:
    return lib().or_c0()


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(n: int) -> None:
    """OpenMP threads of later calls (the loop bodies and results are unchanged)."""
    lib().or_set_threads(int(n))


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _ip_(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def coeffs_e(eps_r, sigma, dt):
    eps_r = np.ascontiguousarray(eps_r, np.float64)
    sigma = np.ascontiguousarray(sigma, np.float64)
    ca = np.empty_like(eps_r)
    cb = np.empty_like(eps_r)
    lib().or_coeffs_e(eps_r.size, _p(eps_r), _p(sigma), dt, _p(ca), _p(cb))
    return ca, cb


def cpml_axis(n, npml, delta, dt, m=CPML_M, alpha_max=CPML_ALPHA_MAX, kappa_max=CPML_KAPPA_MAX):
    arrs = [np.zeros(n, np.float64) for _ in range(6)]
    lib().or_cpml_axis(n, npml, delta, dt, m, alpha_max, kappa_max, *[_p(a) for a in arrs])
    return dict(zip(["bE", "cE", "kE", "bH", "cH", "kH"], arrs))


_WAVE_KIND = {"ricker": 0, "gauss_mod": 1, "gauss": 2, "sine": 3}


def waveform(kind: str, param: float, dt: float, nsteps: int) -> np.ndarray:
    out = np.zeros(nsteps, np.float64)
    lib().or_waveform(_WAVE_KIND[kind], param, dt, nsteps, _p(out))
    return out


def source_samples(src, dt, nsteps) -> np.ndarray:
    if src.kind == "sampled":
        s = np.zeros(nsteps, np.float64)
        m = min(nsteps, len(src.samples))
        s[:m] = np.asarray(src.samples, np.float64)[:m]
        return s
    return waveform(src.kind, src.params[0], dt, nsteps)


# ---------------------------------------------------------------------------------
# 2D TMz
# ---------------------------------------------------------------------------------

class _P2(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dt", C.c_double), ("ca", _dp), ("cb", _dp)] + \
               [(n, _dp) for n in ("bex", "cex", "kex", "bhx", "chx", "khx",
                                   "bey", "cey", "key", "bhy", "chy", "khy")] + \
               [("src_i", C.c_int), ("src_j", C.c_int), ("src", _dp), ("src_len", C.c_int64), ("src_nj", C.c_int)]


class _S2(C.Structure):
    _fields_ = [(n, _dp) for n in ("ez", "hx", "hy", "pezx", "pezy", "phxy", "phyx")]


class _M2(C.Structure):
    _fields_ = [("n_samp", C.c_int), ("si", _ip), ("sj", _ip), ("scomp", _ip), ("samp", _dp),
                ("n_dft", C.c_int), ("di", _ip), ("dj", _ip), ("n_freq", C.c_int),
                ("freq", _dp), ("dre", _dp), ("dim", _dp)]


_S2_NAMES = ("ez", "hx", "hy", "pezx", "pezy", "phxy", "phyx")
_COMP2 = {"ez": 0, "hx": 1, "hy": 2}


class TMz:
    """FP64 2D TMz run over a Scene2D (or explicit grid parameters).

    eps_cell / sigma_cell override the per-cell material (default: the scene's
    material map and table, with the scene's design region written in)."""

    def __init__(self, scene=None, *, nx=None, ny=None, dx=None, dy=None, dt=None, npml=0,
                 eps_cell=None, sigma_cell=None, source=None, nsteps_src=None, with_source=True):
        if scene is not None:
            nx, ny, dx, dy, dt, npml = scene.nx, scene.ny, scene.dx, scene.dy, scene.dt, scene.npml
            if eps_cell is None:
                eps_cell = scene.eps_r[scene.mat].astype(np.float64)
                if scene.design is not None:
                    i0, j0, w, h = scene.design
                    eps_cell[j0:j0 + h, i0:i0 + w] = scene.design_eps
            if sigma_cell is None:
                sigma_cell = scene.sigma[scene.mat].astype(np.float64)
            if source is None and with_source:
                source = scene.source
            if nsteps_src is None:
                nsteps_src = scene.nsteps
        self.nx, self.ny, self.dx, self.dy, self.dt, self.npml = nx, ny, dx, dy, dt, npml
        if eps_cell is None:
            eps_cell = np.ones((ny, nx))
        if sigma_cell is None:
            sigma_cell = np.zeros((ny, nx))
        self.eps_cell = np.ascontiguousarray(eps_cell, np.float64)
        self.sigma_cell = np.ascontiguousarray(sigma_cell, np.float64)
        self.ca, self.cb = coeffs_e(self.eps_cell, self.sigma_cell, dt)
        self.px = cpml_axis(nx, npml, dx, dt)
        self.py = cpml_axis(ny, npml, dy, dt)
        self.state = {k: np.zeros((ny, nx), np.float64) for k in _S2_NAMES}
        self.n = 0
        self.source = source if with_source else None
        self.src = None
        if self.source is not None:
            self.src = source_samples(self.source, dt, nsteps_src or 0)
        self._build_structs()

    def _build_structs(self):
        p = _P2()
        p.nx, p.ny, p.dx, p.dy, p.dt = self.nx, self.ny, self.dx, self.dy, self.dt
        p.ca, p.cb = _p(self.ca), _p(self.cb)
        for ax, prof in (("x", self.px), ("y", self.py)):
            for k in ("bE", "cE", "kE", "bH", "cH", "kH"):
                setattr(p, k[0] + k[1].lower() + ax, _p(prof[k]))
        if self.source is not None and self.src is not None:
            p.src_i, p.src_j = self.source.i, self.source.j
            p.src, p.src_len = _p(self.src), len(self.src)
            p.src_nj = getattr(self.source, "length", 1)
        else:
            p.src_i, p.src_j, p.src, p.src_len, p.src_nj = -1, -1, None, 0, 0
        self._p = p
        self._bind_state()

    def _bind_state(self):
        s = _S2()
        for k in _S2_NAMES:
            setattr(s, k, _p(self.state[k]))
        self._s = s

    def set_state(self, **fields):
        for k, v in fields.items():
            self.state[k][...] = v
        self._bind_state()

    def run(self, nsteps, samples=None, dft_cells=None, freqs=None):
        """Advance nsteps.  samples: list of (i, j, comp) -> [nsteps, n] values after
        each step; dft_cells + freqs: running DFT of Ez (accumulated in self.dft)."""
        m = _M2()
        keep = []
        out = {}
        if samples is not None and len(samples):
            si = np.array([s[0] for s in samples], np.int32)
            sj = np.array([s[1] for s in samples], np.int32)
            sc = np.array([_COMP2[s[2]] if isinstance(s[2], str) else s[2] for s in samples], np.int32)
            buf = np.zeros((nsteps, len(samples)), np.float64)
            keep += [si, sj, sc]
            m.n_samp, m.si, m.sj, m.scomp, m.samp = len(samples), _ip_(si), _ip_(sj), _ip_(sc), _p(buf)
            out["samples"] = buf
        if dft_cells is not None and len(dft_cells):
            di = np.ascontiguousarray(np.asarray(dft_cells)[:, 0], np.int32)
            dj = np.ascontiguousarray(np.asarray(dft_cells)[:, 1], np.int32)
            fr = np.ascontiguousarray(freqs, np.float64)
            if not hasattr(self, "dft") or self.dft[0].shape != (len(di), len(fr)):
                self.dft = (np.zeros((len(di), len(fr))), np.zeros((len(di), len(fr))))
            keep += [di, dj, fr]
            m.n_dft, m.di, m.dj, m.n_freq, m.freq = len(di), _ip_(di), _ip_(dj), len(fr), _p(fr)
            m.dre, m.dim = _p(self.dft[0]), _p(self.dft[1])
        lib().or2_run(C.byref(self._p), C.byref(self._s), C.c_int64(self.n), C.c_int64(nsteps),
                      C.byref(m))
        self.n += nsteps
        return out

    def layer_h(self):
        lib().or2_layer_h(C.byref(self._p), C.byref(self._s))

    def layer_e(self):
        lib().or2_layer_e(C.byref(self._p), C.byref(self._s))

    def energy(self, hx_prev, hy_prev):
        hx_prev = np.ascontiguousarray(hx_prev, np.float64)
        hy_prev = np.ascontiguousarray(hy_prev, np.float64)
        return lib().or2_energy(C.byref(self._p), _p(self.eps_cell), C.byref(self._s),
                                _p(hx_prev), _p(hy_prev))

    # ---- literal graph (Prop. 1 / Prop. 2) ----
    def graph_nodes(self) -> int:
        return lib().or2_graph_nodes(C.byref(self._p))

    def node_index(self, kind, i, j) -> int:
        k = {"t": 0, "ez": 0, "u": 1, "hx": 1, "q": 2, "hy": 2}[kind]
        return lib().or2_node_index(C.byref(self._p), k, i, j)

    def graph_layer(self, layer):
        n = self.graph_nodes()
        nnz = lib().or2_graph_layer(C.byref(self._p), layer, None, None, None)
        rowptr = np.zeros(n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        w = np.zeros(nnz, np.float64)
        lib().or2_graph_layer(C.byref(self._p), layer, rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                              col.ctypes.data_as(C.POINTER(C.c_int32)), _p(w))
        return rowptr, col, w

    def to_nodes(self) -> np.ndarray:
        h = np.zeros(self.graph_nodes(), np.float64)
        lib().or2_state_to_nodes(C.byref(self._p), C.byref(self._s), _p(h))
        return h

    def from_nodes(self, h):
        h = np.ascontiguousarray(h, np.float64)
        lib().or2_nodes_to_state(C.byref(self._p), _p(h), C.byref(self._s))

    @staticmethod
    def csr_mv(rowptr, col, w, x):
        y = np.zeros(len(rowptr) - 1, np.float64)
        x = np.ascontiguousarray(x, np.float64)
        lib().or_csr_mv(C.c_int64(len(y)), rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                        col.ctypes.data_as(C.POINTER(C.c_int32)), _p(w), _p(x), _p(y))
        return y

    @staticmethod
    def csr_mtv(rowptr, col, w, x):
        y = np.zeros(len(rowptr) - 1, np.float64)
        x = np.ascontiguousarray(x, np.float64)
        lib().or_csr_mtv(C.c_int64(len(y)), rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                         col.ctypes.data_as(C.POINTER(C.c_int32)), _p(w), _p(x), _p(y))
        return y

    # ---- reverse mode ----
    def adjoint_step(self, adj: dict):
        """In-place adjoint of one forward step (no source, no loss) on a dict of
        arrays with the state's names."""
        s = _S2()
        arrs = {k: np.ascontiguousarray(adj[k], np.float64) for k in _S2_NAMES}
        for k in _S2_NAMES:
            setattr(s, k, _p(arrs[k]))
        lib().or2_adjoint_step(C.byref(self._p), C.byref(s))
        for k in _S2_NAMES:
            adj[k][...] = arrs[k]
        return adj

    def adjoint_grad(self, nsteps, ckpt, monitors, freqs, design):
        """dL/deps_r over design = (i0, j0, w, h) for L = sum |F|^2 (DFT of Ez at
        the monitor cells).  Returns (loss, F_re, F_im, grad[h, w])."""
        i0, j0, w, h = design
        mi = np.ascontiguousarray(np.asarray(monitors)[:, 0], np.int32)
        mj = np.ascontiguousarray(np.asarray(monitors)[:, 1], np.int32)
        fr = np.ascontiguousarray(freqs, np.float64)
        fre = np.zeros((len(mi), len(fr)))
        fim = np.zeros((len(mi), len(fr)))
        grad = np.zeros((h, w))
        loss = C.c_double(0.0)
        rc = lib().or2_adjoint_grad(C.byref(self._p), _p(self.eps_cell), _p(self.sigma_cell),
                                    C.c_int64(nsteps), C.c_int64(ckpt), len(mi), _ip_(mi), _ip_(mj),
                                    len(fr), _p(fr), i0, j0, w, h, C.byref(loss), _p(fre), _p(fim),
                                    _p(grad))
        if rc != 0:
            raise RuntimeError(f"or2_adjoint_grad failed ({rc})")
        return loss.value, fre, fim, grad


    # ---- learnable edge weights: reverse mode over the literal graph ----
    # The 11 weights a cell (i, j) owns as a destination (Prop. 1, TMz naming),
    # as (layer, destination kind, source kind, di, dj of the source).
    EDGE_CLASSES = (
        (2, "t", "t", 0, 0),    # Ez <- Ez        Ca            (eq. 7)
        (2, "t", "q", 0, 0),    # Ez <- Hy(i)     +Cb/dx
        (2, "t", "q", -1, 0),   # Ez <- Hy(i-1)   -Cb/dx
        (2, "t", "u", 0, 0),    # Ez <- Hx(j)     -Cb/dy
        (2, "t", "u", 0, -1),   # Ez <- Hx(j-1)   +Cb/dy
        (1, "u", "u", 0, 0),    # Hx <- Hx        1             (eq. 8)
        (1, "u", "t", 0, 1),    # Hx <- Ez(j+1)   -Db/dy
        (1, "u", "t", 0, 0),    # Hx <- Ez(j)     +Db/dy
        (1, "q", "q", 0, 0),    # Hy <- Hy        1             (eq. 9)
        (1, "q", "t", 1, 0),    # Hy <- Ez(i+1)   +Db/dx
        (1, "q", "t", 0, 0),    # Hy <- Ez(i)     -Db/dx
    )

    def source_nodes(self):
        """Electric nodes that receive the soft source (one per cell of a line)."""
        if self.source is None or self.src is None:
            return np.zeros(0, np.int64)
        nj = max(1, getattr(self.source, "length", 1))
        return np.array([self.node_index("t", self.source.i, self.source.j + q) for q in range(nj)], np.int64)

    def graph_forward(self, nsteps, layers=None, monitors=None, freqs=None, keep=False):
        """nsteps of Prop. 2 on node values, from the current state: h <- W2 (W1 h),
        then the soft source s[n] on the source's electric nodes and the running
        DFT F(f) += Ez^{n+1} exp(-i 2 pi f (n+1) dt) dt at the monitor cells.
        layers: ((rowptr, col, w) of layer 1, of layer 2), default graph_layer.
        Returns (h, F [n_mon, n_freq] complex, [h^n before each step] if keep).
        Does not change self.state."""
        W1, W2 = layers if layers is not None else (self.graph_layer(1), self.graph_layer(2))
        h = self.to_nodes()
        tm = np.array([self.node_index("t", int(i), int(j)) for i, j in monitors], np.int64) \
            if monitors is not None else np.zeros(0, np.int64)
        fr = np.asarray(freqs if freqs is not None else [], np.float64)
        F = np.zeros((len(tm), len(fr)), np.complex128)
        ts = self.source_nodes()
        hist = []
        for k in range(nsteps):
            n = self.n + k
            if keep:
                hist.append(h)
            h = TMz.csr_mv(*W2, TMz.csr_mv(*W1, h))
            if len(ts) and n < len(self.src):
                h[ts] += self.src[n]
            if len(tm):
                F += h[tm][:, None] * np.exp(-2j * np.pi * fr[None, :] * ((n + 1) * self.dt)) * self.dt
        return h, F, hist

    def graph_edge_grad(self, nsteps, monitors, freqs, dLdF_re, dLdF_im):
        """Reverse mode of graph_forward for the linear loss
        L = sum_{m,f} dLdF_re[m,f] Re F[m,f] + dLdF_im[m,f] Im F[m,f]:
        dL/dw for every edge of both layers, in the CSR order of graph_layer.
        With lam the adjoint of the node vector after step n, the layers are
        reversed newest first: dL/dw2[e] += lam[dst] h1^n[src], lam1 = W2^T lam,
        dL/dw1[e] += lam1[dst] h^n[src], lam = W1^T lam1; dL/dEz^n at the monitors
        is dt sum_f (dLdF_re cos(2 pi f n dt) - dLdF_im sin(2 pi f n dt)).
        Returns (g1, g2, F)."""
        W1, W2 = self.graph_layer(1), self.graph_layer(2)
        nn = len(W1[0]) - 1
        dst1 = np.repeat(np.arange(nn), np.diff(W1[0]))
        dst2 = np.repeat(np.arange(nn), np.diff(W2[0]))
        _, F, hist = self.graph_forward(nsteps, (W1, W2), monitors, freqs, keep=True)
        tm = np.array([self.node_index("t", int(i), int(j)) for i, j in monitors], np.int64)
        fr = np.asarray(freqs, np.float64)
        a = np.asarray(dLdF_re, np.float64).reshape(len(tm), len(fr))
        b = np.asarray(dLdF_im, np.float64).reshape(len(tm), len(fr))
        g1 = np.zeros(len(W1[2]))
        g2 = np.zeros(len(W2[2]))
        lam = np.zeros(nn)
        for k in range(nsteps - 1, -1, -1):
            ph = 2 * np.pi * fr * ((self.n + k + 1) * self.dt)
            np.add.at(lam, tm, self.dt * (a @ np.cos(ph) - b @ np.sin(ph)))
            h0 = hist[k]
            h1 = TMz.csr_mv(*W1, h0)
            g2 += lam[dst2] * h1[W2[1]]
            lam1 = TMz.csr_mtv(*W2, lam)
            g1 += lam1[dst1] * h0[W1[1]]
            lam = TMz.csr_mtv(*W1, lam1)
        return g1, g2, F

    def edge_class_grad(self, g1, g2, design):
        """The 11 per-cell edge classes (EDGE_CLASSES) of the cells of design =
        (i0, j0, w, h), picked out of per-edge gradients in CSR order:
        [11, h, w]."""
        i0, j0, w, h = design
        lay = {1: (self.graph_layer(1), g1), 2: (self.graph_layer(2), g2)}
        out = np.zeros((len(self.EDGE_CLASSES), h, w))
        for ci, (layer, kd, ks, di, dj) in enumerate(self.EDGE_CLASSES):
            (rowptr, col, _), g = lay[layer]
            for jj in range(h):
                for ii in range(w):
                    i, j = i0 + ii, j0 + jj
                    d = self.node_index(kd, i, j)
                    sidx = self.node_index(ks, i + di, j + dj)
                    row = np.arange(rowptr[d], rowptr[d + 1])
                    hit = row[col[row] == sidx]
                    if len(hit) != 1:
                        raise ValueError(f"edge class {ci} missing at ({i}, {j})")
                    out[ci, jj, ii] = g[hit[0]]
        return out


# ---------------------------------------------------------------------------------
# 2D TMz with the paper's split-field PML (split_pml.c)
# ---------------------------------------------------------------------------------

class _P2S(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dt", C.c_double), ("eps_cell", _dp), ("sig_cell", _dp), ("sxe", _dp), ("sxh", _dp),
                ("sye", _dp), ("syh", _dp), ("src_i", C.c_int), ("src_j", C.c_int), ("src", _dp),
                ("src_len", C.c_int64), ("src_nj", C.c_int)]


class _S2S(C.Structure):
    _fields_ = [(n, _dp) for n in ("ezx", "ezy", "hx", "hy")]


def split_axis(n, npml, delta, m=3.0):
    """Berenger layer conductivity (S/m) at the E nodes and H nodes of one axis."""
    sE = np.zeros(n)
    sH = np.zeros(n)
    lib().or_split_axis(int(n), int(npml), C.c_double(delta), C.c_double(m), _p(sE), _p(sH))
    return sE, sH


class TMzSplit:
    """FP64 2D TMz run with the paper's split-field PML (Berenger, Sec. III-C):
    the scene's npml cells on every side form the graded layer.  State: ezx,
    ezy, hx, hy; self.ez() is their Ez = Ezx + Ezy."""

    def __init__(self, scene, *, nsteps_src=None, eps_cell=None, sigma_cell=None, m=3.0):
        self.nx, self.ny, self.dx, self.dy, self.dt = scene.nx, scene.ny, scene.dx, scene.dy, scene.dt
        self.npml = scene.npml
        if eps_cell is None:
            eps_cell = scene.eps_r[scene.mat].astype(np.float64)
            if scene.design is not None:
                i0, j0, w, h = scene.design
                eps_cell[j0:j0 + h, i0:i0 + w] = scene.design_eps
        if sigma_cell is None:
            sigma_cell = scene.sigma[scene.mat].astype(np.float64)
        self.eps_cell = np.ascontiguousarray(eps_cell, np.float64)
        self.sigma_cell = np.ascontiguousarray(sigma_cell, np.float64)
        self.sxe, self.sxh = split_axis(self.nx, self.npml, self.dx, m)
        self.sye, self.syh = split_axis(self.ny, self.npml, self.dy, m)
        self.state = {k: np.zeros((self.ny, self.nx), np.float64) for k in ("ezx", "ezy", "hx", "hy")}
        self.source = scene.source
        self.src = source_samples(scene.source, self.dt, nsteps_src or scene.nsteps) if scene.source else None
        self.n = 0
        p = _P2S()
        p.nx, p.ny, p.dx, p.dy, p.dt = self.nx, self.ny, self.dx, self.dy, self.dt
        p.eps_cell, p.sig_cell = _p(self.eps_cell), _p(self.sigma_cell)
        p.sxe, p.sxh, p.sye, p.syh = _p(self.sxe), _p(self.sxh), _p(self.sye), _p(self.syh)
        if self.src is not None:
            p.src_i, p.src_j, p.src, p.src_len = self.source.i, self.source.j, _p(self.src), len(self.src)
            p.src_nj = getattr(self.source, "length", 1)
        else:
            p.src_i, p.src_j, p.src, p.src_len, p.src_nj = -1, -1, None, 0, 0
        self._p = p
        self._bind()

    def _bind(self):
        s = _S2S()
        for k in ("ezx", "ezy", "hx", "hy"):
            setattr(s, k, _p(self.state[k]))
        self._s = s

    def ez(self):
        return self.state["ezx"] + self.state["ezy"]

    def run(self, nsteps, samples=None, dft_cells=None, freqs=None):
        """As TMz.run; samples and the DFT see Ez = Ezx + Ezy."""
        m = _M2()
        keep = []
        out = {}
        if samples is not None and len(samples):
            si = np.array([q[0] for q in samples], np.int32)
            sj = np.array([q[1] for q in samples], np.int32)
            sc = np.array([_COMP2[q[2]] if isinstance(q[2], str) else q[2] for q in samples], np.int32)
            buf = np.zeros((nsteps, len(samples)), np.float64)
            keep += [si, sj, sc]
            m.n_samp, m.si, m.sj, m.scomp, m.samp = len(samples), _ip_(si), _ip_(sj), _ip_(sc), _p(buf)
            out["samples"] = buf
        if dft_cells is not None and len(dft_cells):
            di = np.ascontiguousarray(np.asarray(dft_cells)[:, 0], np.int32)
            dj = np.ascontiguousarray(np.asarray(dft_cells)[:, 1], np.int32)
            fr = np.ascontiguousarray(freqs, np.float64)
            if not hasattr(self, "dft") or self.dft[0].shape != (len(di), len(fr)):
                self.dft = (np.zeros((len(di), len(fr))), np.zeros((len(di), len(fr))))
            keep += [di, dj, fr]
            m.n_dft, m.di, m.dj, m.n_freq, m.freq = len(di), _ip_(di), _ip_(dj), len(fr), _p(fr)
            m.dre, m.dim = _p(self.dft[0]), _p(self.dft[1])
        lib().or2s_run(C.byref(self._p), C.byref(self._s), C.c_int64(self.n), C.c_int64(nsteps), C.byref(m))
        self.n += nsteps
        return out

    def set_state(self, **fields):
        for k, v in fields.items():
            self.state[k][...] = v
        self._bind()

    def layer_h(self):
        lib().or2s_layer_h(C.byref(self._p), C.byref(self._s))

    def layer_e(self):
        lib().or2s_layer_e(C.byref(self._p), C.byref(self._s))

    # ---- literal 4-node graph (Sec. IV-B) ----
    def node_index(self, kind, i, j) -> int:
        k = {"u": 0, "hx": 0, "q": 1, "hy": 1, "tx": 2, "ezx": 2, "tz": 3, "ezy": 3}[kind]
        return lib().or2s_node_index(self.nx, k, i, j)

    def graph_layer(self, layer):
        n = 4 * self.nx * self.ny
        nnz = lib().or2s_graph_layer(C.byref(self._p), layer, None, None, None)
        rowptr = np.zeros(n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        w = np.zeros(nnz, np.float64)
        lib().or2s_graph_layer(C.byref(self._p), layer, rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                               col.ctypes.data_as(C.POINTER(C.c_int32)), _p(w))
        return rowptr, col, w

    def to_nodes(self) -> np.ndarray:
        h = np.zeros(4 * self.nx * self.ny, np.float64)
        lib().or2s_state_to_nodes(C.byref(self._p), C.byref(self._s), _p(h))
        return h

    def from_nodes(self, h):
        h = np.ascontiguousarray(h, np.float64)
        lib().or2s_nodes_to_state(C.byref(self._p), _p(h), C.byref(self._s))


# ---------------------------------------------------------------------------------
# 3D Yee
# ---------------------------------------------------------------------------------

class _P3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double), ("ca", _dp),
                ("cb", _dp)] + \
               [(n, _dp) for ax in ("x", "y", "z") for n in
                ("be" + ax, "ce" + ax, "ke" + ax, "bh" + ax, "ch" + ax, "kh" + ax)] + \
               [("src_i", C.c_int), ("src_j", C.c_int), ("src_k", C.c_int), ("src_comp", C.c_int),
                ("src", _dp), ("src_len", C.c_int64)]


_S3_NAMES = ("ex", "ey", "ez", "hx", "hy", "hz", "pexy", "pexz", "peyz", "peyx", "pezx", "pezy",
             "phxy", "phxz", "phyz", "phyx", "phzx", "phzy")


class _S3(C.Structure):
    _fields_ = [(n, _dp) for n in _S3_NAMES]


class _M3(C.Structure):
    _fields_ = [("n_samp", C.c_int), ("si", _ip), ("sj", _ip), ("sk", _ip), ("scomp", _ip),
                ("samp", _dp), ("plane_k", C.c_int), ("n_pc", C.c_int), ("pcomp", _ip),
                ("n_freq", C.c_int), ("freq", _dp), ("pre", _dp), ("pim", _dp)]


_COMP3 = {"ex": 0, "ey": 1, "ez": 2, "hx": 3, "hy": 4, "hz": 5}


class Yee3D:
    """FP64 3D Yee run over a Scene3D (or explicit parameters)."""

    def __init__(self, scene=None, *, nx=None, ny=None, nz=None, dx=None, dy=None, dz=None,
                 dt=None, npml=0, eps_cell=None, sigma_cell=None, source=None, nsteps_src=None,
                 with_source=True):
        if scene is not None:
            nx, ny, nz = scene.nx, scene.ny, scene.nz
            dx, dy, dz, dt, npml = scene.dx, scene.dy, scene.dz, scene.dt, scene.npml
            if eps_cell is None:
                eps_cell = scene.eps_r[scene.mat]
            if sigma_cell is None:
                sigma_cell = scene.sigma[scene.mat]
            if source is None and with_source:
                source = scene.source
            if nsteps_src is None:
                nsteps_src = scene.nsteps
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dx, self.dy, self.dz, self.dt, self.npml = dx, dy, dz, dt, npml
        shape = (nz, ny, nx)
        self.eps_cell = np.ascontiguousarray(np.ones(shape) if eps_cell is None else eps_cell, np.float64)
        self.sigma_cell = np.ascontiguousarray(np.zeros(shape) if sigma_cell is None else sigma_cell,
                                               np.float64)
        self.ca, self.cb = coeffs_e(self.eps_cell, self.sigma_cell, dt)
        self.prof = {"x": cpml_axis(nx, npml, dx, dt), "y": cpml_axis(ny, npml, dy, dt),
                     "z": cpml_axis(nz, npml, dz, dt)}
        self.state = {k: np.zeros(shape, np.float64) for k in _S3_NAMES}
        self.n = 0
        self.source = source if with_source else None
        self.src = source_samples(source, dt, nsteps_src or 0) if self.source is not None else None
        p = _P3()
        p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, p.dt = nx, ny, nz, dx, dy, dz, dt
        p.ca, p.cb = _p(self.ca), _p(self.cb)
        for ax in ("x", "y", "z"):
            for k in ("bE", "cE", "kE", "bH", "cH", "kH"):
                setattr(p, k[0] + k[1].lower() + ax, _p(self.prof[ax][k]))
        if self.source is not None:
            p.src_i, p.src_j, p.src_k = self.source.i, self.source.j, self.source.k
            p.src_comp = _COMP3[self.source.component]
            p.src, p.src_len = _p(self.src), len(self.src)
        else:
            p.src_i = p.src_j = p.src_k = -1
            p.src_comp, p.src, p.src_len = 2, None, 0
        self._p = p
        self._bind_state()

    def _bind_state(self):
        s = _S3()
        for k in _S3_NAMES:
            setattr(s, k, _p(self.state[k]))
        self._s = s

    def set_state(self, **fields):
        for k, v in fields.items():
            self.state[k][...] = v
        self._bind_state()

    def run(self, nsteps, samples=None, plane_k=-1, plane_comps=("ex", "ey", "ez"), freqs=None):
        m = _M3()
        keep = []
        out = {}
        if samples is not None and len(samples):
            cols = [np.array([s[a] for s in samples], np.int32) for a in range(3)]
            sc = np.array([_COMP3[s[3]] for s in samples], np.int32)
            buf = np.zeros((nsteps, len(samples)))
            keep += cols + [sc]
            m.n_samp, m.si, m.sj, m.sk = len(samples), _ip_(cols[0]), _ip_(cols[1]), _ip_(cols[2])
            m.scomp, m.samp = _ip_(sc), _p(buf)
            out["samples"] = buf
        m.plane_k = -1
        if plane_k >= 0 and freqs is not None:
            pc = np.array([_COMP3[c] for c in plane_comps], np.int32)
            fr = np.ascontiguousarray(freqs, np.float64)
            shape = (len(pc), len(fr), self.ny, self.nx)
            if not hasattr(self, "plane") or self.plane[0].shape != shape:
                self.plane = (np.zeros(shape), np.zeros(shape))
            keep += [pc, fr]
            m.plane_k, m.n_pc, m.pcomp, m.n_freq, m.freq = plane_k, len(pc), _ip_(pc), len(fr), _p(fr)
            m.pre, m.pim = _p(self.plane[0]), _p(self.plane[1])
        lib().or3_run(C.byref(self._p), C.byref(self._s), C.c_int64(self.n), C.c_int64(nsteps),
                      C.byref(m))
        self.n += nsteps
        return out

    def energy(self, hx_prev, hy_prev, hz_prev):
        a = [np.ascontiguousarray(x, np.float64) for x in (hx_prev, hy_prev, hz_prev)]
        return lib().or3_energy(C.byref(self._p), _p(self.eps_cell), C.byref(self._s),
                                *[_p(x) for x in a])

