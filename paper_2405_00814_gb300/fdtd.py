"""Thin ctypes binding of the C ABI in include/gem_fdtd.h.

Argument marshalling only: every step of the time loop runs in the sm_103a
kernels of libgemfdtd.so.  There is no fallback: if the library has not been
built, importing works but creating a Simulation raises.
PyTorch, when used, only supplies device buffers (``get_field(out=tensor)``)
and the CUDA stream the work is ordered on.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgemfdtd.so")
_LIB = None

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
PEC, CPML, SPLIT_PML = 0, 1, 2
COMP = {"ex": 0, "ey": 1, "ez": 2, "hx": 3, "hy": 4, "hz": 5}
SRC = {"ricker": 0, "gauss_mod": 1, "gauss": 2, "sampled": 3, "sine": 4}
OPT = {"kernel": 0, "tblock": 1, "segment": 2, "warps": 3, "graph": 4, "spin_limit": 5, "debug_stall_item": 6,
       "adj_store": 7, "segment_b": 8, "check_every": 9, "taper": 10,
       "warps_b": 11, "playout": 12, "bulk": 13}


class FDTDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("dims", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("pml_cells", C.c_int), ("boundary", C.c_int), ("dy", C.c_double), ("dz", C.c_double)]


class Material(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("mu_r", C.c_double), ("sigma", C.c_double)]


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        vp, i64, dp, fp, ip = C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.c_void_p, C.c_int
        L.fdtd_create.argtypes = [C.POINTER(Grid), C.c_double, C.c_double, C.c_double, vp,
                                  C.POINTER(Material), ip, vp, C.POINTER(vp)]
        L.fdtd_create_batch.argtypes = [ip, C.POINTER(Grid), dp, dp, C.POINTER(vp),
                                        C.POINTER(C.POINTER(Material)), C.POINTER(C.c_int), vp, C.POINTER(vp)]
        L.fdtd_select_scene.argtypes = [vp, ip]
        L.fdtd_num_scenes.argtypes = [vp]
        L.fdtd_destroy.argtypes = [vp]
        L.fdtd_destroy.restype = None
        L.fdtd_last_error.argtypes = [vp]
        L.fdtd_last_error.restype = C.c_char_p
        L.fdtd_set_option.argtypes = [vp, ip, i64]
        L.fdtd_get_option.argtypes = [vp, ip]
        L.fdtd_get_option.restype = i64
        L.fdtd_set_source.argtypes = [vp, ip, ip, ip, ip, ip, dp, vp, i64]
        L.fdtd_set_line_source.argtypes = [vp, ip, ip, ip, ip, dp, vp, i64]
        L.fdtd_set_design.argtypes = [vp, ip, ip, ip, ip, vp, vp, ip]
        L.fdtd_set_materials.argtypes = [vp, vp, vp, ip]
        L.fdtd_add_probe.argtypes = [vp, ip, ip, ip, ip, C.POINTER(C.c_int)]
        L.fdtd_add_dft_monitor.argtypes = [vp, vp, ip, dp, ip, C.POINTER(C.c_int)]
        L.fdtd_add_dft_plane.argtypes = [vp, ip, ip, dp, ip, C.POINTER(C.c_int)]
        L.fdtd_step.argtypes = [vp, i64]
        L.fdtd_step_edgelist.argtypes = [vp, i64]
        L.fdtd_export_graph.argtypes = [vp, ip, C.POINTER(i64), C.POINTER(i64), vp, vp, vp]
        L.fdtd_read_probe.argtypes = [vp, ip, fp, i64]
        L.fdtd_read_dft.argtypes = [vp, ip, fp, fp]
        L.fdtd_get_field.argtypes = [vp, ip, vp, ip]
        L.fdtd_set_field.argtypes = [vp, ip, vp, ip]
        L.fdtd_reset.argtypes = [vp]
        L.fdtd_time_step.argtypes = [vp]
        L.fdtd_time_step.restype = i64
        L.fdtd_launch_count.argtypes = [vp]
        L.fdtd_launch_count.restype = i64
        L.fdtd_save_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.fdtd_load_state.argtypes = [vp, vp, C.c_size_t]
        L.fdtd_check_finite.argtypes = [vp]
        L.fdtd_sync.argtypes = [vp]
        L.fdtd_autotune.argtypes = [vp, ip, C.POINTER(C.c_double)]
        L.fdtd_set_checkpointing.argtypes = [vp, ip]
        L.fdtd_adjoint_grad.argtypes = [vp, vp, vp, vp, ip]
        L.fdtd_edge_grad.argtypes = [vp, vp, vp, vp, ip]
        L.fdtd_mp_steps_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, i64, vp]
        L.fdtd_create_slab.argtypes = [C.POINTER(Grid), ip, ip, ip, C.c_double, C.c_double, C.c_double, vp,
                                       C.POINTER(Material), ip, vp, C.POINTER(vp)]
        L.fdtd_halo_count.argtypes = [vp]
        L.fdtd_halo_count.restype = i64
        L.fdtd_halo_export.argtypes = [vp, ip, vp, ip]
        L.fdtd_halo_import.argtypes = [vp, ip, vp, ip]
        L.fdtd_slab_rows.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        _LIB = L
    return _LIB


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    h = getattr(stream, "cuda_stream", None)
    if h is not None:
        return h or None
    raise TypeError("stream must be None, an int handle or a torch.cuda.Stream")


def _mat_table(eps_r, sigma):
    n = len(eps_r)
    tab = (Material * n)()
    for k in range(n):
        tab[k].eps_r, tab[k].mu_r, tab[k].sigma = float(eps_r[k]), 1.0, float(sigma[k])
    return tab


def _grid_of(scene, boundary=None):
    """boundary: None (CPML when the scene has a layer, else PEC), "cpml",
    "split" (the paper's split-field PML) or "pec"."""
    g = Grid()
    if hasattr(scene, "nz"):
        g.dims, g.nx, g.ny, g.nz = 3, scene.nx, scene.ny, scene.nz
        g.dz = scene.dz
    else:
        g.dims, g.nx, g.ny, g.nz = 2, scene.nx, scene.ny, 1
        g.dz = 0.0
    g.pml_cells = scene.npml
    if boundary is None:
        g.boundary = CPML if scene.npml > 0 else PEC
    else:
        g.boundary = {"pec": PEC, "cpml": CPML, "split": SPLIT_PML}[boundary]
    g.dy = scene.dy
    return g


class Simulation:
    """One context of the C ABI: one scene, or a batch of 2D scenes."""

    def __init__(self, scene=None, *, stream=None, boundary=None, _handle=None):
        self._L = lib()
        self._h = None
        self.dims = 2
        self.shape = None           # (nx, ny, nz) of a single-scene context
        self.split = False
        self._cells = []            # cells of each scene, for the buffer-size checks
        self._sel = 0
        if _handle is not None:
            self._h = _handle
            return
        g = _grid_of(scene, boundary)
        self.dims = g.dims
        self.shape = (g.nx, g.ny, g.nz)
        self._cells = [g.nx * g.ny * g.nz]
        self.split = g.boundary == SPLIT_PML
        mat = np.ascontiguousarray(scene.mat, np.uint8)
        tab = _mat_table(scene.eps_r, scene.sigma)
        h = C.c_void_p()
        rc = self._L.fdtd_create(C.byref(g), scene.dx, scene.dt, 0.0, mat.ctypes.data, tab, len(scene.eps_r),
                                 _stream_handle(stream), C.byref(h))
        self._h = h
        self._check(rc)

    @classmethod
    def batch(cls, scenes, *, stream=None):
        L = lib()
        n = len(scenes)
        grids = (Grid * n)(*[_grid_of(s) for s in scenes])
        dx = (C.c_double * n)(*[s.dx for s in scenes])
        dt = (C.c_double * n)(*[s.dt for s in scenes])
        mats = [np.ascontiguousarray(s.mat, np.uint8) for s in scenes]
        mp = (C.c_void_p * n)(*[m.ctypes.data for m in mats])
        tabs = [_mat_table(s.eps_r, s.sigma) for s in scenes]
        tp = (C.POINTER(Material) * n)(*[C.cast(t, C.POINTER(Material)) for t in tabs])
        nm = (C.c_int * n)(*[len(s.eps_r) for s in scenes])
        h = C.c_void_p()
        rc = L.fdtd_create_batch(n, grids, dx, dt, mp, tp, nm, _stream_handle(stream), C.byref(h))
        sim = cls(_handle=h)
        sim._check(rc)
        sim._cells = [s.nx * s.ny for s in scenes]
        return sim

    @classmethod
    def slab(cls, scene, j0, j1, ghost, *, stream=None, boundary=None):
        """A y-slab sub-domain owning rows [j0, j1) of a 2D scene plus `ghost`
        rows on each side with a neighbour (fdtd_create_slab).  Local row r is
        scene row r + row_offset.  The scene's source is set when its cells fall
        in the local rows (in local coordinates); probes and monitors are left to
        the caller (on the slab that owns the cell)."""
        L = lib()
        g = _grid_of(scene, boundary)
        glo = ghost if j0 > 0 else 0
        ghi = ghost if j1 < scene.ny else 0
        lo, hi = max(0, j0 - glo), min(scene.ny, j1 + ghi)
        mat = np.ascontiguousarray(scene.mat[lo:hi], np.uint8)
        tab = _mat_table(scene.eps_r, scene.sigma)
        h = C.c_void_p()
        rc = L.fdtd_create_slab(C.byref(g), int(j0), int(j1), int(ghost), scene.dx, scene.dt, 0.0, mat.ctypes.data,
                                tab, len(scene.eps_r), _stream_handle(stream), C.byref(h))
        sim = cls(_handle=h)
        sim._check(rc)
        sim.shape = (scene.nx, hi - lo, 1)
        sim._cells = [scene.nx * (hi - lo)]
        sim.slab_rows = (j0, j1, lo)
        src = getattr(scene, "source", None)
        if src is not None:
            n = getattr(src, "length", 1)
            a, b = max(src.j, lo), min(src.j + n, hi)
            if a < b and not (a == 0 and lo == 0):
                if src.kind == "sampled":
                    sim.set_line_source("sampled", src.i, a - lo, b - lo, samples=src.samples)
                else:
                    sim.set_line_source(src.kind, src.i, a - lo, b - lo, param=src.params[0])
        return sim

    def halo_count(self) -> int:
        return int(self._L.fdtd_halo_count(self._h))

    def _halo_buf(self, buf):
        self._need(buf, self.halo_count(), "halo")
        if hasattr(buf, "data_ptr"):
            if buf.dtype.__str__() != "torch.float32":
                raise ValueError("halo buffers are float32")
            return buf.data_ptr(), 1 if buf.is_cuda else 0
        if not (isinstance(buf, np.ndarray) and buf.dtype == np.float32 and buf.flags.c_contiguous):
            raise ValueError("halo buffers are contiguous float32")
        return buf.ctypes.data, 0

    def halo_export(self, side: int, out):
        """The owned rows next to cut `side` (0 lower, 1 upper), packed
        [array][ghost][nx], into out (CUDA tensor, CPU tensor or numpy array)."""
        ptr, dev = self._halo_buf(out)
        self._check(self._L.fdtd_halo_export(self._h, int(side), ptr, dev))
        return out

    def halo_import(self, side: int, buf):
        """Overwrite the ghost rows beyond cut `side` from the neighbour's export."""
        ptr, dev = self._halo_buf(buf)
        self._check(self._L.fdtd_halo_import(self._h, int(side), ptr, dev))

    # ---------------------------------------------------------------- basics
    def _check(self, rc):
        if rc != OK:
            msg = self._L.fdtd_last_error(self._h).decode() if self._h else "creation failed"
            raise FDTDError(rc, msg)

    def close(self):
        if self._h:
            self._L.fdtd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def num_scenes(self) -> int:
        return self._L.fdtd_num_scenes(self._h)

    def select(self, scene: int):
        self._check(self._L.fdtd_select_scene(self._h, scene))
        self._sel = scene
        return self

    def _need(self, buf, n, what):
        """The library writes or reads exactly n float32 (or uint8) elements of buf:
        refuse a buffer of another size before it can overrun."""
        size = buf.numel() if hasattr(buf, "numel") else np.asarray(buf).size
        if size != n:
            raise ValueError(f"{what}: buffer holds {size} elements, the library uses {n}")
        if hasattr(buf, "is_contiguous") and not buf.is_contiguous():
            raise ValueError(f"{what}: the tensor must be contiguous")

    def _field_cells(self):
        return self._cells[self._sel] if self._sel < len(self._cells) else None

    def set_option(self, name: str, value: int):
        self._check(self._L.fdtd_set_option(self._h, OPT[name], int(value)))

    def get_option(self, name: str) -> int:
        return self._L.fdtd_get_option(self._h, OPT[name])

    @property
    def time_step(self) -> int:
        return self._L.fdtd_time_step(self._h)

    @property
    def launch_count(self) -> int:
        return self._L.fdtd_launch_count(self._h)

    # ---------------------------------------------------------------- inputs
    def set_source(self, kind, i, j, k=0, component="ez", param=None, samples=None):
        par = (C.c_double * 1)(float(param) if param is not None else 0.0)
        if samples is not None:
            smp = np.ascontiguousarray(samples, np.float32)
            rc = self._L.fdtd_set_source(self._h, SRC[kind], i, j, k, COMP[component], par, smp.ctypes.data,
                                         len(smp))
        else:
            rc = self._L.fdtd_set_source(self._h, SRC[kind], i, j, k, COMP[component], par, None, 0)
        self._check(rc)

    def set_line_source(self, kind, i, j0, j1, param=None, samples=None):
        """Ez of cells (i, j0 .. j1-1) all get the same waveform (2D)."""
        par = (C.c_double * 1)(float(param) if param is not None else 0.0)
        if samples is not None:
            smp = np.ascontiguousarray(samples, np.float32)
            rc = self._L.fdtd_set_line_source(self._h, SRC[kind], i, j0, j1, par, smp.ctypes.data, len(smp))
        else:
            rc = self._L.fdtd_set_line_source(self._h, SRC[kind], i, j0, j1, par, None, 0)
        self._check(rc)

    def set_scene_source(self, src):
        if getattr(src, "length", 1) > 1:
            if src.kind == "sampled":
                self.set_line_source("sampled", src.i, src.j, src.j + src.length, samples=src.samples)
            else:
                self.set_line_source(src.kind, src.i, src.j, src.j + src.length, param=src.params[0])
            return
        if src.kind == "sampled":
            self.set_source("sampled", src.i, src.j, src.k, src.component, samples=src.samples)
        else:
            self.set_source(src.kind, src.i, src.j, src.k, src.component, param=src.params[0])

    def set_materials(self, mat, eps_r, sigma):
        """New material map [ny][nx] (uint8; a page-locked array makes the upload
        asynchronous) and table for the selected 2D scene (fdtd_set_materials)."""
        m = mat if (isinstance(mat, np.ndarray) and mat.dtype == np.uint8 and mat.flags.c_contiguous) \
            else np.ascontiguousarray(mat, np.uint8)
        n = self._field_cells()
        if n is not None:
            self._need(m, n, "set_materials")
        tab = _mat_table(eps_r, sigma)
        self._check(self._L.fdtd_set_materials(self._h, m.ctypes.data, tab, len(eps_r)))

    def set_design(self, i0, j0, eps_r, sigma=None):
        """Design rectangle at (i0, j0) with per-cell eps_r [h][w] (and sigma).
        A CUDA float64 tensor goes to the library as a device pointer (the
        coefficients are formed on the GPU, no host copy); anything else is taken
        as host values."""
        if hasattr(eps_r, "data_ptr") and eps_r.is_cuda:
            import torch
            eps = eps_r.detach().to(torch.float64).contiguous()
            sg = None if sigma is None else sigma.detach().to(device=eps.device, dtype=torch.float64).contiguous()
            h, w = eps.shape
            with torch.cuda.device(eps.device):
                self._check(self._L.fdtd_set_design(self._h, i0, j0, w, h, eps.data_ptr(),
                                                    None if sg is None else sg.data_ptr(), 1))
            return
        eps = np.ascontiguousarray(eps_r, np.float64)
        h, w = eps.shape
        sg = None if sigma is None else np.ascontiguousarray(sigma, np.float64)
        self._check(self._L.fdtd_set_design(self._h, i0, j0, w, h, eps.ctypes.data,
                                            None if sg is None else sg.ctypes.data, 0))

    def add_probe(self, i, j, k=0, component="ez") -> int:
        pid = C.c_int()
        self._check(self._L.fdtd_add_probe(self._h, i, j, k, COMP[component], C.byref(pid)))
        return pid.value

    def add_dft_monitor(self, cells, freqs) -> int:
        cells = np.ascontiguousarray(cells, np.int32)
        fr = np.ascontiguousarray(freqs, np.float64)
        mid = C.c_int()
        self._check(self._L.fdtd_add_dft_monitor(self._h, cells.ctypes.data, cells.shape[0],
                                                 fr.ctypes.data_as(C.POINTER(C.c_double)), len(fr), C.byref(mid)))
        self._mon_shape = getattr(self, "_mon_shape", {})
        self._mon_shape[mid.value] = (cells.shape[0], len(fr))
        return mid.value

    def add_dft_plane(self, k, comps, freqs) -> int:
        mask = 0
        for c in comps:
            mask |= 1 << COMP[c]
        fr = np.ascontiguousarray(freqs, np.float64)
        mid = C.c_int()
        self._check(self._L.fdtd_add_dft_plane(self._h, k, mask, fr.ctypes.data_as(C.POINTER(C.c_double)),
                                               len(fr), C.byref(mid)))
        self._mon_shape = getattr(self, "_mon_shape", {})
        self._mon_shape[mid.value] = (len(comps), len(fr), self._plane_ny, self._plane_nx)
        return mid.value

    # ---------------------------------------------------------------- stepping
    def step(self, n: int):
        self._check(self._L.fdtd_step(self._h, int(n)))

    def step_edgelist(self, n: int):
        self._check(self._L.fdtd_step_edgelist(self._h, int(n)))

    def reset(self):
        self._check(self._L.fdtd_reset(self._h))

    def check_finite(self):
        self._check(self._L.fdtd_check_finite(self._h))

    def sync(self):
        """Wait for the stream; raises FDTDError(ETIMEOUT) if a bounded device
        wait gave up since the last call, else FDTDError(EUNSTABLE) if the
        periodic finite check (option "check_every") found a NaN or Inf."""
        self._check(self._L.fdtd_sync(self._h))

    def autotune(self, trial_steps=32, cache=None, key=None):
        """Pick (kernel, T, segment, warps) by timing candidates on the current
        scenes (leaves the context reset).  With a cache path, results are kept
        in a JSON file keyed by `key` and the GPU name."""
        import json
        import os
        name = None
        try:
            import torch
            name = torch.cuda.get_device_name()
        except Exception:
            name = "cuda"
        ck = f"{name}|{key}"
        if cache and key and os.path.exists(cache):
            data = json.load(open(cache))
            if ck in data:
                for k, v in data[ck]["options"].items():
                    self.set_option(k, v)
                return data[ck]
        best = C.c_double(0.0)
        self._check(self._L.fdtd_autotune(self._h, int(trial_steps), C.byref(best)))
        res = {"ms_per_step": best.value,
               "options": {k: self.get_option(k) for k in ("kernel", "tblock", "segment", "warps", "segment_b", "taper",
                                                      "warps_b", "playout")}}
        if cache and key:
            data = json.load(open(cache)) if os.path.exists(cache) else {}
            data[ck] = res
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1)
            os.replace(tmp, cache)
        return res

    # ---------------------------------------------------------------- outputs
    def field_shape(self, scene):
        return (scene.nz, scene.ny, scene.nx) if hasattr(scene, "nz") else (scene.ny, scene.nx)

    def get_field(self, component, shape=None, out=None):
        """Copy a field out.  out: a CUDA torch tensor (device copy) or None (host
        numpy array of the given shape)."""
        n = self._field_cells()
        if out is not None and hasattr(out, "data_ptr"):
            if n is not None:
                self._need(out, n, "get_field")
            self._check(self._L.fdtd_get_field(self._h, COMP[component], out.data_ptr(), 1))
            return out
        arr = np.empty(shape, np.float32) if out is None else out
        if n is not None:
            self._need(arr, n, "get_field")
        if arr.dtype != np.float32 or not arr.flags.c_contiguous:
            raise ValueError("get_field: out must be a C-contiguous float32 array")
        self._check(self._L.fdtd_get_field(self._h, COMP[component], arr.ctypes.data, 0))
        return arr

    def get_field_te(self, component, shape):
        """A 2D field under the paper's own TE naming (Sec. III-B: Ey, Hx, Hz in the
        x-z plane, k the second index).  The library computes TMz; the rotation
        x' = x, y' = z, z' = -y maps Ey = -Ez', Hx = Hx', Hz = Hy' with cell (i, j)
        <-> (i, k), so "ey", "hx", "hz" are read from "ez" (negated), "hx", "hy".
        The node numbering of the literal graph (t, u, q) is the paper's with
        k -> j (fdtd_export_graph)."""
        if component == "ey":
            return -self.get_field("ez", shape)
        return self.get_field({"hx": "hx", "hz": "hy"}[component], shape)

    def set_field(self, component, values):
        n = self._field_cells()
        if hasattr(values, "data_ptr"):
            if n is not None:
                self._need(values, n, "set_field")
            self._check(self._L.fdtd_set_field(self._h, COMP[component], values.data_ptr(), 1))
            return
        arr = np.ascontiguousarray(values, np.float32)
        if n is not None:
            self._need(arr, n, "set_field")
        self._check(self._L.fdtd_set_field(self._h, COMP[component], arr.ctypes.data, 0))

    def read_probe(self, pid, n=None) -> np.ndarray:
        n = self.time_step if n is None else n
        out = np.empty(n, np.float32)
        self._check(self._L.fdtd_read_probe(self._h, pid, out.ctypes.data, n))
        return out

    def read_dft(self, mid) -> np.ndarray:
        shape = self._mon_shape[mid]
        re = np.empty(shape, np.float32)
        im = np.empty(shape, np.float32)
        self._check(self._L.fdtd_read_dft(self._h, mid, re.ctypes.data, im.ctypes.data))
        return re.astype(np.float64) + 1j * im.astype(np.float64)

    def save_state(self) -> bytes:
        n = C.c_size_t(0)
        self._check(self._L.fdtd_save_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self._L.fdtd_save_state(self._h, buf, C.byref(n)))
        return buf.raw[:n.value]

    def load_state(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        self._check(self._L.fdtd_load_state(self._h, buf, len(data)))

    def set_checkpointing(self, every: int):
        self._check(self._L.fdtd_set_checkpointing(self._h, int(every)))

    def adjoint_grad(self, dLdF, grad_shape, out=None):
        """dL/deps_r over the design rectangles given dL/dF (complex, every cell
        monitor's [n_cells][n_freq] block concatenated).  Returns a host array of
        grad_shape, or fills the CUDA tensor `out`."""
        g = np.ascontiguousarray(np.concatenate([np.ravel(x) for x in dLdF]) if isinstance(dLdF, (list, tuple))
                                 else np.ravel(dLdF))
        re = np.ascontiguousarray(g.real, np.float32)
        im = np.ascontiguousarray(g.imag, np.float32)
        if out is not None and hasattr(out, "data_ptr"):
            self._need(out, int(np.prod(grad_shape)), "adjoint_grad")
            self._check(self._L.fdtd_adjoint_grad(self._h, re.ctypes.data, im.ctypes.data, out.data_ptr(), 1))
            return out
        res = np.empty(grad_shape, np.float32)
        self._check(self._L.fdtd_adjoint_grad(self._h, re.ctypes.data, im.ctypes.data, res.ctypes.data, 0))
        return res

    def edge_grad(self, dLdF, design_shapes, out=None):
        """dL/dw of the EDGE_CLASSES weights every design cell owns (fdtd_edge_grad)
        after a forward run recorded with option adj_store = 2.  dLdF: as for
        adjoint_grad; design_shapes: (h, w) of each scene's design rectangle.
        Returns a list of [EDGE_CLASSES, h, w] host arrays, or fills the CUDA
        tensor `out` (all scenes' blocks concatenated)."""
        g = np.ascontiguousarray(np.concatenate([np.ravel(x) for x in dLdF]) if isinstance(dLdF, (list, tuple))
                                 else np.ravel(dLdF))
        re = np.ascontiguousarray(g.real, np.float32)
        im = np.ascontiguousarray(g.imag, np.float32)
        sizes = [EDGE_CLASSES * h * w for h, w in design_shapes]
        if out is not None and hasattr(out, "data_ptr"):
            self._need(out, sum(sizes), "edge_grad")
            self._check(self._L.fdtd_edge_grad(self._h, re.ctypes.data, im.ctypes.data, out.data_ptr(), 1))
            return out
        res = np.empty(sum(sizes), np.float32)
        self._check(self._L.fdtd_edge_grad(self._h, re.ctypes.data, im.ctypes.data, res.ctypes.data, 0))
        parts = np.split(res, np.cumsum(sizes)[:-1])
        return [p.reshape(EDGE_CLASSES, h, w) for p, (h, w) in zip(parts, design_shapes)]

    def graph_size(self, layer: int):
        """(nodes, edges) of message-passing layer 1 or 2 of the current scene."""
        nn, ne = C.c_int64(), C.c_int64()
        self._check(self._L.fdtd_export_graph(self._h, layer, C.byref(nn), C.byref(ne), None, None, None))
        return nn.value, ne.value

    def export_graph(self, layer: int, te: bool = False):
        """(n_nodes, src, dst, w) of one message-passing layer (Prop. 1/2).  te:
        weights for node values under the paper's TE naming (Ey = -Ez on the
        electric nodes, te_node_signs); the numbering is the same."""
        n, src, dst, w = self._export_graph(layer)
        if te:
            if self.shape is None:
                raise ValueError("te=True needs a single-scene context")
            sg = te_node_signs(self.shape[0], self.shape[1], n, self.split)
            w = w * sg[src] * sg[dst]
        return n, src, dst, w

    def _export_graph(self, layer: int):
        nn, ne = C.c_int64(), C.c_int64()
        self._check(self._L.fdtd_export_graph(self._h, layer, C.byref(nn), C.byref(ne), None, None, None))
        src = np.empty(ne.value, np.int32)
        dst = np.empty(ne.value, np.int32)
        w = np.empty(ne.value, np.float32)
        self._check(self._L.fdtd_export_graph(self._h, layer, C.byref(nn), C.byref(ne), src.ctypes.data,
                                              dst.ctypes.data, w.ctypes.data))
        return nn.value, src, dst, w


def te_node_signs(nx: int, ny: int, n_nodes: int, split: bool = False) -> np.ndarray:
    """+1 or -1 per node of the exported graph: -1 on the electric nodes (t of
    Prop. 1; tx and tz of the split-field graph, Sec. IV-B), whose value is Ez
    in the library's TMz and Ey = -Ez under the paper's TE naming.  Magnetic and
    auxiliary (CPML) nodes keep their sign.  With S = diag(signs) the TE layer is
    S W S, and S h maps node values between the two namings."""
    idx = np.arange(n_nodes)
    per = 4 if split else 3
    r = idx % (per * nx)
    grid = idx < per * nx * ny
    if split:
        e = grid & (r >= nx) & ((r - nx) % 3 != 0)      # (q, tx, tz) triples after the u block
    else:
        e = grid & (r >= nx) & ((r - nx) % 2 == 1)      # (q, t) pairs after the u block
    sg = np.ones(n_nodes, np.float32)
    sg[e] = -1.0
    return sg


EDGE_CLASSES = 11   # FDTD_EDGE_CLASSES: weights a design cell owns as a destination

MP_NOALLOC_MAX_NODES = 1 << 22


def check_noalloc_args(layer1, layer2, h, require_cuda=True):
    """Reject, before anything is launched, arguments fdtd_mp_steps_noalloc's
    kernel would read out of bounds or across devices: tensors that are not
    torch tensors, not on CUDA (when require_cuda), of the wrong dtype
    (int32 rowptr/col, float32 w/h), not contiguous, not all on h's device;
    a rowptr without n_nodes + 1 entries; w and col of different lengths.
    Returns n_nodes."""
    import torch
    r1, c1, w1 = layer1
    r2, c2, w2 = layer2
    named = (("h", h, torch.float32), ("rowptr1", r1, torch.int32), ("col1", c1, torch.int32),
             ("w1", w1, torch.float32), ("rowptr2", r2, torch.int32), ("col2", c2, torch.int32),
             ("w2", w2, torch.float32))
    for name, t, dt in named:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name}: expected a torch tensor")
        if require_cuda and not t.is_cuda:
            raise ValueError(f"{name}: must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name}: dtype {t.dtype}, expected {dt}")
        if not t.is_contiguous():
            raise ValueError(f"{name}: must be contiguous")
        if t.device != h.device:
            raise ValueError(f"{name}: on {t.device}, h on {h.device}")
    n = int(h.numel())
    for k, (rp, col, w) in enumerate(((r1, c1, w1), (r2, c2, w2)), 1):
        if rp.dim() != 1 or rp.numel() != n + 1:
            raise ValueError(f"rowptr{k}: {rp.numel()} entries, expected n_nodes + 1 = {n + 1}")
        if w.numel() != col.numel():
            raise ValueError(f"w{k}: {w.numel()} entries, col{k} has {col.numel()}")
    return n


def mp_steps_noalloc(layer1, layer2, h, n_steps, stream=None):
    """Allocation-free two-layer message passing (fdtd_mp_steps_noalloc).

    layer1/layer2: (rowptr, col, w) CUDA tensors (int32, int32, float32); h:
    CUDA float32 tensor of node values, updated in place.  For callers that
    cannot allocate device memory (see the C header).  The kernel trusts the
    graph's shape, so check_noalloc_args vets every tensor first; the call runs
    with h's device current (the scratch array is per device)."""
    import torch
    n = check_noalloc_args(layer1, layer2, h)
    L = lib()
    r1, c1, w1 = layer1
    r2, c2, w2 = layer2
    with torch.cuda.device(h.device):
        rc = L.fdtd_mp_steps_noalloc(r1.data_ptr(), c1.data_ptr(), w1.data_ptr(), r2.data_ptr(), c2.data_ptr(),
                                     w2.data_ptr(), h.data_ptr(), n, int(n_steps), _stream_handle(stream))
    if rc != OK:
        raise FDTDError(rc, "fdtd_mp_steps_noalloc rejected its arguments or failed to launch"
                        f" (n_nodes {n}, limit {MP_NOALLOC_MAX_NODES})")


def from_scene(scene, *, stream=None, probes=True, monitors=True, source=True, boundary=None) -> Simulation:
    """A Simulation for a seeded scene: its source, its probes (Ez) and, if it
    has monitor cells and frequencies, one DFT monitor over them.  boundary: see
    _grid_of (default: CPML when the scene has a layer)."""
    sim = Simulation(scene, stream=stream, boundary=boundary)
    if hasattr(scene, "nz"):
        sim._plane_ny, sim._plane_nx = scene.ny, scene.nx
    if source and scene.source is not None:
        sim.set_scene_source(scene.source)
    if getattr(scene, "design", None) is not None:
        i0, j0, w, h = scene.design
        sim.set_design(i0, j0, scene.design_eps)
    sim.probe_ids = []
    if probes and getattr(scene, "probes", None) is not None:
        for p in scene.probes:
            sim.probe_ids.append(sim.add_probe(int(p[0]), int(p[1])))
    sim.mon_id = None
    if monitors and getattr(scene, "monitors", None) is not None and scene.freqs is not None:
        sim.mon_id = sim.add_dft_monitor(scene.monitors, scene.freqs)
    return sim
