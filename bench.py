#!/usr/bin/env python
"""Throughput benchmark: FDTD cell-updates/s on the 4096^2 heterogeneous 2D TMz
workload (200 seeded ellipses, eps_r ~ U[1,12], sigma ~ U[0,0.05] S/m, uint8
material map, 16-cell CPML, Gaussian-modulated 2.4 GHz soft source, 4000 steps).

One benchmark step = one complete solve: fields reset, 4000 leapfrog steps with
the source and 4 probes.  `value` is device time with inputs resident in HBM;
`e2e` is the same metric through the C ABI from host buffers: one context, and
per solve the material map uploaded from page-locked host memory, the reset,
the solve, Ez and the probe records copied back (`fresh_context_value`: the
same with a context created and destroyed around every solve).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CU = 25.0        # 3 fields x 4 B read + 3 x 4 B written + 1 B material (single sweep)
WORKLOAD = "tmz2d_4096x4096_ellipses200_cpml16_gaussmod2.4GHz_4000steps"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler run during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


TRAFFIC_KEYS = ("tblock", "segment", "warps", "warps_b", "segment_b", "taper")


def _traffic_record(tune):
    """DRAM bytes per T-step block of the fused kernel pair from the committed
    ncu summary: the record taken with the same kernel options, valid only while
    the kernel source is unchanged (else None)."""
    p = os.path.join(ROOT, "profiles", "k_tmz_fused_traffic.json")
    src = os.path.join(ROOT, "paper_2405_00814_gb300", "csrc", "k_tmz.cu")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != h:
        return None
    want = {k: int(tune[k]) for k in TRAFFIC_KEYS}
    for r in rec.get("records", []):
        if {k: int(r["options"][k]) for k in TRAFFIC_KEYS} == want:
            return r["dram_bytes_per_block"]
    return None


def cpu_baseline(sc, budget_s=12.0):
    """The FP64 oracle as it stands, on the host cores, over a bounded prefix of
    the same workload: chunks of 10 steps until the budget is used, with every
    core (OpenMP over rows) and then with one thread."""
    import oracle
    cores = oracle.num_threads()

    def timed(threads, budget):
        oracle.set_threads(threads)
        sim = oracle.TMz(sc, nsteps_src=sc.nsteps)
        sim.run(2)
        t0 = time.perf_counter()
        steps = 0
        while time.perf_counter() - t0 < budget:
            sim.run(10)
            steps += 10
        return sc.cells * steps / (time.perf_counter() - t0), steps

    try:
        v_all, s_all = timed(cores, budget_s)
        v_one, s_one = timed(1, budget_s / 3)
    finally:
        oracle.set_threads(cores)
    return {"value": v_all, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{s_all} leapfrog steps of the full {sc.nx}x{sc.ny} scene (FP64, OpenMP over rows)",
            "single_thread": {"value": v_one, "sample": f"{s_one} leapfrog steps, 1 thread"},
            "paper_sweep": oracle_sweep()}


def oracle_sweep(sides=(250, 1000, 2000, 3000, 4000, 5000, 6400), budget_s=1.5):
    """The paper's free-space sweep on the oracle (all cores): a bounded prefix
    of each 1024-step solve, at least 2 steps, about budget_s seconds per side."""
    import oracle
    from paper_2405_00814_gb300 import scenes
    out = {}
    for side in sides:
        sc = scenes.free_space(side)
        sim = oracle.TMz(sc, nsteps_src=sc.nsteps)
        sim.run(1)
        t0 = time.perf_counter()
        steps = 0
        while steps < 2 or (time.perf_counter() - t0 < budget_s and steps < sc.nsteps):
            sim.run(1)
            steps += 1
        out[str(side)] = {"cell_updates_per_s": sc.cells * steps / (time.perf_counter() - t0), "steps": steps}
    return out


def paper_sweep(stream, tune, sides=(250, 1000, 2000, 3000, 4000, 5000, 6400), nsteps=1024, runs=5):
    """The paper's timing workload (Sec. V-C, Fig. 5): free space with a 16-cell
    absorbing boundary, square grids of the listed sides, 1024 steps, 5 runs per
    side; mean and 95% confidence half-width (Student t, 4 dof) of the device
    time per solve, and cell-updates/s.  tune None: the library's autotuner
    picks the kernel options per side."""
    import torch
    from paper_2405_00814_gb300 import fdtd, scenes
    t95 = 2.776
    out = {}
    for side in sides:
        sc = scenes.free_space(side, nsteps=nsteps)
        sim = fdtd.from_scene(sc, stream=stream)
        if tune is None:
            tune_used = sim.autotune(trial_steps=16)["options"]
        else:
            tune_used = dict(tune)
            for k, v in tune.items():
                sim.set_option(k, v)
        sim.step(nsteps)            # warm-up solve
        ms = []
        for _ in range(runs):
            sim.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(nsteps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        sim.close()
        mean = sum(ms) / runs
        sd = (sum((x - mean) ** 2 for x in ms) / (runs - 1)) ** 0.5
        out[str(side)] = {"ms_mean": mean, "ms_ci95": t95 * sd / runs ** 0.5,
                          "cell_updates_per_s": sc.cells * nsteps / (mean / 1e3), "options": tune_used}
    return {"workload": "paper_sweep_free_space_cpml16_1024steps", "runs": runs, "sides": out,
            "timing": "CUDA events around fdtd_step per solve after one warm-up solve"}


def adjoint_ratio(stream, reps=2, nsteps=None):
    """Time of one adjoint gradient (forward with checkpoints every 100 steps +
    reverse sweep) over the time of one plain forward solve, on the 1024^2
    inverse-design workload (8 designs, 256^2 design regions, 8 monitors,
    3000 steps): dL/deps_r, and dL/dw of the 11 edge classes of every design
    cell (fdtd_edge_grad)."""
    import numpy as np
    import torch
    from paper_2405_00814_gb300 import autograd, scenes
    scs = scenes.adjoint_scenes() if nsteps is None else scenes.adjoint_scenes(nsteps=nsteps)
    eps = np.stack([s.design_eps for s in scs])
    plain = autograd.DesignBatch(scs, ckpt_every=0, stream=stream)
    ckpt = autograd.DesignBatch(scs, ckpt_every=100, stream=stream)

    def t_of(fn):
        best = None
        for _ in range(reps + 1):          # first run warms up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        return best
    t_fwd = t_of(lambda: plain.forward(eps))
    t_grad = t_of(lambda: ckpt.gradient(2.0 * ckpt.forward(eps)))
    plain.close()
    ckpt.close()
    edges = autograd.DesignBatch(scs, ckpt_every=100, stream=stream, edges=True)
    t_edge = t_of(lambda: edges.edge_gradient(2.0 * edges.forward(eps)))
    edges.close()
    cu = scs[0].cells * len(scs) * scs[0].nsteps
    return {"workload": f"adjoint_tmz2d_1024x1024_x8designs_{scs[0].nsteps}steps_ckpt100", "forward_ms": 1e3 * t_fwd,
            "gradient_ms": 1e3 * t_grad, "ratio": t_grad / t_fwd, "forward_cups": cu / t_fwd,
            "edge_gradient_ms": 1e3 * t_edge, "edge_ratio": t_edge / t_fwd,
            "timing": "host wall clock around synchronised calls, best of %d after one warm-up" % reps}


def batch_throughput(stream, reps=2):
    """64 uneven scenes (sides log-uniform 256..2048, 12-cell CPML), 2000 steps:
    one autotuned context, timed solve (reset + 2000 steps) with CUDA events."""
    import torch
    from paper_2405_00814_gb300 import fdtd, scenes
    scs = scenes.batch_scenes()
    sim = fdtd.Simulation.batch(scs, stream=stream)
    for k, s in enumerate(scs):
        sim.select(k)
        sim.set_scene_source(s.source)
    tune = sim.autotune(trial_steps=16)
    sim.set_option("graph", 1)
    nsteps = scs[0].nsteps
    best = None
    for _ in range(reps + 1):
        sim.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(nsteps)
        e1.record(stream)
        sim.sync()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    # the same solve as one persistent cooperative launch (FDTD_OPT_KERNEL = 2:
    # every scene's work items, all 2000 steps, each item waiting only for its
    # neighbours' previous block), captured in a CUDA graph: the autotuner's
    # persistent options if it chose them, else T = 4 and the best of three
    # segment heights and three CTA layouts (FDTD_OPT_PLAYOUT)
    opts = tune["options"]
    sim.set_option("kernel", 2)
    trials = ([(opts["segment"], opts["playout"])] if opts["kernel"] == 2 else
              [(seg, pl) for seg in (64, 96, 128) for pl in (0, 48, 64)])
    pbest, pseg, pplay = None, None, None
    for seg, pl in trials:
        if opts["kernel"] != 2:
            sim.set_option("tblock", 4)
            sim.set_option("segment", seg)
            sim.set_option("playout", pl)
        for _ in range(reps + 1):
            sim.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(nsteps)
            e1.record(stream)
            sim.sync()
            ms = e0.elapsed_time(e1)
            if pbest is None or ms < pbest:
                pbest, pseg, pplay = ms, seg, pl
    sim.close()
    cells = sum(s.cells for s in scs)
    return {"workload": "batch64_tmz2d_sides256-2048_cpml12_2000steps", "cells": cells,
            "cell_updates_per_s": cells * nsteps / (best / 1e3), "ms_per_solve": best,
            "autotuned": tune["options"], "graph": True,
            "persistent_one_launch": {"cell_updates_per_s": cells * nsteps / (pbest / 1e3), "ms_per_solve": pbest,
                                      "tblock": 4 if opts["kernel"] != 2 else opts["tblock"],
                                      "segment": pseg, "playout": pplay},
            "timing": "CUDA events around one solve replayed from a CUDA graph, best of %d after one warm-up" % reps}


def yee3d_throughput(stream, nsteps=200, side=512, kernel=None, segment=None, tblock=None):
    """512^3 box workload (64 dielectric boxes, 10-cell CPML, Ez dipole, DFT plane
    at 3 frequencies): cell-updates/s over nsteps steps.  Roofline: 49 B per cell
    per HBM pass (E, H, material read; E, H written), one pass per `tblock`
    steps."""
    import torch
    from paper_2405_00814_gb300 import fdtd, scenes
    sc = scenes.box_scene() if side == 512 else scenes.box_scene(side=side)
    sim = fdtd.from_scene(sc, stream=stream)
    if kernel is not None:
        sim.set_option("kernel", kernel)
    if segment is not None:
        sim.set_option("segment", segment)
    if tblock is not None:
        sim.set_option("tblock", tblock)
    tb, seg = sim.get_option("tblock"), sim.get_option("segment")
    if seg == 0:   # automatic: 24 planes for the one-step kernel, 48 for the two-step one
        seg = 48 if tb == 2 else 24
    sim.add_dft_plane(sc.dft_plane_k, ("ex", "ey", "ez"), sc.freqs)
    sim.step(10)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(nsteps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sim.close()
    peak, _ = _peaks()
    cu = sc.cells * nsteps / (ms / 1e3)
    return {"workload": f"yee3d_{side}^3_boxes64_cpml10_dftplane", "cell_updates_per_s": cu, "ms_per_step": ms / nsteps,
            "tblock": tb, "segment": seg,
            # against the kernel's own bound (49 B per cell per pass of tblock steps)
            "hbm_roofline_frac": cu * 49.0 / tb / (peak * 1e9),
            # against the bound of any one-step-per-pass kernel (49 B per cell-update)
            "hbm_roofline_frac_at_49B_per_cell_update": cu * 49.0 / (peak * 1e9)}


def edgelist_throughput(stream, side=2048, nsteps=200):
    """The literal message-passing form (Prop. 1/2: two CSR layers per step) on
    the heterogeneous CPML scene scaled to side^2: cell-updates/s, and the
    algorithmic bytes per cell-update of the two gathers (8 B per edge for
    column index and weight, 12 B per node for row pointer, value and result)."""
    import torch
    from paper_2405_00814_gb300 import fdtd, scenes
    sc = scenes.ellipse_scene(side=side)
    sim = fdtd.from_scene(sc, stream=stream)
    sim.step_edgelist(4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step_edgelist(nsteps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    b = 0
    for layer in (1, 2):
        nn, ne = sim.graph_size(layer)
        b += 8 * ne + 12 * nn
    sim.close()
    peak, _ = _peaks()
    cu = sc.cells * nsteps / (ms / 1e3)
    bpc = b / sc.cells
    return {"workload": f"edgelist_tmz2d_{side}x{side}_ellipses_cpml16", "cell_updates_per_s": cu,
            "bytes_per_cell_update": bpc, "hbm_frac": cu * bpc / (peak * 1e9), "ms_per_step": ms / nsteps}


def split_pml_throughput(stream, side=4096, nsteps=200, side_graph=2048):
    """The paper's own absorber (split-field PML, FDTD_SPLIT_PML) on the
    heterogeneous scene: the temporally blocked split variant (autotuned, graph
    replay), the unfused stencil pair at side^2 (with the same pair under CPML
    beside it), and the literal 4-node graph at side_graph^2."""
    import torch
    from paper_2405_00814_gb300 import fdtd, scenes
    peak, _ = _peaks()

    def timed(sim, fn, n):
        fn(4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    out = {"workload": f"split_pml_tmz2d_{side}_ellipses_layer16_{nsteps}steps"}
    sc = scenes.ellipse_scene(side=side)
    # the temporally blocked split variant, autotuned, solves replayed from a CUDA graph
    sim = fdtd.from_scene(sc, stream=stream, boundary="split")
    tune = sim.autotune(trial_steps=16)
    sim.set_option("graph", 1)
    best = None
    for _ in range(3):
        sim.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    sim.close()
    cu = sc.cells * nsteps / (best / 1e3)
    out["split_fused"] = {"cell_updates_per_s": cu, "options": tune["options"],
                          "hbm_frac_at_25B_per_cell_update": cu * 25.0 / (peak * 1e9)}
    for name, boundary in (("split_stencil", "split"), ("cpml_unfused", "cpml")):
        sim = fdtd.from_scene(sc, stream=stream, boundary=boundary)
        sim.set_option("kernel", 1)
        ms = timed(sim, sim.step, nsteps)
        sim.close()
        cu = sc.cells * nsteps / (ms / 1e3)
        out[name] = {"cell_updates_per_s": cu, "hbm_frac_at_37B_per_cell_update": cu * 37.0 / (peak * 1e9)}
    sg = scenes.ellipse_scene(side=side_graph)
    sim = fdtd.from_scene(sg, stream=stream, boundary="split")
    ms = timed(sim, sim.step_edgelist, nsteps)
    b = sum(8 * ne + 12 * nn for nn, ne in (sim.graph_size(1), sim.graph_size(2)))
    sim.close()
    cu = sg.cells * nsteps / (ms / 1e3)
    out["split_edgelist"] = {"side": side_graph, "cell_updates_per_s": cu, "bytes_per_cell_update": b / sg.cells,
                             "hbm_frac": cu * (b / sg.cells) / (peak * 1e9)}
    return out


def phc_waveguide_time(stream, reps=3):
    """The photonic-crystal example (Sec. V-B: 75 THz pulse from a line source in
    an eps_r = 12 waveguide with two groups of 3 air holes) solved to the end of
    its 3000 steps with both probes: milliseconds per solve (best of reps) on
    the temporally blocked path with the autotuner's options, one CUDA-graph
    replay per solve."""
    import torch
    from paper_2405_00814_gb300 import fdtd, scenes
    sc = scenes.phc_waveguide()
    sim = fdtd.from_scene(sc, stream=stream)
    tune = sim.autotune()
    sim.set_option("graph", 1)
    best = None
    for _ in range(reps + 1):
        sim.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(sc.nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    sim.close()
    return {"workload": f"phc_waveguide_{sc.nx}x{sc.ny}_line_source_{sc.nsteps}steps", "ms_per_solve": best,
            "options": tune["options"],
            "cell_updates_per_s": sc.cells * sc.nsteps / (best / 1e3)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2405_00814_gb300 import scenes
    import oracle
    oracle.lib()
    sc = scenes.ellipse_scene()
    sim = oracle.TMz(sc, nsteps_src=sc.nsteps)
    per = args.ref_sample
    for _ in range(args.warmup):
        sim.run(per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.run(per)
    dt = time.perf_counter() - t0
    val = sc.cells * per * args.steps / dt
    cores = oracle.num_threads()
    line = {"metric": "FDTD cell-updates/s", "value": val, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_steps_per_bench_step": per},
            "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per} leapfrog steps of the full scene per bench step"},
            "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gem", choices=["gem", "reference"])
    ap.add_argument("--tblock", type=int, default=None)
    ap.add_argument("--segment", type=int, default=None)
    ap.add_argument("--warps", type=int, default=None)
    ap.add_argument("--segment-b", type=int, default=None, help="FDTD_OPT_SEGMENT_B (boundary task rows; 0 = automatic)")
    ap.add_argument("--kernel", type=int, default=None, help="FDTD_OPT_KERNEL (default 0)")
    ap.add_argument("--warps-b", type=int, default=None, help="FDTD_OPT_WARPS_B (warps per CPML CTA)")
    ap.add_argument("--taper", type=int, default=None, help="FDTD_OPT_TAPER (percent of interior rows in "
                    "half-height tail segments; 0 = uniform)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-sample", type=int, default=20)
    ap.add_argument("--nsteps", type=int, default=None, help="leapfrog steps per solve (default: the workload's 4000)")
    ap.add_argument("--size", type=int, default=4096, help="grid side (profiling runs use smaller sides)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every block from the host instead of replaying each solve from a CUDA graph")
    ap.add_argument("--workload", default="main",
                    choices=["main", "adjoint", "batch", "yee3d", "sweep", "edgelist", "split", "phc"],
                    help="main: the JSON line of record; the others time one secondary workload alone "
                         "(for profiling; --nsteps and, for yee3d, --size, --kernel, --segment and --tblock apply)")
    ap.add_argument("--no-extras", action="store_true", help="skip the adjoint-ratio measurement")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_00814_gb300 import fdtd, scenes

    stream = torch.cuda.current_stream()
    if args.workload != "main":
        if args.workload == "adjoint":
            res = adjoint_ratio(stream, nsteps=args.nsteps)
        elif args.workload == "batch":
            res = batch_throughput(stream)
        elif args.workload == "yee3d":
            res = yee3d_throughput(stream, nsteps=args.nsteps or 200, side=args.size if args.size != 4096 else 512,
                                   kernel=args.kernel, segment=args.segment, tblock=args.tblock)
        elif args.workload == "split":
            res = split_pml_throughput(stream, nsteps=args.nsteps or 200)
        elif args.workload == "edgelist":
            res = edgelist_throughput(stream, side=args.size if args.size != 4096 else 2048, nsteps=args.nsteps or 200)
        elif args.workload == "phc":
            res = phc_waveguide_time(stream)
        else:
            res = paper_sweep(stream, None)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return

    sc = scenes.ellipse_scene(side=args.size)
    nsteps = args.nsteps or sc.nsteps
    sim = fdtd.from_scene(sc, stream=stream)
    # kernel options: the library's autotuner on this scene, unless given
    manual = any(getattr(args, k) is not None for k in ("tblock", "segment", "warps", "kernel", "segment_b", "taper",
                                                   "warps_b"))
    if manual:
        tune = {"tblock": 4, "segment": 24, "warps": 8, "segment_b": 0, "taper": 0, "warps_b": 2}
        for k in ("tblock", "segment", "warps", "segment_b", "taper", "warps_b"):
            if getattr(args, k) is not None:
                tune[k] = getattr(args, k)
        if args.kernel is None:
            args.kernel = 0
        sim.set_option("kernel", args.kernel)
        for k, v in tune.items():
            sim.set_option(k, v)
    else:
        sim.autotune(trial_steps=32)
        args.kernel = sim.get_option("kernel")
        tune = {k: sim.get_option(k) for k in ("tblock", "segment", "warps", "segment_b", "taper", "warps_b")}
    # each solve (reset + n steps from t = 0) is recorded once into a CUDA graph
    # and replayed (FDTD_OPT_GRAPH); the warm-up solves record it
    graph = not args.no_graph and args.kernel != 1
    if graph:
        sim.set_option("graph", 1)

    def solve():
        sim.reset()
        sim.step(nsteps)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = sim.launch_count
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 2)]
    ev[0].record(stream)
    for k in range(args.steps):
        sim.reset()
        ev[1 + 2 * k].record(stream)
        sim.step(nsteps)
        ev[2 + 2 * k].record(stream)
    ev[-1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = sim.launch_count - l0
    ms_total = ev[0].elapsed_time(ev[-1])
    ms_step_only = sum(ev[1 + 2 * k].elapsed_time(ev[2 + 2 * k]) for k in range(args.steps))
    clk = clocks.stop()
    if dist:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_per = ms_total / args.steps
    cell_updates = sc.cells * nsteps
    value = cell_updates * args.steps * world / (ms_total / 1e3)

    # dominant kernel: the fused stream, one launch per tblock steps
    T = tune["tblock"] if args.kernel in (0, 2) else 1
    fused_launches = args.steps * math.ceil(nsteps / T)
    avg_launch_s = (ms_step_only / 1e3) / fused_launches
    peak, peak_kind = _peaks()
    alg_bytes = BYTES_PER_CU * sc.cells            # bytes one launch must move (state in + out, material)
    achieved = alg_bytes / avg_launch_s / 1e9
    traffic = _traffic_record(tune) if args.kernel == 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": (f"k_tmz_interior<{T}> + k_tmz_cpml_mixed<{T}> (one T-step block, run concurrently)"
                           if args.kernel == 0 else
                           f"k_tmz_persistent<{T}> (T-step blocks of dependency-ordered work items)" if args.kernel == 2
                           else "k_tmz_h + k_tmz_e"),
                "unit_bytes": "25 B per grid cell per launch (each launch advances every cell T steps)"}
    hbm_frac_cu = value / world * BYTES_PER_CU / (peak * 1e9)

    workload = WORKLOAD if (args.size == 4096 and nsteps == 4000) else f"tmz2d_{args.size}_ellipses_cpml16_{nsteps}steps"
    out = {"metric": "FDTD cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload, "cells": sc.cells, "leapfrog_steps_per_bench_step": nsteps,
                      "tblock": T, "segment": tune["segment"], "warps_per_cta": tune["warps"],
                      "segment_b": tune["segment_b"], "taper": tune["taper"], "warps_b": tune["warps_b"],
                      "kernel_options": "manual" if manual else "fdtd_autotune on this scene",
                      "cuda_graph": graph,
                      "l2": "inputs larger than L2 (fields 2x3x70 MB + material 17 MB)",
                      "parallelism": "replicas" if world > 1 else "single"},
           "roofline": roofline,
           "hbm_roofline_frac_at_25B_per_cell_update": hbm_frac_cu,
           "gpu_launches": launches, "clocks": clk}

    # end to end through the C ABI from host buffers
    if not args.no_e2e:
        import numpy as np
        sim.close()
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 3))
        h2d = sc.mat.nbytes + 24 * len(sc.eps_r)
        d2h = sc.cells * 4 + 4 * nsteps * len(sc.probes)
        # serving form: one context, and per solve the geometry uploaded from
        # page-locked host memory (fdtd_set_materials), reset, the solve (graph
        # replay), Ez and the probe records read back into host memory
        mat_pin = torch.empty(sc.mat.shape, dtype=torch.uint8, pin_memory=True).numpy()
        mat_pin[...] = sc.mat
        ez_pin = torch.empty((sc.ny, sc.nx), dtype=torch.float32, pin_memory=True).numpy()
        s2 = fdtd.from_scene(sc, stream=stream)
        s2.set_option("kernel", args.kernel)
        for k, v in tune.items():
            s2.set_option(k, v)
        if graph:
            s2.set_option("graph", 1)

        def e2e_solve():
            s2.set_materials(mat_pin, sc.eps_r, sc.sigma)
            s2.reset()
            s2.step(nsteps)
            s2.get_field("ez", out=ez_pin)
            for p in s2.probe_ids:
                s2.read_probe(p, nsteps)

        e2e_solve()                     # warm-up (records the graph)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_solve()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        s2.close()
        out["e2e"] = {"value": cell_updates * e2e_steps * world / e2e_s, "unit": "cell-updates/s",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "form": "one context; per solve: material map upload from pinned memory, reset, "
                              "solve, Ez + probe records read back"}
        # the same with a context created and destroyed around every solve
        host_ez = np.empty((sc.ny, sc.nx), np.float32)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            s3 = fdtd.from_scene(sc, stream=stream)
            s3.set_option("kernel", args.kernel)
            for k, v in tune.items():
                s3.set_option(k, v)
            s3.step(nsteps)
            s3.get_field("ez", out=host_ez)
            for p in s3.probe_ids:
                s3.read_probe(p, nsteps)
            s3.close()
        torch.cuda.synchronize()
        out["e2e"]["fresh_context_value"] = cell_updates * e2e_steps * world / (time.perf_counter() - t0)
    if not args.no_extras:
        out["adjoint"] = adjoint_ratio(stream)
        out["batch"] = batch_throughput(stream)
        out["yee3d"] = yee3d_throughput(stream)
        out["paper_sweep"] = paper_sweep(stream, None)
        out["edgelist"] = edgelist_throughput(stream)
        out["split_pml"] = split_pml_throughput(stream)
        out["phc_waveguide"] = phc_waveguide_time(stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sc, args.cpu_budget)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
