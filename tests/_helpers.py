"""Shared test helpers: relative errors and oracle / CUDA runs of a scene."""
import numpy as np

# GPU FP32 fields vs the FP64 oracle: relative L2 at the last step (and over
# probe series), the tolerance the parity bar states.
TOL_FIELD = 1e-4


def rel_l2(x, ref, floor=0.0):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    den = max(float(np.linalg.norm(ref)), floor)
    if den == 0.0:
        return float(np.linalg.norm(x))
    return float(np.linalg.norm(x - ref)) / den


def oracle_run(scene, nsteps, probes=None, monitors=None, freqs=None):
    import oracle
    sim = oracle.TMz(scene, nsteps_src=nsteps)
    samples = [(int(i), int(j), "ez") for i, j in probes] if probes is not None else None
    out = sim.run(nsteps, samples=samples, dft_cells=monitors, freqs=freqs)
    res = {k: sim.state[k].copy() for k in ("ez", "hx", "hy")}
    res["probes"] = out.get("samples")
    if monitors is not None:
        res["dft"] = sim.dft[0] + 1j * sim.dft[1]
    return res


def gpu_run(scene, nsteps, *, kernel=0, tblock=4, segment=128, warps=2, probes=True, monitors=True, options=None):
    from paper_2405_00814_gb300 import fdtd
    sim = fdtd.from_scene(scene, probes=probes, monitors=monitors)
    sim.set_option("kernel", kernel)
    sim.set_option("tblock", tblock)
    sim.set_option("segment", segment)
    sim.set_option("warps", warps)
    for k, v in (options or {}).items():
        sim.set_option(k, v)
    sim.step(nsteps)
    shape = (scene.ny, scene.nx)
    res = {c: sim.get_field(c, shape) for c in ("ez", "hx", "hy")}
    res["probes"] = np.stack([sim.read_probe(p, nsteps) for p in sim.probe_ids], axis=1) if sim.probe_ids else None
    if sim.mon_id is not None:
        res["dft"] = sim.read_dft(sim.mon_id)
    res["launches"] = sim.launch_count
    sim.close()
    return res


def assert_fields_close(g, o, tol=TOL_FIELD, comps=("ez", "hx", "hy")):
    for c in comps:
        e = rel_l2(g[c], o[c])
        assert e <= tol, f"{c}: rel L2 {e:.3e} > {tol}"
