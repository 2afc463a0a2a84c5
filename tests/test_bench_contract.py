"""bench.py's reference arm (the FP64 oracle timed on the host cores) prints
the contract's JSON line; runs on CPU with a two-step sample."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--ref-sample", "2"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference" and d["metric"] == "FDTD cell-updates/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("tmz2d_4096x4096")


def test_traffic_record_matches_options_and_source():
    """roofline.traffic comes from the committed ncu record whose kernel options
    equal the run's, and only while k_tmz.cu is the file it was taken with."""
    sys.path.insert(0, ROOT)
    import bench
    import hashlib
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_tmz_fused_traffic.json")))
    r = rec["records"][0]
    opts = {k: r["options"][k] for k in bench.TRAFFIC_KEYS}
    src = os.path.join(ROOT, "paper_2405_00814_gb300", "csrc", "k_tmz.cu")
    current = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == rec["source_sha256_16"]
    assert bench._traffic_record(opts) == (r["dram_bytes_per_block"] if current else None)
    assert 0.95 < r["dram_bytes_per_block"] / rec["algorithmic_bytes_per_block"] < 1.2
    other = dict(opts, segment=opts["segment"] + 1)
    assert bench._traffic_record(other) is None
    for x in rec["records"]:
        assert len(x["blocks"]) == 2 and "ncu" in x["command"] and "--clock-control none" in x["command"]
