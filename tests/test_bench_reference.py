"""The reference arm of bench.py (the FP64 oracle timed on the host cores)
prints one well-formed JSON line.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--n", "4000", "--cpu-seconds", "0.3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "pair/s" and d["higher_is_better"] is True
    assert d["config"]["n_particles"] == 4000
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["gpu_launches"] == 0


def test_oracle_step_scaling_rows():
    """The host leg of the N sweep (the paper's Fig. 7 with the oracle): one
    full oracle step per N on all cores and one per core count."""
    sys.path.insert(0, ROOT)
    import bench
    d = bench.oracle_step_scaling(ns=(400, 800), sweep_n=400)
    assert d["kind"] == "oracle" and d["cores"] >= 1
    assert [r["n"] for r in d["n_rows"]] == [400, 800]
    assert all(r["s_per_step"] > 0 and r["pairs_per_s"] > 0 for r in d["n_rows"])
    counts = [r["cores"] for r in d["core_rows"]]
    assert counts[0] == 1 and counts[-1] == d["cores"] and counts == sorted(set(counts))
    assert d["core_rows"][0]["speedup"] == 1.0
