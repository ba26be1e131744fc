"""The benchmark's output contract, checked on the CPU through its reference
arm (the FP64 oracle timed on the host cores): one JSON line with the
metric, the whole-job value, the timing and the CPU-baseline and end-to-end
objects the GPU arm prints as well."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_line(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_prints_one_contract_line():
    j = _bench_line("--impl", "reference", "--workload", "mesh32_dg1", "--steps", "2",
                    "--warmup", "1")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference"
    assert j["n_gpus"] == 1 and j["steps"] == 2 and j["warmup"] == 1
    assert j["higher_is_better"] is True and j["scaling"] == "weak"
    assert j["dtype"] == "f64" and j["data"] == "synthetic" and j["vs_baseline"] is None
    assert j["unit"] == "element-subcycles/s" and j["value"] > 0
    c = j["config"]
    assert c["workload"] == "mesh32_dg1" and (c["nx"], c["ny"], c["n_stress"]) == (32, 32, 3)
    assert 1 <= c["n_sub_per_step"] <= c["n_sub_workload"]
    # value = elements x subcycles per step / seconds per step
    assert abs(j["value"] - 32 * 32 * c["n_sub_per_step"] / (j["ms_per_step"] / 1e3)) \
        <= 1e-6 * j["value"]
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1
    assert cb["unit"] == j["unit"] and "subcycles" in cb["sample"]
    e = j["e2e"]
    assert e["value"] == j["value"] and e["unit"] == j["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
