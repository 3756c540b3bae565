"""The reference arm of bench.py on the CPU (it times the oracle only): one
JSON line with the contract's keys, a cpu_baseline describing the run, and an
e2e object with no copies."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [t for t in r.stdout.splitlines() if t.strip()]
    assert len(lines) == 1
    assert len(lines[0].encode()) <= 1400
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["dtype"] == "f64" and "workload" in d["config"]
    # the repo arm's cpu_baseline names the same sample in its config
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"]["cpu_sample"] == bench.CPU_SAMPLE_SHORT
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_cpu_sample_record_matches_the_reference_arm():
    """The repo arm's cpu_baseline comes from `bench.py --cpu-sample S` in a
    fresh process: the same named sample and oracle call as the reference arm."""
    r = subprocess.run([sys.executable, "bench.py", "--cpu-sample", "0.3"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench
    assert d["kind"] == "oracle" and d["cores"] == 1 and d["value"] > 0
    assert d["sample"].startswith(bench.CPU_SAMPLE)
    assert d["all_cores"]["cores"] >= 1 and d["all_cores"]["value"] > 0
