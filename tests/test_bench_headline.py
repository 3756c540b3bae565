"""bench.py's stdout line on the CPU: the headline builder applied to a fake
full record with every leg present keeps the contract's keys, parses as JSON
and stays under the size limit, so that a log tail of the run holds it whole;
the sweep's calls cover every (offset, alias) pair; the CPU sample is the one
both arms name."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def fake_record():
    sweep_rows = [{"n": n, "offset_bytes": 8 * o, "alias": al, "calls_per_flushed_run": 1,
                   "gbs_l2_flushed": 7012.3456789, "us_l2_flushed": 123.456789,
                   "gbs_l2_resident": 9000.123, "frac_of_peak_flushed": 1.0321}
                  for (n, o, al) in bench.sweep_calls()]
    for k in (24, 26, 28):
        for (name, ox, oy, ow, al) in bench.CLASS_CASES:
            sweep_rows.append({"n": 1 << k, "case": name, "alias": al, "x_offset_bytes": ox,
                               "y_offset_bytes": oy, "w_offset_bytes": ow,
                               "gbs_l2_flushed": 6543.21, "frac_of_peak_flushed": 0.9631})
    served_rows = [{"rate": r, "p99_ms": 12.3456, "p50_ms": 1.2345, "elem_per_s": 2.345678e11}
                   for r in bench.SERVE_RATES]
    return {
        "metric": bench.METRIC, "value": 7012.123456789, "unit": "GB/s", "n_gpus": 1,
        "steps": 20, "warmup": 5, "ms_per_step": 3.6881234567, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": bench.WORKLOAD, "step_bytes": 12345678901,
                   "l2": "inputs larger than L2: each step streams 12.9 GB against a 129 MB L2",
                   "parallelism": "single GPU", "cpu_sample": bench.CPU_SAMPLE,
                   "variant_n_2e28": 43219, "variant_source": "tuned"},
        "roofline": {"bound": "hbm", "achieved": 7252.123456, "peak": 6788.3, "unit": "GB/s",
                     "frac": 1.06834567, "traffic": 5.9e9, "kernel": "long name " * 10,
                     "peak_source": "measured hbm_gbs", "frac_of_nominal_8TBs": 0.9},
        "gpu_launches": 1560,
        "tuning": {"buckets": [{"k": k, "variant": 1234} for k in range(10, 29)] * 2},
        "variants": [{"n": 1 << 20, "variant": 1}] * 38,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 13},
        "sweep": {"reps": 9, "rows": sweep_rows},
        "e2e": {"value": 287.123456, "unit": "GB/s", "h2d_bytes_per_step": 8589935000,
                "d2h_bytes_per_step": 4294967500, "steps": 3, "how": "x" * 400},
        "config1": {"gbs_l2_flushed": 3015.123, "gbs_l2_resident": 3631.2,
                    "gbs_graph_flushed": 3300.1, "us_l2_flushed": 8.3456, "n": 1 << 20},
        "streams": {"results": [{"streams": s, "gbs": 7100.123} for s in (1, 2, 4, 8)]},
        "batched": {"graph_replay": {"gbs": 6740.1234}, "per_call_launches": {"gbs": 4000.1},
                    "speedup_graph_vs_per_call": 1.6854321, "search": {"x": "y" * 3000}},
        "served": {"rates": list(bench.SERVE_RATES), "seconds_per_rate": 2.0,
                   "batched": served_rows, "serial": served_rows,
                   "batched_backfill": served_rows},
        "reduce": {"norm2": {"frac_of_peak": 0.6912345}, "dot": {"frac_of_peak": 0.80123}},
        "vecops": {"defaults": [{"op": "axpy", "gbs": 1.0}] * 40},
        "cpu_family": {"sizes": [{"n": 1, "x": "z" * 500}] * 10},
        "cpu_baseline": {"value": 31.5304689648731, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": bench.CPU_SAMPLE + "; 196 passes in 10.0 s, one thread",
                         "all_cores": {"value": 81.88144252498941, "cores": 16, "passes": 9,
                                       "how": "each call split"}},
        "extras_file": "bench_out/extras.json",
    }


def test_headline_is_compact_and_complete():
    full = fake_record()
    assert len(json.dumps(full)) > 20000  # the full record would not fit a log tail
    line = json.dumps(bench.headline(full))
    assert len(line.encode()) <= bench.HEADLINE_MAX_BYTES, len(line)
    d = json.loads(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["config"]["workload"] == bench.WORKLOAD
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in d["roofline"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in d["cpu_baseline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"], k
    assert d["e2e"]["h2d_bytes_per_step"] == 8589935000
    assert abs(d["value"] - 7012.12) < 0.01 and abs(d["roofline"]["frac"] - 1.068) < 1e-3
    legs = d["legs"]
    assert legs["n2e20_gbs"] == [3015.0, 3631.0]
    assert legs["min_frac_n_ge_2e24"] == 1.03 and legs["mixed_frac_2e28"] == 0.963
    assert len(legs["p99_ms_batched"]) == len(legs["p99_ms_serial"]) == len(bench.SERVE_RATES)
    assert legs["batch_gbs_x"] == [6740.0, 1.69]


def test_headline_without_extras():
    full = fake_record()
    for k in ("sweep", "config1", "streams", "batched", "served", "reduce", "vecops",
              "cpu_family"):
        del full[k]
    d = json.loads(json.dumps(bench.headline(full)))
    assert "legs" not in d and d["cpu_baseline"]["cores"] == 1


def test_sweep_calls_cover_every_offset_alias_pair():
    calls = bench.sweep_calls()
    assert len(calls) == 38
    assert {(o, al) for _, o, al in calls} == {(o // 8, al) for o in bench.OFFSETS
                                               for al in bench.ALIASES}
    assert sorted(n for n, _, _ in calls) == sorted(
        [(1 << k) + d for k in bench.SWEEP_K for d in (0, 3)])
    sample = bench.sweep_calls(bench.CPU_SAMPLE_K)
    assert len(sample) == 30 and max(n for n, _, _ in sample) == (1 << 24) + 3
    gb = sum(24 * n for n, _, _ in sample) / 1e9
    assert f"{gb:.2f} GB" in bench.CPU_SAMPLE


def test_in_place_alpha_is_contracting():
    for a in (-1.999, -0.5, 0.0, 1.5, 1.99999):
        assert abs(bench.call_alpha(a, "w=x")) < 1.0
        assert bench.call_alpha(a, "w=y") == a and bench.call_alpha(a, "distinct") == a
    px, py, pw = 1000, 2000, 3000
    assert bench.call_pointers(px, py, pw, 5, 1, "w=x") == (1008, 2008, 1008)
    assert bench.call_pointers(px, py, pw, 5, 1, "w=y") == (1008, 2008, 2008)
    assert bench.call_pointers(px, py, pw, 5, 1, "distinct") == (1008, 2008, 3008)


def test_served_only_rejects_unknown_modes():
    import subprocess
    r = subprocess.run([sys.executable, "bench.py", "--served-only", "batched,sideways"],
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "unknown served modes" in r.stderr
