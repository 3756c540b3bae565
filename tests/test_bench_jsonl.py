"""bench.py's per-case JSON lines (--jsonl) on the CPU: every list of records
in the bench line becomes rows tagged with its path, scalars stay in their
row, and the top-level step is its own row."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_case_rows_and_file(tmp_path):
    line = {"metric": "m", "value": 1.5, "n_gpus": 1,
            "roofline": {"frac": 1.07, "unit": "GB/s"},
            "sweep": [{"n": 1024, "gbs": 6.0}, {"n": 2048, "gbs": 12.0}],
            "reduce": {"norm2": {"gbs": 4477.0},
                       "search": {"kinds": [{"kind": 0, "variant": 0}, {"kind": 1, "variant": 0}]}}}
    path = tmp_path / "cases.jsonl"
    bench.write_jsonl(str(path), line)
    rows = [json.loads(t) for t in path.read_text().splitlines()]
    cases = [r["case"] for r in rows]
    assert cases.count("sweep") == 2 and cases.count("reduce.search.kinds") == 2
    assert {"step", "roofline", "reduce.norm2"} <= set(cases)
    step = next(r for r in rows if r["case"] == "step")
    assert step["value"] == 1.5 and "sweep" not in step
    assert [r["n"] for r in rows if r["case"] == "sweep"] == [1024, 2048]
    assert all(r["metric"] == "m" for r in rows)
