"""The host VecWXPY family (libwxpy_cpu.so; the paper's own CPU experiment,
Sec. 3, Fig. 1): its exports, validation, every variant bit for bit against the
oracle (sizes across every vector width x unroll step and ragged tail, 8-byte
offsets, exact aliasing, several thread counts), and the search.  No GPU."""
import os
import subprocess

import numpy as np
import pytest

import abi
import oracle
from paper_1309_1894_gb300 import build as wbuild
from paper_1309_1894_gb300 import cpu_family as cf
from paper_1309_1894_gb300 import synth
from paper_1309_1894_gb300.binding import WxpyError


@pytest.fixture(scope="module", autouse=True)
def built():
    wbuild.build_cpu()
    cf.lib()
    cf.tune_clear()
    yield
    cf.tune_clear()


def bits_equal(got, want):
    return np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_every_declared_symbol_is_exported():
    names = abi.declared_functions("wxpy_cpu.h")
    assert "wxpy_cpu" in names and len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", cf.LIBRARY],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert not [n for n in names if n not in exported]
    assert set(names) <= set(cf.SIGNATURES)


def test_variant_space():
    count = cf.variant_count()
    ncpu = os.cpu_count() or 1
    assert count % (3 * 13) == 0
    threads = sorted({cf.describe(i)["threads"] for i in range(count // 39)})
    assert threads[0] == 1 and threads[-1] == min(ncpu, 256)
    base = cf.describe(cf.baseline_variant())
    assert (base["flavour"], base["kernel"], base["threads"]) == (1, 0, 1)
    assert base["flags"] == "-O3"
    ref = cf.describe(cf.reference_variant())
    assert (ref["flavour"], ref["kernel"], ref["threads"]) == (0, 0, 1)
    assert "-fno-tree-vectorize" in ref["flags"]
    seen = set()
    for i in range(count):
        d = cf.describe(i)
        seen.add((d["flavour"], d["kernel"], d["threads"]))
        assert (d["vec"], d["unroll"]) == ((0, 0) if d["kernel"] == 0 else
                                         ([1, 2, 4, 8][(d["kernel"] - 1) // 3],
                                          [1, 2, 4][(d["kernel"] - 1) % 3]))
    assert len(seen) == count
    with pytest.raises(WxpyError):
        cf.describe(count)


@pytest.mark.parametrize("args,status", [
    ((-1,), 1), ((10, "null"), 1), ((10, "misaligned"), 1), ((10, "partial"), 2)])
def test_validation(args, status):
    L = cf.lib()
    x = np.zeros(64)
    y = np.zeros(64)
    w = np.zeros(64)
    px, py, pw = x.ctypes.data, y.ctypes.data, w.ctypes.data
    n = args[0]
    if len(args) > 1 and args[1] == "null":
        px = None
    elif len(args) > 1 and args[1] == "misaligned":
        py += 4
    elif len(args) > 1 and args[1] == "partial":
        pw = px + 8
    assert L.wxpy_cpu(n, 1.0, px, py, pw) == status
    assert L.wxpy_cpu_run_variant(0, n, 1.0, px, py, pw) == status
    assert L.wxpy_cpu(0, 1.0, None, None, None) == 0


SIZES = [0, 1, 2, 3, 7, 8, 9, 31, 33, 67, 1000, 4099, 100003]


def variants_one_thread():
    wbuild.build_cpu()  # parametrisation runs at collection, before the fixture
    nt = cf.variant_count() // 39
    return [(f * 13 + k) * nt for f in range(3) for k in range(13)]


@pytest.mark.parametrize("vid", variants_one_thread())
def test_every_kernel_matches_oracle(vid):
    for n in SIZES:
        alpha, x, y = synth.vectors(synth.BASE_SEED + n, n)
        want = oracle.wxpy(alpha, x, y)
        assert bits_equal(cf.wxpy_cpu(alpha, x, y, variant=vid), want), (cf.describe(vid), n)
        # 8-byte offsets: views one element into larger arrays
        xb, yb, wb = np.empty(n + 1), np.empty(n + 2), np.empty(n + 3)
        xo, yo, wo = xb[1:], yb[2:], wb[3:]
        xo[:] = x
        yo[:] = y
        cf.wxpy_cpu(alpha, xo, yo, wo, variant=vid)
        assert bits_equal(wo, want)
        # exact aliasing: w == x, w == y
        xa, ya = x.copy(), y.copy()
        cf.wxpy_cpu(alpha, xa, y, xa, variant=vid)
        assert bits_equal(xa, want)
        cf.wxpy_cpu(alpha, x, ya, ya, variant=vid)
        assert bits_equal(ya, want)


def test_threaded_variants_match_oracle():
    nt = cf.variant_count() // 39
    n = 1_000_003
    alpha, x, y = synth.vectors(synth.BASE_SEED + 7, n)
    want = oracle.wxpy(alpha, x, y)
    for f, k in ((1, 0), (2, 8), (0, 12)):
        for t in range(nt):
            vid = (f * 13 + k) * nt + t
            assert bits_equal(cf.wxpy_cpu(alpha, x, y, variant=vid), want), cf.describe(vid)
    # tiny n with many threads: parts below 8 elements fall back to one thread
    alpha, x, y = synth.vectors(synth.BASE_SEED + 8, 13)
    vid = (1 * 13 + 0) * nt + nt - 1
    assert bits_equal(cf.wxpy_cpu(alpha, x, y, variant=vid), oracle.wxpy(alpha, x, y))


def test_special_values_every_flavour():
    import pins
    sv = np.array(pins.special_values())
    x = np.repeat(sv, len(sv))
    y = np.tile(sv, len(sv))
    nt = cf.variant_count() // 39
    for alpha in (1.0, -0.5, pins.DBL_MAX, 2.0 ** -1074, 0.0, -0.0):
        want = oracle.wxpy(alpha, x, y)
        for f in range(3):
            for k in (0, 3, 6, 12):
                got = cf.wxpy_cpu(alpha, x, y, variant=(f * 13 + k) * nt)
                ok = (got.view(np.uint64) == want.view(np.uint64)) | (np.isnan(got) & np.isnan(want))
                assert ok.all(), (alpha, f, k)


def test_search_then_lookup():
    res = cf.tune(1 << 16)
    assert res["rejected"] == 0
    assert res["candidates"] == 39 + cf.variant_count() // 39 - 1
    assert res["bucket"] == 16 and cf.tune_get(16) == res["best"]
    assert res["best_us"] <= res["best_single_us"] and res["baseline_us"] > 0
    alpha, x, y = synth.vectors(synth.BASE_SEED + 3, (1 << 16) + 5)
    assert bits_equal(cf.wxpy_cpu(alpha, x, y), oracle.wxpy(alpha, x, y))
    single = cf.tune(1 << 12, single_thread=True)
    assert single["best"] == single["best_single"] and single["candidates"] == 39
    assert cf.describe(single["best"])["threads"] == 1
    cf.tune_set(16, -1)
    assert cf.tune_get(16) == -1
    with pytest.raises(WxpyError):
        cf.tune_set(64, 0)
    with pytest.raises(WxpyError):
        cf.tune_set(3, cf.variant_count())


def test_tune_cache_round_trip_and_refusals(tmp_path):
    import json
    cf.tune_clear()
    cf.tune_set(12, 5)
    cf.tune_set(20, cf.variant_count() - 1)
    path = str(tmp_path / "cpu.json")
    cf.tune_cache_save(path)
    doc = json.load(open(path))
    assert doc["format"] == "wxpy-cpu-tune-1" and len(doc["entries"]) == 2
    cf.tune_clear()
    cf.tune_cache_load(path)
    assert cf.tune_get(12) == 5 and cf.tune_get(20) == cf.variant_count() - 1
    # another machine's file is refused unless the check is off
    doc["machine"] = "elsewhere"
    other = tmp_path / "other.json"
    other.write_text(json.dumps(doc))
    cf.tune_clear()
    with pytest.raises(WxpyError) as e:
        cf.tune_cache_load(str(other))
    assert e.value.status == 1 and cf.tune_get(12) == -1
    cf.tune_cache_load(str(other), check_machine=False)
    assert cf.tune_get(12) == 5
    # a malformed entry stores nothing
    doc["entries"].append({"bucket": 70, "variant": 1})
    bad = tmp_path / "bad.json"
    bad.write_text(json.dumps(doc))
    cf.tune_clear()
    with pytest.raises(WxpyError):
        cf.tune_cache_load(str(bad), check_machine=False)
    assert cf.tune_get(12) == -1
    with pytest.raises(WxpyError) as e:
        cf.tune_cache_load(str(tmp_path / "missing.json"))
    assert e.value.status == 7
    cf.tune_clear()
