"""Runs every empirical search of the library on the current GPU and saves the
results in one tune cache (paper Sec. 2: the variants are run, checked against
the reference results and timed once, and the selected ones are kept).

    python -m paper_1309_1894_gb300.tune_all --cache tune.json

Later processes load the file with ``wxpy_tune_cache_load`` or through the
``WXPY_TUNE_CACHE`` environment variable; the file records the device it was
tuned on and is refused on another.  The searches are:

- ``wxpy_tune`` for every size bucket 2^kmin .. 2^kmax and every requested call
  class (common alignment 32 / 16 / 8 bytes, x == y, w == x);
- ``wxpy_batch_tune`` (tile shapes of the batched launch, its grid);
- ``wxpy_vecops_tune`` (the sibling kernels' pipe split);
- ``wxpy_reduce_tune`` (the fused reductions' configuration).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

from . import binding as wx

CLASSES = {
    "aligned": 0,
    "align16": wx.TUNE_ALIGN16,
    "align8": wx.TUNE_ALIGN8,
    "xy": wx.TUNE_XY,
    "walias": wx.TUNE_WALIAS,
}


def tune_all(cache: str | None = None, kmin: int = 10, kmax: int = 28,
             classes: tuple[str, ...] = ("aligned",), quick: bool = False,
             batch: bool = True, vecops_n: int = 1 << 24, reduce_n: int = 1 << 24) -> dict:
    """Runs the searches and, when ``cache`` is given, saves the tune cache there.
    Returns a summary: per search its seconds and winners."""
    if not 0 <= kmin <= kmax <= 40:
        raise ValueError("need 0 <= kmin <= kmax <= 40")
    unknown = [c for c in classes if c not in CLASSES]
    if unknown:
        raise ValueError(f"unknown call classes {unknown}; choose from {sorted(CLASSES)}")
    flags_extra = wx.TUNE_QUICK if quick else 0
    out: dict = {"buckets": []}
    t0 = time.perf_counter()
    for name in classes:
        for k in range(kmin, kmax + 1):
            r = wx.wxpy_tune(1 << k, CLASSES[name] | flags_extra)
            out["buckets"].append({"class": name, "k": k, "variant": r["best"]["id"],
                                   "us": r["best_us"], "default_us": r["default_us"],
                                   "candidates": r["candidates"], "rejected": r["rejected"]})
    out["wxpy_seconds"] = time.perf_counter() - t0
    if batch:
        t0 = time.perf_counter()
        b = wx.wxpy_batch_tune(0, min(20, kmax), 0)
        out["batch"] = {"seconds": time.perf_counter() - t0, "blocks_per_sm": b["blocks_per_sm"],
                        "fp64_offload": b["fp64_offload"], "candidates": b["candidates"],
                        "rejected": b["rejected"]}
    if vecops_n > 0:
        t0 = time.perf_counter()
        v = wx.wxpy_vecops_tune(vecops_n)
        out["vecops"] = {"seconds": time.perf_counter() - t0,
                         "classes": [{"op": r["op"], "add_offload": r["add_offload"],
                                      "mul_sixteenths": r["mul_sixteenths"]} for r in v]}
    if reduce_n > 0:
        t0 = time.perf_counter()
        rr = wx.wxpy_reduce_tune(reduce_n)
        out["reduce"] = {"seconds": time.perf_counter() - t0,
                         "kinds": [{"op": r["op"], "variant": r["variant"],
                                    "mul_sixteenths": r["mul_sixteenths"],
                                    "sum_levels": r["sum_levels"]} for r in rr]}
    if cache:
        wx.wxpy_tune_cache_save(cache)
        out["cache"] = cache
    return out


def main(argv: list[str] | None = None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--cache", required=True, help="tune cache file to write")
    ap.add_argument("--kmin", type=int, default=10)
    ap.add_argument("--kmax", type=int, default=28)
    ap.add_argument("--classes", default="aligned",
                    help="comma-separated call classes: " + ", ".join(sorted(CLASSES))
                    + ", or all")
    ap.add_argument("--quick", action="store_true", help="the narrower wxpy search")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--vecops-n", type=int, default=1 << 24, help="0 skips the sibling search")
    ap.add_argument("--reduce-n", type=int, default=1 << 24, help="0 skips the reduction search")
    a = ap.parse_args(argv)
    classes = tuple(sorted(CLASSES)) if a.classes == "all" else tuple(a.classes.split(","))
    summary = tune_all(a.cache, a.kmin, a.kmax, classes, a.quick, not a.no_batch, a.vecops_n,
                       a.reduce_n)
    print(json.dumps(summary), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
