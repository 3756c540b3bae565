#!/usr/bin/env python
"""Benchmark of the GB300 VecWXPY library: FP64 w = alpha*x + y.

Timed step: one pass of the size sweep through the C ABI ``wxpy()`` call,
n = 2^k and 2^k + 3 for k = 10..28 (38 calls), inputs resident in HBM.  The
start offset (the same on x, y and w) cycles 0/8/24 bytes with k, and the
alias class cycles distinct / w == x / w == y, so every (offset, alias) pair
of the sweep is timed.  ``value`` is the algorithmic bytes (24 per element:
read x, read y, write w -- in place too) of all timed steps over their device
time, in GB/s.  Each step streams 12.9 GB, far more than the 129 MB L2, so the
data of one step is gone from L2 when the next step reads it.

Output.  stdout gets ONE compact JSON line (a few KB at most): the contract's
keys (metric, value, roofline, cpu_baseline, e2e, clocks, gpu_launches, ...)
and a short summary of every other measured leg.  The full record of those
legs -- GB/s per n L2-flushed and L2-resident, the alias and mixed-offset rows,
the tuner's buckets, the stream split at n = 2^30, the batched and served
workloads, the sibling kernels, the fused reductions and the host family --
goes to the ``--extras`` file (one JSON object), and ``--jsonl`` appends one
row per measured case.

``--impl reference`` times the CPU oracle, as it stands, on the named CPU
sample of the same sweep (the calls with n <= 2^24 + 3), the sample the repo
arm's ``cpu_baseline`` times as well, and prints the same metric with
"impl": "reference".

Multi-GPU: one process per GPU (torchrun); each rank runs an independent
replica of the step on its own GPU (the operation has no exchange step), the
timing is the max over ranks and ``value`` the sum of all ranks' bytes.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "wxpy achieved HBM GB/s vs peak; batched/served elem/s and p99 vs per-call launch"
UNIT = "GB/s"
BYTES_PER_ELEM = 24
SWEEP_K = range(10, 29)
OFFSETS = (0, 8, 24)
ALIASES = ("distinct", "w=x", "w=y")
DOMINANT_K = 28
WORKLOAD = ("FP64 wxpy sweep n=2^k,2^k+3 k=10..28, offsets 0/8/24 B, "
            "alias distinct/w=x/w=y, 38 calls/step")
# The CPU sample both arms time: the sweep's calls with n <= 2^24 + 3.
CPU_SAMPLE_K = 24
CPU_SAMPLE = ("one pass = the sweep's 30 calls with k = 10..24 (n = 2^k and 2^k+3, same "
              "offsets and alias classes, 1.61 GB of algorithmic bytes), CPU oracle")
# A log tail of about 1500 characters must hold the whole stdout line.
HEADLINE_MAX_BYTES = 1400
CPU_SAMPLE_SHORT = f"n <= 2^{CPU_SAMPLE_K}+3 calls of the sweep"
EXTRAS_DEFAULT = os.path.join("bench_out", "extras.json")


def sweep_calls(max_k: int = SWEEP_K[-1]):
    """(n, element offset, alias class) of the calls of one step, k <= max_k.

    The offset cycles with k % 3; the alias class with k // 3 for the 2^k call
    and k // 3 + 1 for the 2^k + 3 call, so that all nine (offset, alias)
    pairs occur."""
    calls = []
    for k in SWEEP_K:
        if k > max_k:
            break
        for j, d in enumerate((0, 3)):
            calls.append(((1 << k) + d, OFFSETS[k % 3] // 8, ALIASES[(k // 3 + j) % 3]))
    return calls


def call_pointers(px, py, pw, n, o, alias):
    """Addresses (x, y, w) of a sweep call on buffers at px, py, pw: w is x or
    y itself for the in-place classes."""
    a, b = px + 8 * o, py + 8 * o
    c = a if alias == "w=x" else (b if alias == "w=y" else pw + 8 * o)
    return a, b, c


def call_alpha(alpha, alias):
    """alpha of a sweep call: the w = x calls use alpha / 2 (|alpha / 2| < 1),
    so that x, updated in place once per step, stays bounded however many
    steps run; the other classes use alpha."""
    return alpha * 0.5 if alias == "w=x" else alpha


# ----------------------------------------------------------------- helpers
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the single-call kernel sources; a profile summary records it, so
    that a stale ncu traffic figure is never reported against a changed kernel."""
    h = hashlib.sha256()
    for name in ("single_kernel.cuh", "fp64_emu.cuh", "fp64_mul.cuh"):
        with open(os.path.join(ROOT, "paper_1309_1894_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, scaled to n = 2^28 + 3, or None if absent or stale."""
    path = os.path.join(ROOT, "profiles", "wxpy_single_kernel_traffic.md")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    fields[k.strip()] = v.strip().split()[0]
        if fields.get("source_hash") != kernel_source_hash():
            return None
        per_elem = float(fields["dram_bytes"]) / float(fields["n"])
        return per_elem * ((1 << DOMINANT_K) + 3)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws):
    if ws <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- CPU oracle legs
class CpuSample:
    """The named CPU sample of the sweep (CPU_SAMPLE): the calls with
    k <= CPU_SAMPLE_K on host vectors from the same seeded generator, run
    through the oracle unchanged.  ``threads`` > 1 splits each call into
    contiguous chunks run by a thread pool (the same oracle function on each
    chunk)."""

    def __init__(self, threads: int = 1):
        import numpy as np
        from paper_1309_1894_gb300 import synth
        self.calls = sweep_calls(CPU_SAMPLE_K)
        nmax = max(n for n, _, _ in self.calls)
        alpha, self.x, self.y = synth.vectors(synth.BASE_SEED, nmax + 3)
        self.alpha = float(alpha)
        self.w = np.empty_like(self.x)
        self.bytes_per_pass = sum(BYTES_PER_ELEM * n for n, _, _ in self.calls)
        self.threads = threads
        self.pool = None
        if threads > 1:
            from concurrent.futures import ThreadPoolExecutor
            self.pool = ThreadPoolExecutor(threads)

    def _one(self, n, o, alias):
        import oracle
        x, y = self.x[o:o + n], self.y[o:o + n]
        w = x if alias == "w=x" else (y if alias == "w=y" else self.w[o:o + n])
        al = call_alpha(self.alpha, alias)
        if self.pool is None:
            oracle.wxpy_into(al, x, y, w)
            return
        t = self.threads
        bounds = [(n * i) // t for i in range(t + 1)]
        futs = [self.pool.submit(oracle.wxpy_into, al, x[p:q], y[p:q], w[p:q])
                for p, q in zip(bounds[:-1], bounds[1:])]
        for f in futs:
            f.result()

    def one_pass(self):
        for c in self.calls:
            self._one(*c)

    def timed(self, passes: int = 0, seconds: float = 0.0):
        """(GB/s, passes, seconds) over ``passes`` passes, or as many passes
        as fit in ``seconds`` (at least one)."""
        done = 0
        t0 = time.perf_counter()
        while True:
            self.one_pass()
            done += 1
            dt = time.perf_counter() - t0
            if (passes and done >= passes) or (not passes and dt >= seconds):
                break
        return self.bytes_per_pass * done / dt / 1e9, done, dt

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()


def cpu_baseline_leg(seconds: float):
    """The repo arm's cpu_baseline, measured in a fresh process (no CUDA
    context, no torch, none of the GPU legs' host memory), like the reference
    arm: ``bench.py --cpu-sample SECONDS`` prints the record as one line."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(seconds)],
                       capture_output=True, text=True, timeout=max(600.0, 20 * seconds))
    if r.returncode != 0:
        raise RuntimeError(f"cpu sample failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_sample_record(seconds: float):
    """The CPU sample single-threaded for about ``seconds``, then on all host
    cores for a third of that."""
    one = CpuSample(1)
    one.one_pass()  # warm-up pass: first touch of the host pages
    rate1, passes, dt = one.timed(seconds=seconds)
    one.close()
    cores = host_cores()
    allc = CpuSample(cores)
    allc.one_pass()
    rate_all, passes_all, _ = allc.timed(seconds=max(2.0, seconds / 3))
    allc.close()
    return {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{CPU_SAMPLE}; {passes} passes in {dt:.1f} s, one thread",
            "all_cores": {"value": rate_all, "cores": cores, "passes": passes_all,
                          "how": "each call split into contiguous chunks, one thread each"}}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle on the host cores: each step is one pass of the CPU sample
    (CPU_SAMPLE), the same sample the repo arm's cpu_baseline times."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    smp = CpuSample(1)
    for _ in range(max(args.warmup, 1)):
        smp.one_pass()
    value, passes, dt = smp.timed(passes=args.steps)
    smp.close()
    sample = f"{CPU_SAMPLE_SHORT}, one pass per step, one thread"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / passes * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cpu_sample": CPU_SAMPLE_SHORT},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "passes": passes},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- our arm
def lookup_ptr(wx, n, a, b, c):
    """(variant, source) that wxpy(n, ., a, b, c) runs; source 0 default, 1 tuned, 2 forced."""
    import ctypes
    info = wx.binding.VariantInfo()
    src = ctypes.c_int()
    wx.check(wx.lib().wxpy_lookup(n, a, b, c, ctypes.byref(info), ctypes.byref(src)),
             "wxpy_lookup")
    return info.as_dict(), src.value


def split_count(v, n):
    """Launches of one wxpy() call: the variant's streams, halved while a
    piece would be under 65536 elements (the rule of the stream split)."""
    s = v["streams"]
    while s > 1 and n // s < 65536:
        s //= 2
    return s


def run_ours(args):
    import torch
    import paper_1309_1894_gb300 as wx
    from paper_1309_1894_gb300 import synth

    ws, rank, local = dist_env()
    dist = init_dist(ws)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = wx.lib()
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream or None

    calls = sweep_calls()
    nmax = max(n for n, _, _ in calls)
    x = torch.empty(nmax + 8, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    w = torch.empty_like(x)
    seed = synth.BASE_SEED + rank
    wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
    wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
    alpha = synth.alpha_scalar(seed)
    px, py, pw = x.data_ptr(), y.data_ptr(), w.data_ptr()
    cargs = [(n, call_alpha(alpha, al), *call_pointers(px, py, pw, n, o, al))
             for (n, o, al) in calls]
    step_bytes = sum(BYTES_PER_ELEM * n for n, _, _ in calls)

    # The method: one empirical search per size bucket of the sweep and per
    # alias group it times (or the cells of a saved tune cache), before
    # anything is timed.
    tuning = tune_buckets(wx, args, torch)

    launches_per_step = 0
    variants = []
    for (n, al, a, b, c) in cargs:
        v, src = lookup_ptr(wx, n, a, b, c)
        launches_per_step += split_count(v, n)
        variants.append((v, src))
    dom = [i for i, (n, _, _) in enumerate(calls) if n >= (1 << DOMINANT_K)]

    def step(ev_pairs=None):
        for i, ca in enumerate(cargs):
            if ev_pairs is not None and i in dom:
                e0, e1 = ev_pairs.pop()
                e0.record(stream)
                rc = lib.wxpy(*ca, sh)
                e1.record(stream)
            else:
                rc = lib.wxpy(*ca, sh)
            if rc != 0:
                wx.check(rc, "wxpy")

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    K = args.steps
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(K * len(dom))]
    used = list(pairs)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start.record(stream)
        for _ in range(K):
            step(pairs)
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = t_start.elapsed_time(t_end)
    ms_max = max_over_ranks(dist, ms)
    total_bytes = sum_over_ranks(dist, step_bytes * K)
    value = total_bytes / (ms_max / 1e3) / 1e9

    dom_ms = sum(a.elapsed_time(b) for a, b in used)
    dom_bytes = sum(BYTES_PER_ELEM * calls[i][0] for i in dom) * K
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    peak, peak_src = load_peaks()
    traffic = profiled_traffic()
    vdom, sdom = variants[dom[0]]

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_max / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step_bytes": step_bytes,
                   "l2": "inputs larger than L2: each step streams "
                         f"{step_bytes / 1e9:.1f} GB against a 129 MB L2",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "cpu_sample": CPU_SAMPLE,
                   "variant_n_2e28": vdom["id"],
                   "variant_source": {0: "default", 1: "tuned", 2: "forced"}[sdom]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "wxpy_single_kernel, the n = 2^28 and 2^28+3 launches",
                     "peak_source": f"{peak_src} hbm_gbs",
                     "frac_of_nominal_8TBs": achieved / 8000.0},
        "gpu_launches": launches_per_step * K,
        "tuning": tuning,
        "variants": [{"n": n, "offset_bytes": 8 * o, "alias": al, "variant": v["id"],
                      "source": s, "launches": split_count(v, n)}
                     for (n, o, al), (v, s) in zip(calls, variants)],
    }
    result["clocks"] = clocks.summary()

    if rank == 0 and not args.no_extras:
        result["sweep"] = measure_sweep(wx, lib, torch, x, y, w, alpha, calls, sh, stream, peak)
        result["fp64_offload"] = measure_offload(wx, lib, torch, x, y, w, alpha, sh, stream,
                                                 peak, vdom)
    result["e2e"] = measure_e2e(wx, lib, torch, dev, alpha, calls, sh, stream, args, dist)
    del x, y, w
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_extras:
        result["config1"] = measure_config1(wx, lib, torch, dev, sh, stream, peak)
        result["streams"] = measure_streams(wx, lib, torch, dev, sh, stream, peak)
        result["batched"] = measure_batched(wx, lib, torch, dev, sh, stream, peak)
        result["vecops"] = measure_vecops(wx, torch, dev, stream, peak)
        result["reduce"] = measure_reduce(wx, torch, dev, stream, peak)
        if args.serve_seconds > 0:
            result["served"] = measure_served(args.serve_seconds)
        result["cpu_family"] = measure_cpu_family()
    if rank == 0:
        result["cpu_baseline"] = cpu_baseline_leg(args.cpu_seconds)
        if args.extras:
            d = os.path.dirname(args.extras)
            if d:
                os.makedirs(d, exist_ok=True)
            with open(args.extras, "w") as f:
                json.dump(result, f, indent=1)
            result["extras_file"] = args.extras
        if args.jsonl:
            write_jsonl(args.jsonl, result)
        print(json.dumps(headline(result)), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _r(v, digits=4):
    """A number rounded to ``digits`` significant digits (None stays None)."""
    if v is None or isinstance(v, bool) or not isinstance(v, (int, float)):
        return v
    if v == 0 or not math.isfinite(v):
        return v
    return float(f"{v:.{digits}g}")


def _pick(d, keys, digits=4):
    return {k: _r(d[k], digits) for k in keys if k in d}


def headline(result):
    """The one stdout line: the contract's keys, and a few numbers of the
    other legs; everything else stays in the extras file.  Kept under
    HEADLINE_MAX_BYTES so that a log tail of the run holds it whole."""
    line = {k: result[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup",
                                   "ms_per_step", "higher_is_better", "scaling",
                                   "vs_baseline", "dtype", "data") if k in result}
    line["value"] = _r(line.get("value"), 6)
    line["ms_per_step"] = _r(line.get("ms_per_step"), 5)
    cfg = result.get("config", {})
    line["config"] = {k: cfg[k] for k in ("workload", "parallelism", "variant_n_2e28")
                      if k in cfg}
    if "step_bytes" in cfg:
        line["config"]["l2"] = f"{cfg['step_bytes'] / 1e9:.1f} GB/step > L2, no flush"
    line["config"]["cpu_sample"] = CPU_SAMPLE_SHORT
    rf = result.get("roofline")
    if rf:
        line["roofline"] = {"bound": rf["bound"], "achieved": _r(rf["achieved"]),
                            "peak": rf["peak"], "unit": rf["unit"], "frac": _r(rf["frac"]),
                            "traffic": _r(rf["traffic"]), "kernel": "n=2^28(+3) launches"}
    cb = result.get("cpu_baseline")
    if cb:
        line["cpu_baseline"] = {"value": _r(cb["value"]), "unit": cb["unit"], "cores": cb["cores"],
                                "kind": cb["kind"], "sample": line["config"]["cpu_sample"],
                                "all_cores": _r(cb.get("all_cores", {}).get("value")),
                                "host_cores": cb.get("all_cores", {}).get("cores")}
    e = result.get("e2e")
    if e:
        line["e2e"] = {"value": _r(e["value"]), "unit": e["unit"],
                       "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": e["d2h_bytes_per_step"]}
    if "clocks" in result:
        c = result["clocks"]
        line["clocks"] = {"sm_mhz": c.get("sm_mhz"), "sm_max_mhz": c.get("sm_max_mhz"),
                          "reasons": c.get("reasons", [])}
    line["gpu_launches"] = result.get("gpu_launches")
    legs = {}
    c1 = result.get("config1")
    if c1:  # GB/s of n = 2^20: L2 flushed, L2 resident
        legs["n2e20_gbs"] = [_r(c1.get("gbs_l2_flushed"), 4), _r(c1.get("gbs_l2_resident"), 4)]
    sw = result.get("sweep")
    if isinstance(sw, dict):
        big = [r for r in sw.get("rows", []) if r["n"] >= (1 << 24) and "case" not in r]
        if big:
            legs["min_frac_n_ge_2e24"] = _r(min(r["frac_of_peak_flushed"] for r in big), 3)
        mixed = [r["frac_of_peak_flushed"] for r in sw.get("rows", [])
                 if r["n"] == (1 << DOMINANT_K) and r.get("case", "").startswith("mixed")]
        if mixed:
            legs["mixed_frac_2e28"] = _r(min(mixed), 3)
    bt = result.get("batched")
    if bt:  # graph-replayed batch GB/s, speedup over per-call launches
        legs["batch_gbs_x"] = [_r(bt["graph_replay"]["gbs"], 4),
                               _r(bt["speedup_graph_vs_per_call"], 3)]
    sv = result.get("served")
    if sv:  # p99 ms at each rate, batched then serial
        for mode, key in (("batched", "p99_ms_batched"), ("serial", "p99_ms_serial")):
            legs[key] = [_r(r["p99_ms"], 3) for r in sv.get(mode, [])]
    rd = result.get("reduce")
    if rd:
        legs["norm2_dot_frac"] = [_r(rd["norm2"]["frac_of_peak"], 3),
                                  _r(rd["dot"]["frac_of_peak"], 3)]
    if legs:
        line["legs"] = legs
    return line


def case_rows(obj, path, common):
    """One row per measured case of the bench line: every list of records under
    ``path`` becomes rows tagged ``"case": path``; scalars of a record stay in
    its row, nested records and lists are followed."""
    rows = []
    if isinstance(obj, list):
        for item in obj:
            if isinstance(item, dict):
                row = {"case": path, **common}
                row.update({k: v for k, v in item.items() if not isinstance(v, (dict, list))})
                rows.append(row)
                for k, v in item.items():
                    if isinstance(v, (dict, list)):
                        rows += case_rows(v, f"{path}.{k}", common)
    elif isinstance(obj, dict):
        flat = {k: v for k, v in obj.items() if not isinstance(v, (dict, list))}
        if flat:
            rows.append({"case": path, **common, **flat})
        for k, v in obj.items():
            if isinstance(v, (dict, list)):
                rows += case_rows(v, f"{path}.{k}" if path else k, common)
    return rows


def write_jsonl(path, result):
    """Writes the bench line's cases as JSON lines (one measured case each)."""
    common = {"metric": result.get("metric"), "n_gpus": result.get("n_gpus"),
              "time": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    rows = case_rows(result, "", common)
    with open(path, "a") as f:
        for r in rows:
            if r["case"] == "":
                r["case"] = "step"
            f.write(json.dumps(r) + "\n")


def tune_buckets(wx, args, torch):
    """Run wxpy_tune for every bucket of the sweep (n = 2^k) and both alias
    groups the step times (distinct, and in place: w = x or w = y), and for
    the x = y and mixed-offset classes at the buckets of the sweep table's
    class rows; or load the cells from --tune-cache when that file exists;
    returns a summary."""
    t0 = time.perf_counter()
    if args.tune_cache and os.path.exists(args.tune_cache):
        wx.wxpy_tune_cache_load(args.tune_cache, check_device=True)
        return {"source": f"loaded {os.path.basename(args.tune_cache)}",
                "seconds": time.perf_counter() - t0}
    if args.no_tune:
        return {"source": "built-in default variant (tuning skipped)"}
    rows = []
    # the step's classes at every bucket; the sweep table's x = y and
    # mixed-offset classes at the buckets it measures
    plan = [(k, g, f) for k in SWEEP_K
            for g, f in (("distinct", 0), ("in_place", wx.binding.TUNE_WALIAS))]
    plan += [(k, g, f) for k in (24, 26, 28)
             for g, f in (("x=y", wx.binding.TUNE_XY), ("mixed", wx.binding.TUNE_ALIGN8))]
    for k, group, flags in plan:
        r = wx.wxpy_tune(1 << k, flags)
        rows.append({"k": k, "group": group, "variant": r["best"], "us": r["best_us"],
                     "default_us": r["default_us"], "reference_us": r["reference_us"],
                     "gbs": r["best_gbs"], "candidates": r["candidates"],
                     "rejected": r["rejected"], "ties": r["ties"],
                     "launch_bound": r["launch_bound"]})
    torch.cuda.synchronize()
    if args.tune_cache:
        wx.wxpy_tune_cache_save(args.tune_cache)
    return {"source": "wxpy_tune per bucket and alias group (L2 flushed, median timing, "
                      "bitwise check against the reference variant)",
            "seconds": time.perf_counter() - t0, "buckets": rows}


def flushed_batch(n):
    """Calls per flushed timing of an n-element call: the device's event
    timestamps advance in 2.048 us steps on GB300, so a call expected to take
    under 200 us is timed as a batch of back-to-back calls on disjoint slices
    of the vectors (each slice cold after the flush), divided by its length."""
    est_us = 24.0 * n / 6.0e6 + 3.0
    return 1 if est_us >= 200.0 else int(min(64, math.ceil(200.0 / est_us)))


def time_flushed(lib, torch, stream, flush, batch, reps):
    """Median per-call ms of ``batch`` (a list of wxpy argument tuples) run
    back to back after an L2 flush, over ``reps`` runs; a device sleep is
    queued ahead of each timed run so that the host's launch latency is not
    part of the device time."""
    tf = []
    for _ in range(reps):
        flush.sum()
        torch.cuda._sleep(100000 + 30000 * len(batch))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for a in batch:
            lib.wxpy(*a)
        e1.record(stream)
        e1.synchronize()
        tf.append(e0.elapsed_time(e1) / len(batch))
    return statistics.median(tf)


def time_resident(lib, torch, stream, args, r=50):
    """Per-call ms of ``r`` back-to-back calls on the same (L2-resident) data."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    lib.wxpy(*args)
    torch.cuda._sleep(2000000)
    e0.record(stream)
    for _ in range(r):
        lib.wxpy(*args)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / r


# Extra classes of the sweep table at n = 2^24, 2^26, 2^28: (name, x, y, w
# start offsets in bytes, alias); "mixed a/b/c" has x, y, w at a, b, c bytes
# past a 256-byte boundary.  x=y moves 16 bytes per element.
CLASS_CASES = (("distinct", 0, 0, 0, "distinct"), ("w=x", 0, 0, 0, "w=x"),
               ("w=y", 0, 0, 0, "w=y"), ("x=y", 0, 0, 0, "x=y"),
               ("mixed 0/8/24", 0, 8, 24, "distinct"),
               ("mixed 8/24/0", 8, 24, 0, "distinct"),
               ("mixed 16/0/8", 16, 0, 8, "distinct"))


def class_batch(px, py, pw, numel, n, ox, oy, ow, alias):
    """(x, y, w) addresses of the calls that time one class row: the step's
    own rule (flushed_batch), so a short call is a batch of calls on disjoint
    slices of the three buffers (numel doubles each, at px, py, pw), 256-byte
    steps apart so every slice keeps the row's offsets; the alias relation
    holds within every call."""
    nb = flushed_batch(n)
    stride = 8 * ((n + 64 + 31) // 32 * 32)  # bytes
    assert max(ox, oy, ow) // 8 + (nb - 1) * stride // 8 + n <= numel
    out = []
    for i in range(nb):
        a, b, c = px + ox + i * stride, py + oy + i * stride, pw + ow + i * stride
        if alias == "w=x":
            c = a
        elif alias == "w=y":
            c = b
        elif alias == "x=y":
            b = a
        out.append((a, b, c))
    return out


def measure_sweep(wx, lib, torch, x, y, w, alpha, calls, sh, stream, peak, reps=9):
    """GB/s per call of the step, median of ``reps`` with the L2 flushed (read
    of a 512 MB buffer) before each timed run -- one call, or a batch of calls
    on disjoint slices for short calls (flushed_batch) -- and L2-resident
    (back-to-back) for n <= 2^22; then the alias and mixed-offset classes
    (CLASS_CASES) at n = 2^24, 2^26 and 2^28."""
    flush = torch.empty(64 << 20, dtype=torch.float64, device=x.device)
    flush.fill_(1.0)
    rows = []
    px, py, pw = x.data_ptr(), y.data_ptr(), w.data_ptr()
    for (n, o, al) in calls:
        al_a = call_alpha(alpha, al)
        b = flushed_batch(n)
        stride = (n + 64 + 31) // 32 * 32  # elements: 256-byte steps keep the offset class
        assert b == 1 or o + (b - 1) * stride + n <= x.numel()
        batch = [(n, al_a, *call_pointers(px, py, pw, n, o + i * stride, al), sh)
                 for i in range(b)]
        ms = time_flushed(lib, torch, stream, flush, batch, reps)
        row = {"n": n, "offset_bytes": 8 * o, "alias": al, "calls_per_flushed_run": b,
               "gbs_l2_flushed": BYTES_PER_ELEM * n / (ms / 1e3) / 1e9, "us_l2_flushed": ms * 1e3}
        if n <= (1 << 22) + 3:
            t = time_resident(lib, torch, stream, batch[0])
            row["gbs_l2_resident"] = BYTES_PER_ELEM * n / (t / 1e3) / 1e9
        row["frac_of_peak_flushed"] = row["gbs_l2_flushed"] / peak
        rows.append(row)
    for k in (24, 26, 28):
        n = 1 << k
        for (name, ox, oy, ow, al) in CLASS_CASES:
            batch = [(n, call_alpha(alpha, al), a, b, c, sh)
                     for (a, b, c) in class_batch(px, py, pw, x.numel(), n, ox, oy, ow, al)]
            nbytes = (16 if al == "x=y" else 24) * n
            v, src = lookup_ptr(wx, n, *batch[0][2:5])
            ms = time_flushed(lib, torch, stream, flush, batch, reps)
            gbs = nbytes / (ms / 1e3) / 1e9
            rows.append({"n": n, "case": name, "alias": al, "x_offset_bytes": ox,
                         "y_offset_bytes": oy, "w_offset_bytes": ow,
                         "bytes_per_elem": nbytes // n, "variant": v["id"],
                         "vec_bytes": v["vec_bytes"], "variant_source": src,
                         "calls_per_flushed_run": len(batch),
                         "gbs_l2_flushed": gbs, "us_l2_flushed": ms * 1e3,
                         "frac_of_peak_flushed": gbs / peak})
    del flush
    return {"reps": reps, "rows": rows}


def measure_config1(wx, lib, torch, dev, sh, stream, peak, reps=15, copies=16):
    """Config 1: n = 1,048,576, alpha ~ U(-2,2), x, y ~ U(-1,1) from seed, three
    separate 64-byte-aligned allocations, w distinct.  L2-flushed: ``copies``
    independent (x, y, w) sets (16 x 24 MiB, together larger than L2), the L2
    flushed, then one call on each set back to back, per-call time = total /
    copies; also replayed from a CUDA graph of those calls.  L2-resident:
    back-to-back calls on one set.  For context, torch.add(x, y, out=w) -- an
    elementwise kernel moving the same 24 bytes per element -- in the same
    flushed forms."""
    from paper_1309_1894_gb300 import synth
    n = 1 << 20
    seed = synth.BASE_SEED + 1
    alpha = synth.alpha_scalar(seed)
    sets = []
    for i in range(copies):
        xs = torch.empty(n, dtype=torch.float64, device=dev)
        ys, wss = torch.empty_like(xs), torch.empty_like(xs)
        wx.wxpy_fill_uniform(xs, seed, synth.TAG_X)
        wx.wxpy_fill_uniform(ys, seed, synth.TAG_Y)
        assert xs.data_ptr() % 64 == 0 and ys.data_ptr() % 64 == 0 and wss.data_ptr() % 64 == 0
        sets.append((xs, ys, wss))
    flush = torch.empty(64 << 20, dtype=torch.float64, device=dev)
    flush.fill_(1.0)
    batch = [(n, alpha, a.data_ptr(), b.data_ptr(), c.data_ptr(), sh) for a, b, c in sets]
    ms_f = time_flushed(lib, torch, stream, flush, batch, reps)
    ms_r = time_resident(lib, torch, stream, batch[0], r=200)
    # The same calls captured into one CUDA graph (launch gaps of the graph).
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    with torch.cuda.stream(cap):
        csh = cap.cuda_stream
        for a in batch:  # warm the capture stream's lazily created state
            lib.wxpy(*a[:-1], csh)
        cap.synchronize()
        with torch.cuda.graph(g, stream=cap):
            for a in batch:
                wx.check(lib.wxpy(*a[:-1], csh), "wxpy (capture)")
    tg = []
    for _ in range(reps):
        flush.sum()
        torch.cuda._sleep(1000000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        e1.synchronize()
        tg.append(e0.elapsed_time(e1) / copies)
    ms_g = statistics.median(tg)
    # Context, not the product: PyTorch's own elementwise kernel moving the
    # same 24 bytes per element (w = x + y in FP64) in the same two forms.
    tbatch = [(a, b, c) for a, b, c in sets]

    def torch_add():
        for a, b, c in tbatch:
            torch.add(a, b, out=c)
    tt = []
    for _ in range(reps):
        flush.sum()
        torch.cuda._sleep(1000000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch_add()
        e1.record(stream)
        e1.synchronize()
        tt.append(e0.elapsed_time(e1) / copies)
    ms_t = statistics.median(tt)
    gt = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        torch_add()
        cap.synchronize()
        with torch.cuda.graph(gt, stream=cap):
            torch_add()
    tt = []
    for _ in range(reps):
        flush.sum()
        torch.cuda._sleep(1000000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gt.replay()
        e1.record(stream)
        e1.synchronize()
        tt.append(e0.elapsed_time(e1) / copies)
    ms_tg = statistics.median(tt)
    del g, gt, sets, tbatch, flush
    gbs = lambda ms: BYTES_PER_ELEM * n / (ms / 1e3) / 1e9
    v, src = lookup_ptr(wx, *batch[0][:1], *batch[0][2:5])
    return {"n": n, "alpha": alpha, "copies": copies, "reps": reps, "variant": v["id"],
            "variant_source": src,
            "gbs_l2_flushed": gbs(ms_f), "us_l2_flushed": ms_f * 1e3,
            "gbs_l2_resident": gbs(ms_r), "us_l2_resident": ms_r * 1e3,
            "gbs_graph_flushed": gbs(ms_g), "us_graph_flushed": ms_g * 1e3,
            "torch_add_us_flushed": ms_t * 1e3, "torch_add_us_graph_flushed": ms_tg * 1e3,
            "frac_of_peak_flushed": gbs(ms_f) / peak,
            "at_peak_us": BYTES_PER_ELEM * n / (peak * 1e9) * 1e6}


def measure_offload(wx, lib, torch, x, y, w, alpha, sh, stream, peak, tuned, reps=20):
    """The tuned n = 2^28 variant with each FP64-offload setting: every sum on
    the FP64 pipeline (0), half (1) or all (2) in the integer pipeline, or
    every product in the integer pipelines (3).  On GB300 the FP64 pipeline
    caps two FP64 instructions per element near 6.2 TB/s; moving half the sums
    or every product off it lifts that ceiling."""
    n = 1 << DOMINANT_K
    out = []
    for of in (0, 1, 2, 3):
        fields = {k: v for k, v in tuned.items() if k != "id"}
        fields["fp64_offload"] = of
        vid = wx.wxpy_variant_encode(**fields)
        args = (vid, n, alpha, x.data_ptr(), y.data_ptr(), w.data_ptr(), sh)
        for _ in range(3):
            wx.check(lib.wxpy_run_variant(*args), "wxpy_run_variant")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            lib.wxpy_run_variant(*args)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = BYTES_PER_ELEM * n / (ms / 1e3) / 1e9
        out.append({"fp64_offload": of, "variant": vid, "gbs": gbs, "frac_of_peak": gbs / peak})
    return {"n": n, "reps": reps, "results": out}


def measure_e2e(wx, lib, torch, dev, alpha, calls, sh, stream, args, dist):
    """The sweep end to end from pinned host memory through the C ABI call
    wxpy_host(): per call the library copies x and y in, runs the tuned kernel
    and copies w out, chunk by chunk, overlapped on its internal streams, all
    inside the timed region; bytes counted from the copies."""
    nmax = max(n for n, _, _ in calls)
    steps = max(1, args.e2e_steps)
    hx = torch.empty(nmax + 8, dtype=torch.float64, pin_memory=True)
    hy = torch.empty_like(hx, pin_memory=True)
    hw = torch.empty_like(hx, pin_memory=True)
    hx.uniform_(-1, 1)
    hy.uniform_(-1, 1)
    h2d = sum(16 * n for n, _, _ in calls)
    d2h = sum(8 * n for n, _, _ in calls)
    px, py, pw = hx.data_ptr(), hy.data_ptr(), hw.data_ptr()
    hargs = [(n, call_alpha(alpha, al), *call_pointers(px, py, pw, n, o, al), sh)
             for (n, o, al) in calls]

    def step():
        for a in hargs:
            wx.check(lib.wxpy_host(*a), "wxpy_host")

    def run(direct):
        wx.wxpy_host_config(1 << 22, 3, direct)
        step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier(dist)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(dist, e0.elapsed_time(e1))
        total = sum_over_ranks(dist, sum(BYTES_PER_ELEM * n for n, _, _ in calls) * steps)
        return total / (ms / 1e3) / 1e9

    staged = run(False)
    direct = run(True)
    wx.wxpy_host_config(1 << 22, 3, direct > staged)  # keep the faster strategy
    del hx, hy, hw
    return {"value": max(staged, direct), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps,
            "staged_gbs": staged, "direct_gbs": direct,
            "how": "per call: wxpy_host() on pinned host x, y, w (the input bytes cross the "
                   "host link into the GPU and the result back, inside the timed region); "
                   "staged = chunked copies in, tuned kernel, copies out on three overlapped "
                   "streams; direct = the kernel reads x, y and writes w over the link "
                   "(mapped pinned memory); value = the faster"}


def batch_layout(ns):
    """Segment starts (elements) at 256-byte boundaries, and the arena length."""
    starts, pos = [], 0
    for n in ns:
        starts.append(pos)
        pos += (int(n) + 31) // 32 * 32
    return starts, pos


def measure_batched(wx, lib, torch, dev, sh, stream, peak, reps=20, per_call_reps=3):
    """4096 independent problems, n log-uniform in [1, 2^20] (about 3.1e8
    elements, 7.4 GB per batch), alpha_i ~ U(-2,2), values U(-1,1): one
    persistent segmented launch replayed from a CUDA graph, versus the same
    launch without the graph, versus 4096 wxpy() calls on one stream."""
    from paper_1309_1894_gb300 import synth
    seed = synth.BASE_SEED + 3
    ns = synth.log_uniform_lengths(seed, 4096, 1, 1 << 20)
    starts, total = batch_layout(ns)
    x = torch.empty(total, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    w = torch.empty_like(x)
    wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
    wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
    alphas = synth.uniform_pm2(seed, synth.TAG_ALPHA, len(ns))
    px, py, pw = x.data_ptr(), y.data_ptr(), w.data_ptr()
    table = wx.desc_table(ns, alphas, [px + 8 * s for s in starts], [py + 8 * s for s in starts],
                          [pw + 8 * s for s in starts])
    dt = wx.table_to_device(table)
    t0 = time.perf_counter()
    tune = wx.wxpy_batch_tune(0, 20, 0)
    tune_s = time.perf_counter() - t0
    plan = wx.wxpy_batch_plan_create(table)
    info = plan.info()
    elems = int(sum(int(n) for n in ns))
    nbytes = BYTES_PER_ELEM * elems

    def timed(fn, r):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(r):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / r

    ms_graph = timed(lambda: plan.graph_launch(dt, stream=sh), reps)
    ms_launch = timed(lambda: plan.launch(dt, stream=sh), reps)
    calls = [(int(n), float(a), px + 8 * s, py + 8 * s, pw + 8 * s)
             for n, a, s in zip(ns, alphas, starts)]

    def per_call():
        for (n, a, xa, ya, wa) in calls:
            lib.wxpy(n, a, xa, ya, wa, sh)

    ms_calls = timed(per_call, per_call_reps)
    plan.close()
    del x, y, w, dt
    torch.cuda.empty_cache()

    def row(ms):
        gbs = nbytes / (ms / 1e3) / 1e9
        return {"ms": ms, "gbs": gbs, "elem_per_s": elems / (ms / 1e3), "frac_of_peak": gbs / peak}

    return {"segments": len(ns), "elements": elems, "bytes": nbytes, "tiles": info["tiles"],
            "grid": info["grid"], "graph_replay": row(ms_graph), "persistent_launch": row(ms_launch),
            "per_call_launches": row(ms_calls), "speedup_graph_vs_per_call": ms_calls / ms_graph,
            "search": {"seconds": tune_s, "candidates": tune["candidates"],
                       "rejected": tune["rejected"], "blocks_per_sm": tune["blocks_per_sm"],
                       "mixed_gbs": tune["mixed_gbs"],
                       "shapes": {r["bucket"]: [r["tile_elems"], r["unroll"]]
                                  for r in tune["buckets"]}}}


def measure_vecops(wx, torch, dev, stream, peak, reps=10):
    """The sibling vector kernels at n = 2^26 (512 MiB per vector): GB/s of
    algorithmic bytes (axpy, aypx, pointwise_mult 24 B/element, axpbypcz 32,
    maxpy with m terms 8(m + 2)) under each operation's default pipe split,
    then axpbypcz and maxpy (m = 4, 8) under a few other splits (add offload,
    product sixteenths) to show what the split buys.  The pipe-split search
    (wxpy_vecops_tune, n = 2^24) runs first, so the default rows are the
    searched splits, as for a user who tuned."""
    n = 1 << 26
    v = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(10)]
    for k, t in enumerate(v):
        wx.wxpy_fill_uniform(t, 100 + k, 1)

    def timed(fn):
        for _ in range(2):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def row(name, nbytes, ms, **kw):
        gbs = nbytes / (ms / 1e3) / 1e9
        return dict(op=name, gbs=gbs, frac_of_peak=gbs / peak, **kw)

    def maxpy(m):
        al = [0.25 * (j + 1) for j in range(m)]
        return lambda: wx.wxpy_maxpy(al, v[1:m + 1], v[0])

    axpbypcz = lambda: wx.wxpy_axpbypcz(0.5, -0.25, 0.5, v[0], v[1], v[2])
    wx.wxpy_vecops_pipes(-1, -1)
    t0 = time.time()
    search = wx.wxpy_vecops_tune(1 << 24)
    search_s = time.time() - t0
    out = [row("axpy", 24 * n, timed(lambda: wx.wxpy_axpy(0.5, v[0], v[1]))),
           row("aypx", 24 * n, timed(lambda: wx.wxpy_aypx(0.5, v[0], v[1]))),
           row("pointwise_mult", 24 * n, timed(lambda: wx.wxpy_pointwise_mult(v[0], v[1], v[2]))),
           row("axpby", 24 * n, timed(lambda: wx.wxpy_axpby(0.5, -0.25, v[0], v[1]))),
           row("axpbypcz", 32 * n, timed(axpbypcz))]
    for m in (1, 2, 4, 8):
        out.append(row(f"maxpy_m{m}", 8 * (m + 2) * n, timed(maxpy(m))))
    splits = []
    for add, mul in ((0, 0), (1, 0), (2, 0), (0, 8), (0, 16)):
        wx.wxpy_vecops_pipes(add, mul)
        splits.append(row("axpbypcz", 32 * n, timed(axpbypcz), add_offload=add, mul_sixteenths=mul))
        for m in (4, 8):
            splits.append(row(f"maxpy_m{m}", 8 * (m + 2) * n, timed(maxpy(m)),
                              add_offload=add, mul_sixteenths=mul))
    wx.wxpy_vecops_pipes(-1, -1)
    status = "ok"
    try:
        wx.wxpy_vecops_status()
    except wx.WxpyError as e:
        status = str(e)
    del v
    torch.cuda.empty_cache()
    return {"n": n, "reps": reps, "defaults": out, "splits": splits, "wait_status": status,
            "search": {"n": 1 << 24, "seconds": search_s,
                       "classes": [{k: r[k] for k in ("op", "add_offload", "mul_sixteenths",
                                                     "candidates", "rejected", "best_us",
                                                     "default_us", "gbs")} for r in search]}}


def measure_reduce(wx, torch, dev, stream, peak, reps=10):
    """The update fused with a reduction of its result, n = 2^26: GB/s of
    algorithmic bytes (norm2: x, y read and w written, 24 B/element; dot: z
    read too, 32 B) after the configuration search (wxpy_reduce_tune, n =
    2^24), under each product split of the searched kernel (sixteenths of the
    tiles whose products run in the integer pipelines), and plain wxpy() on
    the same vectors for the cost of the fused reduction."""
    n = 1 << 26
    x, y, z = (torch.empty(n, dtype=torch.float64, device=dev) for _ in range(3))
    for k, t in enumerate((x, y, z)):
        wx.wxpy_fill_uniform(t, 300 + k, 1)
    w = torch.empty_like(x)
    res = torch.empty(1, dtype=torch.float64, device=dev)
    ws = wx.reduce_workspace(n, dev)

    def timed(fn):
        for _ in range(2):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    norm2 = lambda: wx.wxpy_norm2(-0.625, x, y, w=w, result=res, workspace=ws)
    dot = lambda: wx.wxpy_dot(-0.625, x, y, z, w=w, result=res, workspace=ws)
    gbs = lambda nbytes, ms: nbytes / (ms / 1e3) / 1e9
    # the configuration search first: the timed calls below use its winners
    t0 = time.time()
    search = wx.wxpy_reduce_tune(1 << 24)
    search_s = time.time() - t0
    splits = []
    for mul in (0, 4, 8, 12, 16):
        wx.wxpy_reduce_pipes(mul)
        splits.append({"mul_sixteenths": mul, "norm2_gbs": gbs(24 * n, timed(norm2)),
                       "dot_gbs": gbs(32 * n, timed(dot))})
    wx.wxpy_reduce_pipes(-1)
    ms_n, ms_d = timed(norm2), timed(dot)
    ms_w = timed(lambda: wx.wxpy(-0.625, x, y, w))
    out = {"n": n, "reps": reps,
           "norm2": {"gbs": gbs(24 * n, ms_n), "frac_of_peak": gbs(24 * n, ms_n) / peak, "ms": ms_n},
           "dot": {"gbs": gbs(32 * n, ms_d), "frac_of_peak": gbs(32 * n, ms_d) / peak, "ms": ms_d},
           "wxpy_alone": {"gbs": gbs(24 * n, ms_w), "ms": ms_w},
           "norm2_time_vs_wxpy": ms_n / ms_w, "splits": splits,
           "search": {"n": 1 << 24, "seconds": search_s, "kinds": search}}
    del x, y, z, w, ws
    torch.cuda.empty_cache()
    return out


def measure_cpu_family():
    """The paper's own experiment on the host cores (Sec. 3, Fig. 1): the host
    VecWXPY family's search against the baseline it reports -- the plain loop
    at -O3, vectorised by the compiler alone, one thread -- per vector size
    as in the paper's figure: n = 2^10 .. 2^20 warm (cache-resident inputs)
    and n = 2^24 (384 MiB, cache flushed).  GB/s of algorithmic bytes (24 per
    element), from the search's median times."""
    from paper_1309_1894_gb300 import build as wbuild
    from paper_1309_1894_gb300 import cpu_family as cf
    wbuild.build_cpu()
    out = {"baseline_variant": cf.describe(cf.baseline_variant()), "sizes": []}
    for n, warm in [(1 << k, True) for k in (10, 12, 14, 16, 18, 20)] + [(1 << 24, False)]:
        t0 = time.time()
        res = cf.tune(n, warm=warm)
        secs = time.time() - t0
        gbs = lambda us: 24 * n / (us * 1e3)
        out["sizes"].append({
            "n": n, "warm": warm, "search_seconds": secs, "candidates": res["candidates"],
            "rejected": res["rejected"],
            "baseline_gbs": gbs(res["baseline_us"]),
            "reference_o2_novec_gbs": gbs(res["reference_us"]),
            "best_one_thread": {"variant": res["best_single_variant"],
                                "gbs": gbs(res["best_single_us"]),
                                "speedup_vs_baseline": res["baseline_us"] / res["best_single_us"]},
            "best": {"variant": res["best_variant"], "gbs": gbs(res["best_us"]),
                     "speedup_vs_baseline": res["baseline_us"] / res["best_us"]}})
    return out


SERVE_RATES = (1e3, 5.62e3, 3.16e4, 1.78e5, 1e6)
SERVE_BACKFILL_US = 5000


SERVED_MODES = ("batched", "batched_backfill", "serial", "fused")


def measure_served(seconds, modes=SERVED_MODES):
    """Poisson arrivals at five rates from 1e3 to 1e6 requests/s, n log-uniform in
    [2^8, 2^24], alpha ~ U(-2,2), a 16 GiB admission budget, each rate for
    ``seconds``: the continuous-batching server (per batch: one fill launch
    writing the requests' x and y into their resident buffers, then one
    segmented launch reading them and writing w), the same with backfill
    admission, the serial baseline over the identical data path (per request:
    fill x, fill y, one wxpy() call), and the fused option (one kernel per
    batch generating x and y in registers; reads nothing).  elem/s counts
    completed elements; GB/s counts wxpy's 24 bytes per element (the fill
    writes 16 more in every mode but the fused one)."""
    from paper_1309_1894_gb300.server import Server, SERVE_BATCHED, SERVE_SERIAL, SERVE_FUSED
    from paper_1309_1894_gb300 import synth
    out = {"budget_gib": 16, "n_range": [1 << 8, 1 << 24], "seconds_per_rate": seconds,
           "rates": list(SERVE_RATES), "backfill_aging_us": SERVE_BACKFILL_US, "n_streams": 2}
    for name, mode, admission in (("batched", SERVE_BATCHED, 0),
                                  ("batched_backfill", SERVE_BATCHED, SERVE_BACKFILL_US),
                                  ("serial", SERVE_SERIAL, 0),
                                  ("fused", SERVE_FUSED, 0)):
        if name not in modes:
            continue
        out[name] = []
        with Server(budget_bytes=16 << 30, max_slots=4096, n_streams=2, max_batch=1024,
                    max_queue=65536, mode=mode, admission_us=admission) as sv:
            for i, rate in enumerate(SERVE_RATES):
                r = sv.loadgen(rate=rate, duration_s=seconds, n_min=1 << 8, n_max=1 << 24,
                               seed=synth.BASE_SEED + 100 + i, drain_timeout_s=120.0,
                               check_drain=False)
                st = sv.stats()
                out[name].append({
                    "head_wait_frag_s": st["head_wait_frag_s"],
                    "head_wait_full_s": st["head_wait_full_s"], "backfilled": st["backfilled"],
                    "rate": rate, "offered": r["offered"], "completed": r["completed"],
                    "rejected": r["rejected"], "failed": r["failed"],
                    "p50_ms": r["p50_s"] * 1e3, "p99_ms": r["p99_s"] * 1e3,
                    "max_ms": r["max_s"] * 1e3, "elem_per_s": r["elem_per_s"],
                    "gbs": r["gbs"], "completed_per_s": r["completed"] / r["wall_s"],
                    "max_queue": r["max_queue"], "backlog_at_end": r["backlog_at_end"],
                    "mean_batch": r["mean_batch"], "launches": r["launches"],
                    "max_inflight": st["max_inflight"], "drained": bool(r["drained"])})
    return out


def measure_streams(wx, lib, torch, dev, sh, stream, peak, reps=50, warm=10):
    """n = 2^30 (8 GiB per vector) split over 1, 2, 4, 8 streams: GB/s over
    ``reps`` back-to-back calls (each 24 GiB, far larger than L2)."""
    n = 1 << 30
    free, _ = torch.cuda.mem_get_info(dev)
    if free < 3 * 8 * n + (2 << 30):
        return {"skipped": f"needs {3 * 8 * n / 2**30:.0f} GiB free, have {free / 2**30:.0f}"}
    x = torch.empty(n, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    w = torch.empty_like(x)
    wx.wxpy_fill_uniform(x, 1, 1)
    wx.wxpy_fill_uniform(y, 1, 2)
    out = []
    for s in (1, 2, 4, 8):
        vid = wx.wxpy_variant_encode(vec_bytes=32, unroll=2, threads=256, blocks_per_sm=0,
                                     cache=1, carveout=-1, streams=s, fp64_offload=1)
        args = (vid, n, 0.5, x.data_ptr(), y.data_ptr(), w.data_ptr(), sh)
        for _ in range(warm):
            wx.check(lib.wxpy_run_variant(*args), "wxpy_run_variant")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            lib.wxpy_run_variant(*args)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps
        gbs = BYTES_PER_ELEM * n / (t / 1e3) / 1e9
        out.append({"streams": s, "ms_per_call": t, "gbs": gbs, "frac_of_peak": gbs / peak})
    del x, y, w
    torch.cuda.empty_cache()
    return {"n": n, "reps": reps, "results": out}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--jsonl", default=None,
                    help="also append one JSON line per measured case to this file")
    ap.add_argument("--extras", default=EXTRAS_DEFAULT,
                    help="write the full record of every measured leg to this JSON file "
                         "('' skips it); stdout gets the compact headline line only")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the per-n sweep and stream-split measurements")
    ap.add_argument("--no-tune", action="store_true",
                    help="time the built-in default variant instead of tuning first")
    ap.add_argument("--tune-cache", default=None,
                    help="load the tuned cells from this file if it exists, else tune and save")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="seconds of Poisson load per rate for the served leg (0 skips it)")
    ap.add_argument("--cpu-sample", type=float, default=0.0,
                    help="only time the CPU sample (the oracle) for this many seconds and print "
                         "the cpu_baseline record (the repo arm runs this in a fresh process)")
    ap.add_argument("--served-only", default="",
                    help="run only the served leg, for these comma-separated modes (batched, "
                         "batched_backfill, serial, fused) at --serve-seconds per rate, and "
                         "print its record as one JSON line")
    ap.add_argument("--single", type=int, default=0,
                    help="profiling mode: only run wxpy() on n = SINGLE, --reps times")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--variant", type=int, default=-1,
                    help="profiling mode: force this variant id instead of the tuned one "
                         "(with --vecop norm2 or dot: the reduction kernel variant)")
    ap.add_argument("--vecop", default="",
                    help="profiling mode: only run this kernel (batch: SINGLE segments; axpbypcz, axpby, maxpy4, maxpy8, "
                         "pointwise_mult, norm2, dot; serve: one 64-request server batch with "
                         "n up to SINGLE) on n = SINGLE, --reps times")
    ap.add_argument("--pipes", default="-1,-1",
                    help="profiling mode: add offload and product sixteenths for --vecop")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.cpu_sample > 0:
        print(json.dumps(cpu_sample_record(args.cpu_sample)), flush=True)
        return 0
    if args.served_only:
        modes = tuple(m.strip() for m in args.served_only.split(","))
        bad = [m for m in modes if m not in SERVED_MODES]
        if bad:
            ap.error(f"unknown served modes {bad}")
        rec = measure_served(args.serve_seconds, modes)
        if args.extras:
            d = os.path.dirname(args.extras)
            if d:
                os.makedirs(d, exist_ok=True)
            with open(args.extras, "w") as f:
                json.dump(rec, f, indent=1)
        print(json.dumps(rec), flush=True)
        return 0
    if args.single and args.vecop:
        return run_vecop(args)
    if args.single:
        return run_single(args)
    return run_ours(args)


def run_single(args):
    """A small fixed case for ncu captures: n = args.single, inputs from the
    device generator, the tuned (or default) variant, args.reps calls."""
    import torch
    import paper_1309_1894_gb300 as wx
    from paper_1309_1894_gb300 import synth
    n = args.single
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    w = torch.empty_like(x)
    wx.wxpy_fill_uniform(x, synth.BASE_SEED, synth.TAG_X)
    wx.wxpy_fill_uniform(y, synth.BASE_SEED, synth.TAG_Y)
    tuning = None
    if args.variant >= 0:
        wx.wxpy_set_variant(args.variant)
    elif args.tune_cache and os.path.exists(args.tune_cache):
        wx.wxpy_tune_cache_load(args.tune_cache, check_device=True)
    elif not args.no_tune:
        tuning = wx.wxpy_tune(n, 0)
    v, src = wx.wxpy_lookup(x, y, w)
    for _ in range(args.reps):
        wx.wxpy(0.75, x, y, w)
    torch.cuda.synchronize()
    print(json.dumps({"single": n, "reps": args.reps, "variant": v, "source": src,
                      "tuning": tuning}), flush=True)
    return 0


def run_vecop(args):
    """A small fixed case for ncu captures of a sibling kernel: n = args.single
    elements per vector from the device generator, args.reps calls."""
    import torch
    import paper_1309_1894_gb300 as wx
    from paper_1309_1894_gb300 import synth
    n = args.single
    if args.vecop == "batch":
        # one persistent segmented launch: SINGLE segments, n log-uniform in [1, 2^20]
        seed = synth.BASE_SEED + 3
        ns = synth.log_uniform_lengths(seed, n, 1, 1 << 20)
        starts, total = batch_layout(ns)
        x = torch.empty(total, dtype=torch.float64, device="cuda")
        y, w = torch.empty_like(x), torch.empty_like(x)
        wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
        wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
        alphas = synth.uniform_pm2(seed, synth.TAG_ALPHA, len(ns))
        px, py, pw = x.data_ptr(), y.data_ptr(), w.data_ptr()
        table = wx.desc_table(ns, alphas, [px + 8 * s for s in starts],
                              [py + 8 * s for s in starts], [pw + 8 * s for s in starts])
        dt = wx.table_to_device(table)
        plan = wx.wxpy_batch_plan_create(table)
        for _ in range(args.reps):
            plan.launch(dt)
        torch.cuda.synchronize()
        print(json.dumps({"vecop": "batch", "segments": n, "elements": int(sum(ns)),
                          "reps": args.reps}), flush=True)
        return 0
    nvec = {"axpbypcz": 3, "axpby": 2, "maxpy4": 5, "maxpy8": 9, "pointwise_mult": 3,
            "norm2": 3, "dot": 4, "serve": 1}[args.vecop]
    v = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(nvec)]
    for k, t in enumerate(v):
        wx.wxpy_fill_uniform(t, synth.BASE_SEED + k, synth.TAG_X)
    add, mul = (int(t) for t in args.pipes.split(","))
    wx.wxpy_vecops_pipes(add, mul)
    if args.vecop == "serve":
        # one batch through the server: 64 requests, n log-uniform in [2^8, n]
        from paper_1309_1894_gb300.server import Server
        del v
        lens = synth.log_uniform_lengths(synth.BASE_SEED + 7, 64, 1 << 8, n)
        with Server(budget_bytes=max(1 << 30, 24 * int(sum(lens)) + (64 << 20)), max_slots=64,
                    n_streams=1, max_batch=64) as sv:
            for _ in range(args.reps):
                tickets = [sv.submit(int(m), 0.75, synth.BASE_SEED + k) for k, m in enumerate(lens)]
                for t in tickets:
                    sv.wait(t)
                    sv.release(t)
        print(json.dumps({"vecop": "serve", "n_max": n, "requests": 64, "reps": args.reps,
                          "elements": int(sum(int(m) for m in lens))}), flush=True)
        return 0
    if args.vecop in ("norm2", "dot"):
        ws = wx.reduce_workspace(n)
        res = torch.empty(1, dtype=torch.float64, device="cuda")
        wx.wxpy_reduce_pipes(mul)
        wx.wxpy_reduce_variant(args.variant)  # -1: the default kernel
    for _ in range(args.reps):
        if args.vecop == "norm2":
            wx.wxpy_norm2(0.5, v[0], v[1], w=v[2], result=res, workspace=ws)
        elif args.vecop == "dot":
            wx.wxpy_dot(0.5, v[0], v[1], v[3], w=v[2], result=res, workspace=ws)
        elif args.vecop == "axpbypcz":
            wx.wxpy_axpbypcz(0.5, -0.25, 0.5, v[0], v[1], v[2])
        elif args.vecop == "axpby":
            wx.wxpy_axpby(0.5, -0.25, v[0], v[1])
        elif args.vecop == "pointwise_mult":
            wx.wxpy_pointwise_mult(v[0], v[1], v[2])
        else:
            m = nvec - 1
            wx.wxpy_maxpy([0.25 * (j + 1) for j in range(m)], v[1:], v[0])
    torch.cuda.synchronize()
    wx.wxpy_vecops_status()
    print(json.dumps({"vecop": args.vecop, "n": n, "reps": args.reps, "pipes": [add, mul]}),
          flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
