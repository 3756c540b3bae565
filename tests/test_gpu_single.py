"""GPU parity of the single-call path through the C ABI: bitwise against the oracle.

The method (paper Sec. 2) accepts a variant only if its outputs equal the
reference results; here every variant family member, every alias class, every
alignment offset and ragged sizes are compared with the CPU oracle bit for bit
(w = RN(RN(alpha*x)+y), Sec. 3 / Fig. 1 vecwxpy), and guard canaries around
each buffer must stay untouched.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth
from gpu_util import Guarded, bits_equal, dev_bits_equal

pytestmark = pytest.mark.gpu

ALIASES = ["none", "w=x", "w=y", "x=y", "w=x=y"]


def make_case(n, off, alias, seed, offs=None):
    """Device vectors (x, y, w) for one case, their host inputs and the expected w."""
    alpha, xh, yh = synth.vectors(seed, n)
    ox, oy, ow = offs if offs is not None else (off, off, off)
    gx = Guarded(n, ox).set(xh)
    gy = Guarded(n, oy).set(yh)
    gw = Guarded(n, ow)
    x, y, w = gx.t, gy.t, gw.t
    guards = [gx, gy, gw]
    if alias == "w=x":
        w, guards = x, [gx, gy]
        want = oracle.wxpy(alpha, xh, yh)
    elif alias == "w=y":
        w, guards = y, [gx, gy]
        want = oracle.wxpy(alpha, xh, yh)
    elif alias == "x=y":
        y, guards = x, [gx, gw]
        want = oracle.wxpy(alpha, xh, xh)
    elif alias == "w=x=y":
        y, w, guards = x, x, [gx]
        want = oracle.wxpy(alpha, xh, xh)
    else:
        want = oracle.wxpy(alpha, xh, yh)
    return alpha, (x, y, w), (xh, yh), want, guards


def restore(alias, x, y, xh, yh):
    """Reset inputs that an in-place call overwrote."""
    if alias in ("w=x", "x=y", "w=x=y"):
        x.copy_(torch.from_numpy(xh))
    if alias == "w=y":
        y.copy_(torch.from_numpy(yh))


def covering_variants():
    """Every (vec, unroll, grid mode, cache) at 256 threads, plus every block
    size, carveout and stream count."""
    enc = wx.wxpy_variant_encode
    vs = []
    for vb in (8, 16, 32):
        for u in (1, 2, 4, 8):
            for bps in (0, 1, 8):
                for c in (0, 1, 2):
                    vs.append(enc(vec_bytes=vb, unroll=u, threads=256, blocks_per_sm=bps,
                                  cache=c, carveout=-1, streams=1))
    for t in (128, 512, 1024):
        for u in (1, 8):
            vs.append(enc(vec_bytes=32, unroll=u, threads=t, blocks_per_sm=2, cache=1,
                          carveout=-1, streams=1))
    for co in (0, 50, 100):
        vs.append(enc(vec_bytes=32, unroll=4, threads=256, blocks_per_sm=0, cache=1,
                      carveout=co, streams=1))
    for s in (2, 4, 8):
        vs.append(enc(vec_bytes=32, unroll=4, threads=256, blocks_per_sm=4, cache=1,
                      carveout=-1, streams=s))
    for of in (1, 2):  # sums in the integer pipeline
        for vb in (8, 16, 32):
            for u in (1, 2, 8):
                vs.append(enc(vec_bytes=vb, unroll=u, threads=256, blocks_per_sm=0 if u < 8 else 2,
                              cache=1, carveout=-1, streams=1, fp64_offload=of))
    return vs


def offload_variants():
    enc = wx.wxpy_variant_encode
    return [enc(vec_bytes=vb, unroll=u, threads=128, blocks_per_sm=0, cache=2, carveout=-1,
                streams=1, fp64_offload=of)
            for of in (1, 2, 3) for vb in (8, 16, 32) for u in (1, 4)]


def _special_pairs():
    """(x, y) pairs aimed at the integer-pipeline adder: every exponent gap
    0..70 with both signs, ties to even, cancellation, carries into the next
    binade, overflow and underflow of the sum, zeros, subnormals, inf, NaN."""
    import pins
    xs, ys = [], []
    base = [1.0, 1.0 + 2.0 ** -52, 1.5, 2.0 - 2.0 ** -52, 1.7976931348623157e308, 2.0 ** -1021,
            3.0, 0.1]
    for b in base:
        for d in range(0, 71):
            for sy in (1.0, -1.0):
                for tweak in (1.0, 1.0 + 2.0 ** -52, 1.5, 2.0 - 2.0 ** -52):
                    xs.append(b)
                    ys.append(sy * np.ldexp(tweak * b, -d) if b < 1e300 else sy * np.ldexp(tweak, 1000 - d))
    # ties: x + half an ulp of x, with x odd and even in the last place
    for k in range(0, 1000, 37):
        x = 1.0 + k * 2.0 ** -52
        xs += [x, x, -x]
        ys += [2.0 ** -53, -(2.0 ** -53), -(2.0 ** -53)]
    sv = pins.special_values()
    for a in sv:
        for b in sv:
            xs.append(a)
            ys.append(b)
    return np.array(xs, dtype=np.float64), np.array(ys, dtype=np.float64)


def test_integer_pipeline_sum_is_exact():
    """fp64_offload variants give the oracle's bits (NaN by class) on inputs
    chosen to hit every branch of the integer-pipeline adder (offload 1, 2)
    and the integer-pipeline product (offload 3: alpha = 1 and random alphas
    times special and wide-exponent x)."""
    import pins
    xh, yh = _special_pairs()
    cases = [(1.0, xh, yh)]
    for seed in (1, 2):
        a, x, y = pins.random_cases(synth.BASE_SEED + 300 + seed, 20000)
        cases.append((a, x, y))
    # the product's branches: alphas whose products with x run subnormal,
    # overflow, round to the next binade, or are not normal themselves
    _, xw, yw = pins.random_cases(synth.BASE_SEED + 303, 20000)
    for alpha in (-0.75, 2.0 ** -600, 2.0 ** 600, 5e-324, -3.0, 1.0 + 2.0 ** -52, 1.5 - 2.0 ** -53):
        cases.append((alpha, xh, yh))
        cases.append((alpha, np.ldexp(xw, 400), yw))
        cases.append((alpha, np.ldexp(xw, -400), yw))
    for alpha, x, y in cases:
        want = oracle.wxpy(alpha, x, y)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        for vid in offload_variants():
            w = wx.wxpy_run_variant(vid, alpha, xd, yd)
            torch.cuda.synchronize()
            got = w.cpu().numpy()
            gb, wb = got.view(np.uint64), want.view(np.uint64)
            bad = np.nonzero((gb != wb) & ~(np.isnan(got) & np.isnan(want)))[0]
            assert bad.size == 0, (
                f"variant {wx.wxpy_variant_describe(vid)}: {bad.size} differ, first alpha={alpha!r} "
                f"x={x[bad[0]]!r} y={y[bad[0]]!r} got {got[bad[0]].hex()} want {want[bad[0]].hex()}")


def test_integer_pipeline_sum_on_golden_fixture():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "special_cases.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    by_alpha = {}
    for a, x, y, w, _ in rows:
        by_alpha.setdefault(a, []).append((float.fromhex(x), float.fromhex(y), float.fromhex(w)))
    for a, trip in by_alpha.items():
        x = np.array([t[0] for t in trip])
        y = np.array([t[1] for t in trip])
        want = np.array([t[2] for t in trip])
        for vid in offload_variants():
            got = wx.wxpy_run_variant(vid, float.fromhex(a), torch.from_numpy(x).cuda(),
                                      torch.from_numpy(y).cuda()).cpu().numpy()
            ok = (got.view(np.uint64) == want.view(np.uint64)) | (np.isnan(got) & np.isnan(want))
            assert ok.all(), (a, wx.wxpy_variant_describe(vid))


@pytest.fixture(autouse=True)
def _reset_forced():
    wx.wxpy_set_variant(-1)
    yield
    wx.wxpy_set_variant(-1)


def test_device_generator_matches_host():
    """Integer-assembled symmetric ranges and the general FP64 path ((0, 1)) both
    reproduce the host generator bit for bit."""
    def u01(seed, tag, count, start=0):
        return synth.u01(seed, tag, start, count)

    for (lo, hi, host) in ((-1.0, 1.0, synth.uniform_pm1), (-2.0, 2.0, synth.uniform_pm2),
                           (0.0, 1.0, u01)):
        d = torch.empty(100003, dtype=torch.float64, device="cuda")
        wx.wxpy_fill_uniform(d, seed=synth.BASE_SEED, tag=synth.TAG_X, lo=lo, hi=hi, start=12345)
        ok, msg = bits_equal(d, host(synth.BASE_SEED, synth.TAG_X, 100003, start=12345))
        assert ok, msg


@pytest.mark.parametrize("alias", ALIASES)
@pytest.mark.parametrize("off", [0, 8, 24])
def test_every_variant_family_member(alias, off):
    vids = covering_variants()
    for n in (1, 5, 67, 4099, 262147, 600005):
        alpha, (x, y, w), (xh, yh), want, guards = make_case(n, off, alias, 1000 + n)
        want_d = torch.from_numpy(want).cuda()
        for vid in vids:
            restore(alias, x, y, xh, yh)
            wx.wxpy_run_variant(vid, alpha, x, y, w)
            torch.cuda.synchronize()
            assert dev_bits_equal(w, want_d), (
                f"variant {wx.wxpy_variant_describe(vid)} n={n} off={off} alias={alias}: "
                + bits_equal(w, want)[1])
        for g in guards:
            g.check()



@pytest.mark.parametrize("alias", ["none", "x=y"])
def test_every_compiled_instance_forced(alias):
    """Every compiled kernel instance, forced through wxpy_run_variant on
    32-byte co-aligned pointers (so nothing narrows the vector width): vector
    width x unroll x grid mode x cache policy x fp64_offload (0..3), with distinct x
    and y or x == y (the template's x == y argument), at a ragged n that has a
    head-free body, several unrolled passes and a tail."""
    enc = wx.wxpy_variant_encode
    n = 3 * 4096 + 37
    alpha, (x, y, w), (xh, yh), want, guards = make_case(n, 0, alias, synth.BASE_SEED + 77)
    count = 0
    for vb in (8, 16, 32):
        for u in (1, 2, 4, 8):
            for bps in (0, 2):  # one-shot grid, grid-stride
                for c in (0, 1, 2):
                    for of in (0, 1, 2, 3):
                        vid = enc(vec_bytes=vb, unroll=u, threads=256, blocks_per_sm=bps,
                                  cache=c, carveout=-1, streams=1, fp64_offload=of)
                        w.fill_(7.0)
                        wx.wxpy_run_variant(vid, alpha, x, y, w)
                        torch.cuda.synchronize()
                        ok, msg = bits_equal(w, want)
                        assert ok, (vb, u, bps, c, of, msg)
                        count += 1
    for g in guards:
        g.check()
    assert count == 288

MIXED_CASES = [(ox, oy, ow) for ox in (0, 8, 16, 24) for oy in (0, 8, 16, 24)
               for ow in (0, 8, 24)]


def test_every_mixed_instance_forced():
    """The mixed-alignment kernel (32-byte variants on pointers whose offsets
    disagree modulo 32 bytes): every pair of input load widths, reached through
    x, y, w offsets whose differences are 0, 8, 16 and 24 bytes, with w's own
    offset moving the head peel; unroll 1/2/4, the non-coherent and coherent
    cache forms, fp64_offload 0/1/3, one-shot and grid-stride grids; at a ragged n
    with several passes and a tail.  Bit for bit against the oracle, guards
    untouched."""
    enc = wx.wxpy_variant_encode
    n = 3 * 4096 + 37
    runs = 0
    pairs = set()
    for (ox, oy, ow) in MIXED_CASES:
        rx, ry = (ox - ow) % 32, (oy - ow) % 32
        if rx == 0 and ry == 0:
            continue
        if (rx, ry) in pairs and ow != 8:
            continue  # each width pair with two different w offsets is enough
        pairs.add((rx, ry))
        alpha, (x, y, w), _, want, guards = make_case(n, 0, "none", 900 + ox + 3 * oy + 7 * ow,
                                                      offs=(ox, oy, ow))
        want_d = torch.from_numpy(want).cuda()
        for u in (1, 2, 4):
            for c in (1, 2):
                for of in (0, 1, 3):
                    for bps in (0, 2):
                        vid = enc(vec_bytes=32, unroll=u, threads=256, blocks_per_sm=bps,
                                  cache=c, carveout=-1, streams=1, fp64_offload=of)
                        w.fill_(7.0)
                        wx.wxpy_run_variant(vid, alpha, x, y, w)
                        torch.cuda.synchronize()
                        assert dev_bits_equal(w, want_d), (ox, oy, ow, u, c, of, bps)
                        runs += 1
        for g in guards:
            g.check()
    assert len(pairs) == 15 and runs >= 15 * 36


@pytest.mark.parametrize("alias,offs", [("x=y", (8, 8, 0)), ("x=y", (16, 16, 0)),
                                        ("x=y", (0, 0, 24)), ("w=x", (8, 0, 8)),
                                        ("w=x", (16, 8, 16)), ("w=y", (0, 24, 24)),
                                        ("w=y", (8, 16, 16))])
def test_mixed_kernel_aliasing(alias, offs):
    """x == y offset from w, and in-place calls (w == x, w == y) whose other
    input is offset from w: the mixed kernel under every unroll and cache form."""
    enc = wx.wxpy_variant_encode
    for n in (5, 4099, 70001):
        alpha, (x, y, w), (xh, yh), want, guards = make_case(n, 0, alias, 31 + n, offs=offs)
        for u in (1, 2, 4):
            for c in (0, 1, 2):
                vid = enc(vec_bytes=32, unroll=u, threads=256, blocks_per_sm=0,
                          cache=c, carveout=-1, streams=1, fp64_offload=1)
                restore(alias, x, y, xh, yh)
                wx.wxpy_run_variant(vid, alpha, x, y, w)
                torch.cuda.synchronize()
                ok, msg = bits_equal(w, want)
                assert ok, (alias, offs, n, u, c, msg)
        for g in guards:
            g.check()


@pytest.mark.parametrize("alias", ALIASES)
def test_tiny_sizes_exhaustive(alias):
    """n = 0..67 at every 8-byte offset, default lookup and reference variant."""
    for off in (0, 8, 16, 24):
        for n in range(68):
            alpha, (x, y, w), (xh, yh), want, guards = make_case(n, off, alias, 77 + n)
            wx.wxpy(alpha, x, y, w)
            torch.cuda.synchronize()
            ok, msg = bits_equal(w, want)
            assert ok, f"n={n} off={off} {msg}"
            restore(alias, x, y, xh, yh)
            wx.wxpy_reference(alpha, x, y, w)
            torch.cuda.synchronize()
            ok, msg = bits_equal(w, want)
            assert ok, f"reference n={n} off={off} {msg}"
            for g in guards:
                g.check()


@pytest.mark.parametrize("offs", [(0, 8, 24), (8, 0, 24), (24, 8, 0), (0, 16, 8), (16, 0, 0),
                                  (8, 8, 24), (0, 0, 8)])
def test_mixed_offsets(offs):
    vids = covering_variants()[::5]
    for n in (3, 1001, 70001):
        alpha, (x, y, w), _, want, guards = make_case(n, 0, "none", 5 + n, offs=offs)
        want_d = torch.from_numpy(want).cuda()
        for vid in [None] + vids:
            w.zero_()
            if vid is None:
                wx.wxpy(alpha, x, y, w)
            else:
                wx.wxpy_run_variant(vid, alpha, x, y, w)
            torch.cuda.synchronize()
            assert dev_bits_equal(w, want_d), f"offs={offs} n={n} vid={vid}"
        for g in guards:
            g.check()


def test_size_sweep_default_lookup():
    """n = 2^k and 2^k + 3, k = 10..22, offsets 0/8/24, against the oracle (full compare)."""
    for k in range(10, 23):
        for n in (1 << k, (1 << k) + 3):
            for off in (0, 8, 24):
                alpha, (x, y, w), _, want, guards = make_case(n, off, "none", k * 10 + off)
                wx.wxpy(alpha, x, y, w)
                torch.cuda.synchronize()
                ok, msg = bits_equal(w, want)
                assert ok, f"n={n} off={off}: {msg}"
                for g in guards:
                    g.check()


def sampled_check(n, alpha, x, y, w, seed, xy_same=False, samples=200000):
    """Compare w at sampled indices (plus both ends) with the oracle on the same
    inputs, regenerated on the host from the counter-based generator."""
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([np.arange(min(n, 4096)),
                                    np.arange(max(0, n - 4096), n),
                                    rng.integers(0, n, samples)]))
    xs = _values_at(seed, synth.TAG_X, idx)
    ys = xs if xy_same else _values_at(seed, synth.TAG_Y, idx)
    want = oracle.wxpy(alpha, xs, ys)
    got = w[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), \
        f"{int(np.sum(got.view(np.uint64) != want.view(np.uint64)))} sampled mismatches"


def _values_at(seed, tag, idx):
    """U(-1,1) values of stream (seed, tag) at arbitrary indices (counter-based access)."""
    return synth.uniform_pm1_at(seed, tag, idx)


@pytest.mark.parametrize("n", [(1 << 24) + 3, (1 << 28) + 3])
def test_full_size_sampled(n):
    """The sizes the benchmark times, in its launch configuration (default lookup)."""
    seed = synth.BASE_SEED + 2
    alpha = synth.alpha_scalar(seed)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    w = torch.full_like(x, float("nan"))
    wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
    wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
    wx.wxpy(alpha, x, y, w)
    torch.cuda.synchronize()
    assert not bool(torch.isnan(w).any())
    sampled_check(n, alpha, x, y, w, seed)
    del x, y, w
    torch.cuda.empty_cache()


def test_bench_dominant_call_compared_in_full():
    """The benchmark's dominant call as it is timed: n = 2^28 + 3, start offset
    8 bytes, in place (w == x), alpha / 2, the variant the search picks for that
    cell -- every one of the 268,435,459 results compared with the oracle on
    host inputs from the seeded generator, chunk by chunk."""
    n = (1 << 28) + 3
    seed = synth.BASE_SEED
    alpha = synth.alpha_scalar(seed) * 0.5
    wx.wxpy_tune(1 << 28, wx.TUNE_WALIAS | wx.TUNE_QUICK)
    try:
        buf = torch.empty(n + 1, dtype=torch.float64, device="cuda")
        ybuf = torch.empty(n + 1, dtype=torch.float64, device="cuda")
        # x and y 8 bytes past a 256-byte boundary, like the benchmark's 2^28 + 3 call
        x, y = buf[1:], ybuf[1:]
        wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
        wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
        v, src = wx.wxpy_lookup(x, y, x)
        assert src == 1
        wx.wxpy(alpha, x, y, x)
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        del buf, ybuf, x, y
        torch.cuda.empty_cache()
        chunk = 1 << 24
        for start in range(0, n, chunk):
            m = min(chunk, n - start)
            xh = synth.uniform_pm1(seed, synth.TAG_X, m, start=start)
            yh = synth.uniform_pm1(seed, synth.TAG_Y, m, start=start)
            want = oracle.wxpy(alpha, xh, yh)
            ok, msg = bits_equal(torch.from_numpy(got[start:start + m]), want)
            assert ok, (start, v, msg)
    finally:
        wx.wxpy_tune_clear()


def test_large_split_streams_sampled():
    """n = 2^30 (8 GiB per vector) through the 8-stream split, sampled."""
    n = 1 << 30
    seed = synth.BASE_SEED + 4
    alpha = synth.alpha_scalar(seed)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    w = torch.full_like(x, float("nan"))
    wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
    wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
    vid = wx.wxpy_variant_encode(vec_bytes=32, unroll=4, threads=256, blocks_per_sm=0,
                                 cache=1, carveout=-1, streams=8)
    wx.wxpy_run_variant(vid, alpha, x, y, w)
    torch.cuda.synchronize()
    assert not bool(torch.isnan(w).any())
    sampled_check(n, alpha, x, y, w, seed, samples=100000)
    del x, y, w
    torch.cuda.empty_cache()


def test_non_default_stream_and_graph_capture():
    n = 300001
    alpha, (x, y, w), _, want, guards = make_case(n, 8, "none", 4242)
    want_d = torch.from_numpy(want).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        wx.wxpy(alpha, x, y, w)
    s.synchronize()
    assert dev_bits_equal(w, want_d)
    # capture a split variant (fork/join across internal streams) in a CUDA graph
    vid = wx.wxpy_variant_encode(vec_bytes=32, unroll=2, threads=512, blocks_per_sm=0,
                                 cache=1, carveout=-1, streams=4)
    w.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        wx.wxpy_run_variant(vid, alpha, x, y, w)
    for _ in range(3):
        w.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert dev_bits_equal(w, want_d)
    for gd in guards:
        gd.check()


def test_injected_launch_error_is_reported_and_cleared():
    n = 1000
    alpha, (x, y, w), _, want, _ = make_case(n, 0, "none", 9)
    wx.wxpy_debug_inject_launch_error(719, 1)  # cudaErrorLaunchFailure
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy(alpha, x, y, w)
    assert e.value.status == wx.WXPY_ECUDA
    assert wx.lib().wxpy_last_cuda_error() == 719
    wx.wxpy(alpha, x, y, w)  # the next call is not affected
    torch.cuda.synchronize()
    assert bits_equal(w, want)[0]
    wx.wxpy_debug_inject_launch_error(0, 0)


def test_lookup_reports_adjusted_variant():
    n = 1000
    _, (x, y, w), _, _, _ = make_case(n, 8, "none", 1, offs=(0, 8, 8))
    v, src = wx.wxpy_lookup(x, y, w)
    # the default's 32-byte width on a mixed class: the mixed-alignment kernel
    assert src == 0 and v["vec_bytes"] == 32 and v["unroll"] <= 4
    wx.wxpy_set_variant(wx.wxpy_variant_encode(vec_bytes=16, unroll=8, threads=256,
                                               blocks_per_sm=0, cache=0, carveout=-1,
                                               streams=1, fp64_offload=2))
    v, src = wx.wxpy_lookup(x, y, w)
    assert src == 2 and v["vec_bytes"] == 8 and v["unroll"] == 8  # narrowed, not mixed
    wx.wxpy_set_variant(-1)
    _, (x, y, w), _, _, _ = make_case(n, 0, "w=x", 1)
    v, src = wx.wxpy_lookup(x, y, w)
    assert v["cache"] != 1
    wx.wxpy_set_variant(5)
    v, src = wx.wxpy_lookup(x, y, w)
    assert src == 2


def test_device_query():
    d = wx.wxpy_device_query()
    assert d["sm_count"] > 0 and d["l2_bytes"] > 0
    assert (d["cc_major"], d["cc_minor"]) >= (10, 0)
