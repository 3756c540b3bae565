"""GPU parity of the update fused with a reduction (wxpy_norm2, wxpy_dot)
through the C ABI: w and the result bit for bit against the oracle of
reduce_oracle.c (NaN by class) -- sizes around every tile boundary and
several tiles per block, the staged and element paths, exact aliasing,
every product split, special values, the tree's worked examples, CUDA-graph
replay, and the full n = 2^26 case compared in full."""
import math

import numpy as np
import pytest
import torch

import oracle
import pins
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth
from gpu_util import Guarded

pytestmark = pytest.mark.gpu

T = 8192
SIZES = (0, 1, 5, T - 1, T, T + 1, 3 * T + 77, 100003, 1_000_003)


@pytest.fixture(autouse=True)
def _pipes():
    yield
    wx.wxpy_reduce_pipes(-1)
    wx.wxpy_reduce_variant(-1)
    wx.wxpy_reduce_sum_levels(-1)


def same_scalar(got, want):
    return (math.isnan(got) and math.isnan(want)) or pins.same_bits(got, want)


def same_vec(got, want):
    ok = (got.view(np.uint64) == want.view(np.uint64)) | (np.isnan(got) & np.isnan(want))
    return bool(ok.all())


def run(kind, alpha, xh, yh, zh, offs):
    n = len(xh)
    gx, gy, gw = Guarded(n, offs[0]).set(xh), Guarded(n, offs[1]).set(yh), Guarded(n, offs[2])
    gz = Guarded(n, offs[3]).set(zh) if kind == "dot" else None
    res = torch.full((1,), 12345.0, dtype=torch.float64, device="cuda")
    if kind == "dot":
        wx.wxpy_dot(alpha, gx.t, gy.t, gz.t, w=gw.t, result=res)
    else:
        wx.wxpy_norm2(alpha, gx.t, gy.t, w=gw.t, result=res)
    torch.cuda.synchronize()
    for g in (gx, gy, gw) + ((gz,) if gz else ()):
        g.check()
    return gw.t.cpu().numpy(), float(res.item())


def want(kind, alpha, xh, yh, zh):
    return oracle.wxpy_dot(alpha, xh, yh, zh) if kind == "dot" else oracle.wxpy_norm2(alpha, xh, yh)


@pytest.mark.parametrize("kind", ["norm2", "dot"])
@pytest.mark.parametrize("variant", [-1, 1, 3, 4, 6])
@pytest.mark.parametrize("mul", [-1, 0, 5, 16])
@pytest.mark.parametrize("offs", [(0, 0, 0, 0), (8, 8, 8, 8), (0, 16, 8, 24)])
def test_parity(kind, variant, mul, offs):
    wx.wxpy_reduce_variant(variant)
    wx.wxpy_reduce_pipes(mul)
    for n in SIZES:
        alpha, xh, yh = synth.vectors(synth.BASE_SEED + 500 + n, n)
        zh = synth.uniform_pm1(synth.BASE_SEED + 501 + n, synth.TAG_Y, n)
        w_got, r_got = run(kind, alpha, xh, yh, zh, offs)
        w_want, r_want = want(kind, alpha, xh, yh, zh)
        assert same_vec(w_got, w_want), (kind, n, offs)
        assert same_scalar(r_got, r_want), (kind, n, offs, r_got, r_want)


@pytest.mark.parametrize("kind", ["norm2", "dot"])
@pytest.mark.parametrize("variant", [-1, 0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("mul", [-1, 0, 7])
@pytest.mark.parametrize("offs", [(0, 0, 0, 0), (32, 64, 96, 160), (16, 16, 16, 16)])
def test_many_tiles_per_block(kind, variant, mul, offs):
    """2^24 + 12345 elements: several tiles per block of every kernel variant
    (every exchange slot and ring stage of the staged ones reused), a ragged
    last tile; the 16-byte offsets take the element path."""
    wx.wxpy_reduce_variant(variant)
    wx.wxpy_reduce_pipes(mul)
    n = (1 << 24) + 12345
    alpha, xh, yh = synth.vectors(synth.BASE_SEED + 520, n)
    zh = synth.uniform_pm1(synth.BASE_SEED + 521, synth.TAG_Y, n)
    w_got, r_got = run(kind, alpha, xh, yh, zh, offs)
    w_want, r_want = want(kind, alpha, xh, yh, zh)
    assert same_vec(w_got, w_want), (kind, offs)
    assert same_scalar(r_got, r_want), (kind, offs, r_got, r_want)


@pytest.mark.parametrize("suml", [1, 2, 3])
@pytest.mark.parametrize("mul", [0, 16])
def test_integer_tree_sums(suml, mul):
    """norm2 with the first 1..3 in-thread tree levels summed in the integer
    pipelines: every size of the parity set, several tiles per block."""
    wx.wxpy_reduce_sum_levels(suml)
    wx.wxpy_reduce_pipes(mul)
    for n in SIZES + ((1 << 24) + 12345,):
        alpha, xh, yh = synth.vectors(synth.BASE_SEED + 540 + n, n)
        w_got, r_got = run("norm2", alpha, xh, yh, None, (0, 0, 0, 0))
        w_want, r_want = oracle.wxpy_norm2(alpha, xh, yh)
        assert same_vec(w_got, w_want), n
        assert same_scalar(r_got, r_want), (n, r_got, r_want)


@pytest.mark.parametrize("variant", [4, 5, 6])
@pytest.mark.parametrize("suml", [1, 3, 4, 5, 6])
@pytest.mark.parametrize("mul", [0, 9, 16])
def test_warp_tiled_integer_tree_sums(variant, suml, mul):
    """norm2 on the warp-tiled kernels with the first 1..6 tree levels (all
    six of a thread's) summed in the integer pipelines: every size of the
    parity set and several tiles per warp with a ragged last tile."""
    wx.wxpy_reduce_variant(variant)
    wx.wxpy_reduce_sum_levels(suml)
    wx.wxpy_reduce_pipes(mul)
    for n in SIZES + ((1 << 23) + 4 * T + 5,):
        alpha, xh, yh = synth.vectors(synth.BASE_SEED + 545 + n, n)
        w_got, r_got = run("norm2", alpha, xh, yh, None, (0, 0, 0, 0))
        w_want, r_want = oracle.wxpy_norm2(alpha, xh, yh)
        assert same_vec(w_got, w_want), n
        assert same_scalar(r_got, r_want), (n, r_got, r_want)


def test_register_loaded_applies_three_levels():
    """The register-loaded kernel sums three levels inside a thread: asked for
    more it applies three and stays exact."""
    wx.wxpy_reduce_variant(0)
    wx.wxpy_reduce_sum_levels(6)
    wx.wxpy_reduce_pipes(16)
    n = 5 * T + 3
    alpha, xh, yh = synth.vectors(synth.BASE_SEED + 546, n)
    w_got, r_got = run("norm2", alpha, xh, yh, None, (0, 0, 0, 0))
    w_want, r_want = oracle.wxpy_norm2(alpha, xh, yh)
    assert same_vec(w_got, w_want) and same_scalar(r_got, r_want)


def test_bounded_wait_reports_timeout_and_context_survives():
    """The producer owning chunk 11 stops before copying it: that block's
    consumers give up after their one-second bound, the host reads
    WXPY_ETIMEOUT, and the next launch on the same context is exact."""
    n = 1 << 20
    alpha, xh, yh = synth.vectors(synth.BASE_SEED + 530, n)
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    wx.wxpy_reduce_variant(1)
    wx.wxpy_reduce_status()  # clean start
    try:
        wx.wxpy_debug_reduce_drop_chunk(11)
        wx.wxpy_norm2(alpha, x, y)
        with pytest.raises(wx.WxpyError) as e:
            wx.wxpy_reduce_status()
        assert e.value.status == wx.WXPY_ETIMEOUT
    finally:
        wx.wxpy_debug_reduce_drop_chunk(-1)
    wx.wxpy_reduce_status()  # the record was cleared
    w, res = wx.wxpy_norm2(alpha, x, y)
    wx.wxpy_reduce_status()
    w_want, r_want = oracle.wxpy_norm2(alpha, xh, yh)
    assert same_vec(w.cpu().numpy(), w_want) and same_scalar(res.item(), r_want)


@pytest.mark.parametrize("kind", ["norm2", "dot"])
@pytest.mark.parametrize("mul", [0, 16])
@pytest.mark.parametrize("suml", [0, 3, 6])
@pytest.mark.parametrize("offs", [(0, 0, 0, 0), (8, 8, 8, 8)])
@pytest.mark.parametrize("variant", [-1, 5])
def test_special_and_wide_values(kind, mul, suml, offs, variant):
    wx.wxpy_reduce_variant(variant)
    wx.wxpy_reduce_pipes(mul)
    wx.wxpy_reduce_sum_levels(suml)
    sv = np.array(pins.special_values())
    rng = np.random.default_rng(3)
    for n in (len(sv) ** 2, 3 * T + 5):
        x = np.resize(np.repeat(sv, len(sv)), n)
        y = np.resize(np.tile(sv, len(sv)), n)
        z = np.ldexp(rng.uniform(-1, 1, n), rng.integers(-300, 300, n))
        for alpha in (1.0, -0.75, 2.0 ** -600):
            w_got, r_got = run(kind, alpha, x, y, z, offs)
            w_want, r_want = want(kind, alpha, x, y, z)
            assert same_vec(w_got, w_want) and same_scalar(r_got, r_want), (kind, alpha, n, offs)
        # finite wide-exponent data: every branch of the integer product
        x = np.ldexp(rng.uniform(-1, 1, n), rng.integers(-500, 500, n))
        y = np.ldexp(rng.uniform(-1, 1, n), rng.integers(-500, 500, n))
        w_got, r_got = run(kind, 1.5, x, y, z, (0, 0, 0, 0))
        w_want, r_want = want(kind, 1.5, x, y, z)
        assert same_vec(w_got, w_want) and same_scalar(r_got, r_want)


def test_worked_examples_of_the_tree():
    """The hand-derived cases of the oracle pins, on the GPU."""
    b = 2.0 ** 53
    for vals, pos, n, expect in (([b, -b, 1.0, 1.0], [0, 1, 4096, 4097], 4098, 1.0),
                                 ([b, -b, 1.0, 1.0], [0, 1, T, T + 1], T + 2, 2.0),
                                 ([b, 1.0, 1.0, -b], [0, T, 2 * T, 4 * T], 4 * T + 1, 2.0)):
        x = np.zeros(n)
        x[pos] = vals
        _, r = run("dot", 1.0, x, np.zeros(n), np.ones(n), (0, 0, 0, 0))
        assert r == expect
    w = np.array([2.0 ** 27, 1, 0, 1, 0, 1, 0, 1])
    _, r = run("norm2", 1.0, w, np.zeros(8), None, (0, 0, 0, 0))
    assert r == 2.0 ** 54 + 4


def test_aliasing():
    n = 3 * T + 11
    alpha, xh, yh = synth.vectors(synth.BASE_SEED + 77, n)
    w_want, s_want = oracle.wxpy_norm2(alpha, xh, yh)
    for target in ("x", "y"):
        x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        w = x if target == "x" else y
        _, res = wx.wxpy_norm2(alpha, x, y, w=w)
        torch.cuda.synchronize()
        assert same_vec(w.cpu().numpy(), w_want) and same_scalar(res.item(), s_want)
    # dot with z == w: z is read (the old w) before w is written
    zh = synth.uniform_pm1(5, synth.TAG_Y, n)
    x, y, z = (torch.from_numpy(a).cuda() for a in (xh, yh, zh))
    _, d_want = oracle.wxpy_dot(alpha, xh, yh, zh)
    _, res = wx.wxpy_dot(alpha, x, y, z, w=z)
    torch.cuda.synchronize()
    assert same_vec(z.cpu().numpy(), w_want) and same_scalar(res.item(), d_want)


def test_graph_replay_and_determinism():
    n = 5 * T + 3
    alpha, xh, yh = synth.vectors(synth.BASE_SEED + 88, n)
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    w = torch.empty_like(x)
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = wx.reduce_workspace(n)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        wx.wxpy_norm2(alpha, x, y, w=w, result=res, workspace=ws, stream=s)  # warm-up outside capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        wx.wxpy_norm2(alpha, x, y, w=w, result=res, workspace=ws, stream=s)
    _, want_s = oracle.wxpy_norm2(alpha, xh, yh)
    for _ in range(3):
        res.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert same_scalar(res.item(), want_s)


def test_full_size():
    """n = 2^26 on generator inputs: w and the result compared in full."""
    n = 1 << 26
    seed = synth.BASE_SEED + 90
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    y, z = torch.empty_like(x), torch.empty_like(x)
    wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
    wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
    wx.wxpy_fill_uniform(z, seed + 1, synth.TAG_X)
    xh, yh, zh = x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy()
    for kind in ("norm2", "dot"):
        if kind == "dot":
            w, res = wx.wxpy_dot(-0.625, x, y, z)
            w_want, r_want = oracle.wxpy_dot(-0.625, xh, yh, zh)
        else:
            w, res = wx.wxpy_norm2(-0.625, x, y)
            w_want, r_want = oracle.wxpy_norm2(-0.625, xh, yh)
        torch.cuda.synchronize()
        assert same_vec(w.cpu().numpy(), w_want) and same_scalar(res.item(), r_want), kind


def test_concurrent_calls_on_separate_streams():
    """Four fused reductions in flight at once on four streams, each with its
    own workspace: every result is the oracle's."""
    cases = []
    for k in range(4):
        n = (k + 1) * T * 3 + k
        alpha, xh, yh = synth.vectors(synth.BASE_SEED + 900 + k, n)
        zh = synth.uniform_pm1(synth.BASE_SEED + 910 + k, synth.TAG_Y, n)
        x, y, z = (torch.from_numpy(a).cuda() for a in (xh, yh, zh))
        cases.append((alpha, xh, yh, zh, x, y, z, torch.cuda.Stream(), wx.reduce_workspace(n)))
    torch.cuda.synchronize()
    outs = []
    for k, (alpha, _, _, _, x, y, z, s, ws) in enumerate(cases):
        with torch.cuda.stream(s):
            if k % 2:
                outs.append(wx.wxpy_dot(alpha, x, y, z, workspace=ws, stream=s))
            else:
                outs.append(wx.wxpy_norm2(alpha, x, y, workspace=ws, stream=s))
    torch.cuda.synchronize()
    for k, ((alpha, xh, yh, zh, *_), (w, res)) in enumerate(zip(cases, outs)):
        w_want, r_want = (oracle.wxpy_dot(alpha, xh, yh, zh) if k % 2
                          else oracle.wxpy_norm2(alpha, xh, yh))
        assert same_vec(w.cpu().numpy(), w_want) and same_scalar(res.item(), r_want), k


def test_small_workspace_is_refused():
    n = 3 * T
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    ws = torch.empty(wx.lib().wxpy_reduce_workspace_bytes(n) - 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy_norm2(1.0, x, x, workspace=ws)
    assert e.value.status == wx.WXPY_EINVAL


def test_configuration_search(tmp_path):
    """wxpy_reduce_tune: every candidate verified (none rejected), the winner
    installed and used by later calls (still the oracle's bits), and saved and
    loaded with the tune cache."""
    try:
        res = wx.wxpy_reduce_tune(1 << 21)
        assert [r["op"] for r in res] == ["norm2", "dot"]
        for r in res:
            assert r["rejected"] == 0, r
            # norm2: 5 product shares, 3 tree levels at the best share and at half of it
            # (one fewer set when half equals the best), 3 staged shapes, 3 warp-tiled
            # shapes, 3 tree-level counts in the best of those; dot: 5 + 3 + 3
            if r["kind"] == 0:
                assert r["candidates"] in (5 + 3 + 3 + 3 + 3, 5 + 6 + 3 + 3 + 3), r
            else:
                assert r["candidates"] == 11 and r["sum_levels"] == 0, r
            assert 0 < r["best_us"] <= r["default_us"] * 1.5, r
            assert wx.wxpy_reduce_tuned_get(r["kind"]) == (r["variant"], r["mul_sixteenths"],
                                                           r["sum_levels"])
        n = 3 * T + 901
        alpha, xh, yh = synth.vectors(synth.BASE_SEED + 560, n)
        zh = synth.uniform_pm1(synth.BASE_SEED + 561, synth.TAG_Y, n)
        for kind in ("norm2", "dot"):
            w_got, r_got = run(kind, alpha, xh, yh, zh, (0, 0, 0, 0))
            w_want, r_want = want(kind, alpha, xh, yh, zh)
            assert same_vec(w_got, w_want) and same_scalar(r_got, r_want), kind
        path = str(tmp_path / "tune.json")
        wx.wxpy_tune_cache_save(path)
        wx.wxpy_tune_clear()
        assert wx.wxpy_reduce_tuned_get(0) == (-1, -1, -1)
        wx.wxpy_tune_cache_load(path, check_device=True)
        for r in res:
            assert wx.wxpy_reduce_tuned_get(r["kind"]) == (r["variant"], r["mul_sixteenths"],
                                                           r["sum_levels"])
    finally:
        wx.wxpy_tune_clear()


def test_squares_one_per_tile():
    """Each term of norm2 exactly: a full tile holding one nonzero element v
    (x = v, y = 0, alpha = 1, so w = v) and zeros sums to that term, RN(v*v).
    The tile sums are read from the caller-owned workspace (a 256-byte header,
    then one double per tile): the cross-tile tree works in place on its lower
    half, so the values sit in the upper half of a power-of-two tile count.
    Values aim at the integer square's branches: exact squares and ties, the
    sqrt(2) boundary where the product gains a bit, the edges of overflow and
    underflow, specials."""
    rng = np.random.default_rng(11)
    vals = list(np.ldexp(1 + rng.integers(0, 1 << 52, 1200) * 2.0 ** -52,
                         rng.integers(-520, 520, 1200)) * rng.choice([-1.0, 1.0], 1200))
    k = np.arange(1, 170, dtype=np.float64)
    vals += list((k * 2 ** 13 + 1) * 2.0 ** -30)                       # 27-bit: exact squares
    vals += list((k * 2 ** 13 + 0.5) * 2.0 ** -30)                     # 28-bit: ties
    vals += list(np.sqrt(2.0) * (1 + k * 2.0 ** -52))
    vals += list(np.nextafter(np.sqrt(2.0), 0) * (1 - k * 2.0 ** -52))
    vals += [1.3407807929942596e154, np.nextafter(1.3407807929942596e154, 0), 1.4916681462400413e-154,
             2.0 ** -511, 2.0 ** -512, 2.0 ** 511, 2.0 ** 512, 5e-324, -0.0, np.inf, np.nan, 1.0]
    vals = np.array(vals, dtype=np.float64)
    tiles = 1 << int(np.ceil(np.log2(2 * len(vals))))
    first = tiles // 2
    n = T * tiles
    xh = np.zeros(n)
    xh[(first + np.arange(len(vals))) * T + 4099] = vals
    x = torch.from_numpy(xh).cuda()
    y = torch.zeros_like(x)
    with np.errstate(over="ignore", invalid="ignore"):
        want = vals * vals
    for variant, mul, suml in ((0, 0, 0), (0, 16, 3), (4, 16, 6), (6, 0, 6)):
        wx.wxpy_reduce_variant(variant)
        wx.wxpy_reduce_pipes(mul)
        wx.wxpy_reduce_sum_levels(suml)
        ws = wx.reduce_workspace(n)
        wx.wxpy_norm2(1.0, x, y, workspace=ws)
        torch.cuda.synchronize()
        sums = ws[256 + 8 * first: 256 + 8 * (first + len(vals))].cpu().numpy().view(np.float64)
        ok = (sums.view(np.uint64) == want.view(np.uint64)) | (np.isnan(sums) & np.isnan(want))
        assert ok.all(), (variant, mul, suml, vals[~ok][:5], sums[~ok][:5], want[~ok][:5])
