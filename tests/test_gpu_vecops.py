"""GPU parity of the sibling vector kernels (VecAXPY, VecAYPX, VecAXPBYPCZ,
VecMAXPY, VecPointwiseMult) through the C ABI: bitwise against the oracle of
vecops_oracle.c, for pipe splits from all-FP64 to all-integer (sums and
products), every alignment class and in-place form; guard canaries around
every buffer."""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth
from gpu_util import Guarded
from test_vecops_oracle import wide

pytestmark = pytest.mark.gpu

# up to about 3M elements: several tiles per block of the persistent staged
# grid, so every block wraps around its shared-memory ring more than once
SIZES = (1, 3, 67, 4099, 262147, 3000007)


# (add offload, product sixteenths): FP64 only, each integer path alone and
# mixed, all-integer, and the defaults (-1, -1)
SPLITS = [(0, 0), (1, 0), (2, 0), (0, 16), (0, 9), (1, 5), (2, 16), (-1, -1)]


@pytest.fixture(autouse=True)
def _pipes():
    yield
    wx.wxpy_vecops_pipes(-1, -1)


def vals(seed, n, special):
    if special:
        v = wide(seed, max(n, 1))
        return np.resize(v, n).astype(np.float64)
    return synth.uniform_pm1(seed, synth.TAG_X, n)


def same(got_dev, want):
    got = got_dev.cpu().numpy()
    ok = (got.view(np.uint64) == want.view(np.uint64)) | (np.isnan(got) & np.isnan(want))
    return bool(ok.all())


@pytest.mark.parametrize("special", [False, True])
@pytest.mark.parametrize("split", SPLITS)
@pytest.mark.parametrize("offs", [(0, 0, 0), (8, 8, 8), (24, 24, 24), (0, 8, 24)])
def test_axpbypcz(split, offs, special):
    wx.wxpy_vecops_pipes(*split)
    for n in SIZES:
        xh, yh, zh = (vals(10 * n + k, n, special) for k in range(3))
        gx, gy, gz = Guarded(n, offs[0]).set(xh), Guarded(n, offs[1]).set(yh), Guarded(n, offs[2]).set(zh)
        a, b, c = 0.75, -1.25, 3.0 + 2.0 ** -50
        wx.wxpy_axpbypcz(a, b, c, gx.t, gy.t, gz.t)
        torch.cuda.synchronize()
        assert same(gz.t, oracle.axpbypcz(a, b, c, xh, yh, zh)), (n, offs)
        for g in (gx, gy, gz):
            g.check()


@pytest.mark.parametrize("special", [False, True])
@pytest.mark.parametrize("split", SPLITS)
@pytest.mark.parametrize("offs", [(0, 0), (8, 8), (0, 24)])
def test_axpby(split, offs, special):
    wx.wxpy_vecops_pipes(*split)
    for n in SIZES:
        xh, yh = (vals(20 * n + k, n, special) for k in range(2))
        gx, gy = Guarded(n, offs[0]).set(xh), Guarded(n, offs[1]).set(yh)
        a, b = -0.625, 1.5 + 2.0 ** -51
        wx.wxpy_axpby(a, b, gx.t, gy.t)
        torch.cuda.synchronize()
        assert same(gy.t, oracle.axpby(a, b, xh, yh)), (n, offs)
        for g in (gx, gy):
            g.check()


@pytest.mark.parametrize("split", SPLITS)
@pytest.mark.parametrize("m", [0, 1, 3, 8, 9, 17])
def test_maxpy(split, m):
    wx.wxpy_vecops_pipes(*split)
    for n in (5, 4099, 70001, 2000003):
        for special in (False, True):
            yh = vals(7 + n, n, special)
            xsh = [vals(100 + 13 * j + n, n, special) for j in range(m)]
            al = list(synth.uniform_pm2(5 + m, synth.TAG_ALPHA, max(m, 1))[:m])
            gy = Guarded(n, 8).set(yh)
            gxs = [Guarded(n, 8).set(x) for x in xsh]
            wx.wxpy_maxpy(al, [g.t for g in gxs], gy.t)
            torch.cuda.synchronize()
            assert same(gy.t, oracle.maxpy(al, xsh, yh)), (n, m, special)
            for g in [gy] + gxs:
                g.check()


@pytest.mark.parametrize("special", [False, True])
@pytest.mark.parametrize("mul", [-1, 16, 7])
def test_pointwise_mult_and_in_place(special, mul):
    wx.wxpy_vecops_pipes(-1, mul)
    for n in SIZES:
        xh, yh = vals(n, n, special), vals(n + 1, n, special)
        gx, gy, gw = Guarded(n, 8).set(xh), Guarded(n, 8).set(yh), Guarded(n, 24)
        wx.wxpy_pointwise_mult(gx.t, gy.t, gw.t)
        torch.cuda.synchronize()
        assert same(gw.t, oracle.pmult(xh, yh))
        wx.wxpy_pointwise_mult(gx.t, gy.t, gx.t)  # w == x
        torch.cuda.synchronize()
        assert same(gx.t, oracle.pmult(xh, yh))
        for g in (gx, gy, gw):
            g.check()


def _product_pairs():
    """(x, y) pairs aimed at the integer-pipeline product: ties to even (odd
    significands times 3/2 and 3/4), products just below and above a power of
    two (the significand product on either side of 2^105, rounding carries
    into the next binade), results at the subnormal and overflow boundaries,
    zeros, subnormals, inf and NaN, and random significands over the whole
    exponent range."""
    import pins
    xs, ys = [], []
    ulp = 2.0 ** -52
    sig = [1.0, 1.0 + ulp, 1.5, 1.5 + ulp, 2.0 - ulp, 2.0 - 2 * ulp, 1.25, 1.75 - ulp,
           1.0 + 3 * ulp, 1.4142135623730951, 1.0000000149011612]
    for k in range(1, 4000, 31):  # ties: odd significand times 3/2, 3/4
        xs += [1.0 + k * ulp, -(1.0 + k * ulp), 1.0 + k * ulp]
        ys += [1.5, 1.5, -0.75]
    for a in sig:
        for b in sig:
            for ea, eb in ((0, 0), (0, 1), (-1, 0), (500, -500), (3, -7)):
                xs.append(np.ldexp(a, ea))
                ys.append(np.ldexp(b, eb))
    # the subnormal boundary (results near 2^-1022) and the overflow one (near 2^1024)
    for a in sig:
        for b in sig:
            for ea in (-1022, -600, -511, 0, 511, 600, 1023):
                for d in (-2, -1, 0, 1):
                    eb = -1022 - ea + d
                    if -1074 <= eb <= 1023:
                        xs.append(np.ldexp(a, ea))
                        ys.append(np.ldexp(b, eb))
                    eb2 = 1023 - ea + d
                    if -1074 <= eb2 <= 1023:
                        xs.append(np.ldexp(a, ea))
                        ys.append(np.ldexp(b, eb2))
    sv = pins.special_values()
    for a in sv:
        for b in sv:
            xs.append(a)
            ys.append(b)
    rng = np.random.default_rng(5)
    m = 20000
    r = rng.uniform(1.0, 2.0, (2, m)) * rng.choice([-1.0, 1.0], (2, m))
    e = rng.integers(-540, 540, (2, m))
    xs += list(np.ldexp(r[0], e[0]))
    ys += list(np.ldexp(r[1], e[1]))
    with np.errstate(over="ignore"):
        return np.array(xs, dtype=np.float64), np.array(ys, dtype=np.float64)


def test_integer_pipeline_product_is_exact():
    """Every product in the integer pipeline: the oracle's bits (NaN by class)
    on inputs chosen to hit every branch of the integer-pipeline product, as
    pointwise_mult and as the three products of axpbypcz."""
    xh, yh = _product_pairs()
    n = len(xh)
    wx.wxpy_vecops_pipes(0, 16)
    for off in (0, 8):  # 32-byte path and the scalar one
        gx, gy, gw = Guarded(n, off).set(xh), Guarded(n, 0).set(yh), Guarded(n, off)
        wx.wxpy_pointwise_mult(gx.t, gy.t, gw.t)
        torch.cuda.synchronize()
        want = oracle.pmult(xh, yh)
        got = gw.t.cpu().numpy()
        bad = np.nonzero((got.view(np.uint64) != want.view(np.uint64)) & ~(np.isnan(got) & np.isnan(want)))[0]
        assert bad.size == 0, (f"{bad.size} differ, first x={xh[bad[0]]!r} y={yh[bad[0]]!r} "
                               f"got {got[bad[0]].hex()} want {want[bad[0]].hex()}")
        for g in (gx, gy, gw):
            g.check()
    z = np.roll(xh, 7)
    for a, b, c in ((1.5, -0.75, 1.0 + 2.0 ** -52), (2.0 ** 600, 2.0 ** -600, -3.0)):
        gx, gy, gz = Guarded(n, 0).set(xh), Guarded(n, 0).set(yh), Guarded(n, 0).set(z)
        wx.wxpy_axpbypcz(a, b, c, gx.t, gy.t, gz.t)
        torch.cuda.synchronize()
        assert same(gz.t, oracle.axpbypcz(a, b, c, xh, yh, z)), (a, b, c)


def test_bounded_wait_reports_timeout_and_context_survives():
    """The producer of the block owning tile 0 stops before copying it: that
    block's consumers give up after their one-second bound, the host reads
    WXPY_ETIMEOUT, and the next launch on the same context is exact."""
    n = 1 << 20
    xh, yh, zh = (vals(900 + k, n, False) for k in range(3))
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    z = torch.from_numpy(zh).cuda()
    wx.wxpy_vecops_status()  # clean start
    try:
        wx.wxpy_debug_vecops_drop_tile(0)
        wx.wxpy_axpbypcz(0.5, 1.5, -2.0, x, y, z)
        with pytest.raises(wx.WxpyError) as e:
            wx.wxpy_vecops_status()
        assert e.value.status == wx.WXPY_ETIMEOUT
    finally:
        wx.wxpy_debug_vecops_drop_tile(-1)
    wx.wxpy_vecops_status()  # the record was cleared
    z.copy_(torch.from_numpy(zh))
    wx.wxpy_axpbypcz(0.5, 1.5, -2.0, x, y, z)
    wx.wxpy_vecops_status()
    assert same(z, oracle.axpbypcz(0.5, 1.5, -2.0, xh, yh, zh))


def test_axpy_aypx_through_the_tuned_path():
    for n in SIZES:
        xh, yh = vals(n + 2, n, True), vals(n + 3, n, True)
        gx, gy = Guarded(n, 0).set(xh), Guarded(n, 0).set(yh)
        wx.wxpy_axpy(-0.5, gx.t, gy.t)
        torch.cuda.synchronize()
        assert same(gy.t, oracle.axpy(-0.5, xh, yh))
        gy.set(yh)
        wx.wxpy_aypx(1.5, gx.t, gy.t)
        torch.cuda.synchronize()
        assert same(gy.t, oracle.aypx(1.5, xh, yh))
        for g in (gx, gy):
            g.check()


def test_full_size_sampled():
    """n = 2^26: axpbypcz and maxpy (m = 4) on generator inputs, checked at sampled indices."""
    n = 1 << 26
    seed = synth.BASE_SEED + 40
    vs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(5)]
    for k, v in enumerate(vs):
        wx.wxpy_fill_uniform(v, seed + k, synth.TAG_X)
    idx = np.unique(np.concatenate([np.arange(64), np.arange(n - 64, n),
                                    np.random.default_rng(1).integers(0, n, 50000)]))
    host = [synth.uniform_pm1_at(seed + k, synth.TAG_X, idx) for k in range(5)]
    wx.wxpy_axpbypcz(0.5, -1.5, 1.25, vs[0], vs[1], vs[2])
    al = [0.25, -2.0, 1.5, 0.75]
    wx.wxpy_maxpy(al, [vs[0], vs[1], vs[2], vs[4]], vs[3])
    torch.cuda.synchronize()
    pos = torch.from_numpy(idx).cuda()
    z_want = oracle.axpbypcz(0.5, -1.5, 1.25, host[0], host[1], host[2])
    assert np.array_equal(vs[2][pos].cpu().numpy().view(np.uint64), z_want.view(np.uint64))
    y_want = oracle.maxpy(al, [host[0], host[1], z_want, host[4]], host[3])
    assert np.array_equal(vs[3][pos].cpu().numpy().view(np.uint64), y_want.view(np.uint64))


def test_pipe_split_search_then_parity(tmp_path):
    """Sec. 2 applied to the pipe split: every candidate verified bitwise
    against the all-FP64 split, none rejected, each winner installed and used;
    the results survive a tune-cache round trip."""
    try:
        res = wx.wxpy_vecops_tune(1 << 20)
        assert [r["op_class"] for r in res] == list(range(wx.VEC_CLASSES))
        for r in res:
            assert r["rejected"] == 0, r
            assert r["candidates"] == (9 if r["op_class"] == wx.VEC_PMULT else 11), r
            assert 0 < r["best_us"] <= r["default_us"] * 1.5, r
            assert wx.wxpy_vecops_tuned_get(r["op_class"]) == (r["add_offload"], r["mul_sixteenths"])
        n = 100003
        xh, yh, zh = (vals(700 + k, n, True) for k in range(3))
        gx, gy, gz = Guarded(n, 8).set(xh), Guarded(n, 8).set(yh), Guarded(n, 8).set(zh)
        wx.wxpy_axpbypcz(1.5, -0.5, 0.25, gx.t, gy.t, gz.t)
        torch.cuda.synchronize()
        assert same(gz.t, oracle.axpbypcz(1.5, -0.5, 0.25, xh, yh, zh))
        xs = [vals(800 + j, n, False) for j in range(5)]
        gxs = [Guarded(n, 8).set(x) for x in xs]
        gy.set(yh)
        al = [0.5, -1.0, 1.5, -2.0, 0.25]
        wx.wxpy_maxpy(al, [g.t for g in gxs], gy.t)
        torch.cuda.synchronize()
        assert same(gy.t, oracle.maxpy(al, xs, yh))
        path = str(tmp_path / "tune.json")
        wx.wxpy_tune_cache_save(path)
        wx.wxpy_tune_clear()
        assert wx.wxpy_vecops_tuned_get(0) == (-1, -1)
        wx.wxpy_tune_cache_load(path, check_device=True)
        for r in res:
            assert wx.wxpy_vecops_tuned_get(r["op_class"]) == (r["add_offload"], r["mul_sixteenths"])
    finally:
        for c in range(wx.VEC_CLASSES):
            wx.wxpy_vecops_tuned_set(c, -1, -1)


def test_stream_and_graph_capture():
    """axpbypcz and maxpy on a non-default stream, captured in a CUDA graph and
    replayed: each replay from restored inputs gives the oracle's bits."""
    n = 3 * 1024 * 256 + 13  # several staged tiles per block
    xh, yh, zh = (vals(950 + k, n, False) for k in range(3))
    x, y, z = (torch.from_numpy(a).cuda() for a in (xh, yh, zh))
    z0 = z.clone()
    xs = [torch.from_numpy(vals(960 + j, n, False)).cuda() for j in range(3)]
    al = [0.5, -1.25, 2.0]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        wx.wxpy_axpbypcz(0.75, -0.5, 1.5, x, y, z, stream=s)  # first call outside capture
        wx.wxpy_maxpy(al, xs, y, stream=s)
    s.synchronize()
    y.copy_(torch.from_numpy(yh))
    z.copy_(z0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        wx.wxpy_axpbypcz(0.75, -0.5, 1.5, x, y, z, stream=s)
        wx.wxpy_maxpy(al, xs, y, stream=s)
    z_want = oracle.axpbypcz(0.75, -0.5, 1.5, xh, yh, zh)
    y_want = oracle.maxpy(al, [t.cpu().numpy() for t in xs], yh)
    for _ in range(2):
        y.copy_(torch.from_numpy(yh))
        z.copy_(z0)
        g.replay()
        torch.cuda.synchronize()
        assert same(z, z_want) and same(y, y_want)
    wx.wxpy_vecops_status()
