"""GPU parity of the sibling vector kernels (VecAXPY, VecAYPX, VecAXPBYPCZ,
VecMAXPY, VecPointwiseMult) through the C ABI: bitwise against the oracle of
vecops_oracle.c, for every FP64-offload setting, alignment class and in-place
form; guard canaries around every buffer."""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth
from gpu_util import Guarded, bits_equal
from test_vecops_oracle import wide

pytestmark = pytest.mark.gpu

SIZES = (1, 3, 67, 4099, 262147)


@pytest.fixture(autouse=True)
def _offload():
    yield
    wx.wxpy_vecops_offload(2)


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
@pytest.mark.parametrize("offload", [0, 1, 2])
@pytest.mark.parametrize("offs", [(0, 0, 0), (8, 8, 8), (24, 24, 24), (0, 8, 24)])
def test_axpbypcz(offload, offs, special):
    wx.wxpy_vecops_offload(offload)
    for n in SIZES:
        xh, yh, zh = (vals(10 * n + k, n, special) for k in range(3))
        gx, gy, gz = Guarded(n, offs[0]).set(xh), Guarded(n, offs[1]).set(yh), Guarded(n, offs[2]).set(zh)
        a, b, c = 0.75, -1.25, 3.0 + 2.0 ** -50
        wx.wxpy_axpbypcz(a, b, c, gx.t, gy.t, gz.t)
        torch.cuda.synchronize()
        assert same(gz.t, oracle.axpbypcz(a, b, c, xh, yh, zh)), (n, offs)
        for g in (gx, gy, gz):
            g.check()


@pytest.mark.parametrize("offload", [0, 1, 2])
@pytest.mark.parametrize("m", [0, 1, 3, 8, 9, 17])
def test_maxpy(offload, m):
    wx.wxpy_vecops_offload(offload)
    for n in (5, 4099, 70001):
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
def test_pointwise_mult_and_in_place(special):
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
