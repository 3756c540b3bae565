"""Programmatic dependent launch of the single-call kernels (GPU, C ABI).

With it on, a kernel may be scheduled while the previous kernel of its stream
still runs, and waits on the device for that kernel's completion before it
touches memory.  Chains of calls where each call reads what the previous one
wrote (in place, and ping-pong between two buffers) must give the oracle's
bits with it on and off, for one-block, multi-block, multi-wave and
stream-split calls, eagerly and replayed from a CUDA graph.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [1, 1027, (1 << 20) + 3, 1 << 22]


def chain_oracle(alphas, xh, yh):
    """x <- RN(RN(a*x) + y) for each a in turn (the in-place chain)."""
    x = xh.copy()
    for a in alphas:
        oracle.wxpy_into(a, x, yh, x)
    return x


def pingpong_oracle(alphas, xh, yh):
    """a -> b -> a ...: b = wxpy(al, a, y), then a = wxpy(al', b, y), ..."""
    bufs = [xh.copy(), np.empty_like(xh)]
    for k, a in enumerate(alphas):
        oracle.wxpy_into(a, bufs[k % 2], yh, bufs[(k + 1) % 2])
    return bufs[len(alphas) % 2]


@pytest.fixture(autouse=True)
def restore_pdl():
    prev = wx.wxpy_launch_pdl(-1)
    yield
    wx.wxpy_launch_pdl(prev)
    wx.wxpy_set_variant(-1)


@pytest.mark.parametrize("pdl", [1, 0])
@pytest.mark.parametrize("n", SIZES)
def test_dependent_chains_eager(pdl, n):
    wx.wxpy_launch_pdl(pdl)
    assert wx.wxpy_launch_pdl(-1) == pdl
    seed = synth.BASE_SEED + 700 + n % 97
    _, xh, yh = synth.vectors(seed, n)
    alphas = [float(a) * 0.5 for a in synth.uniform_pm2(seed, synth.TAG_ALPHA, 12)]
    x = torch.from_numpy(xh).cuda()
    y = torch.from_numpy(yh).cuda()
    for a in alphas:
        wx.wxpy(a, x, y, x)  # in place: each call reads the previous call's w
    a_buf = torch.from_numpy(xh).cuda()
    b_buf = torch.empty_like(a_buf)
    bufs = [a_buf, b_buf]
    for k, a in enumerate(alphas):
        wx.wxpy(a, bufs[k % 2], y, bufs[(k + 1) % 2])
    torch.cuda.synchronize()
    want = chain_oracle(alphas, xh, yh)
    assert np.array_equal(x.cpu().numpy().view(np.uint64), want.view(np.uint64))
    want2 = pingpong_oracle(alphas, xh, yh)
    got2 = bufs[len(alphas) % 2].cpu().numpy()
    assert np.array_equal(got2.view(np.uint64), want2.view(np.uint64))


@pytest.mark.parametrize("streams", [2, 4])
def test_dependent_chain_through_the_stream_split(streams):
    """A split call (pieces on forked streams) between split and unsplit calls."""
    wx.wxpy_launch_pdl(1)
    n = (1 << 22) + 5
    seed = synth.BASE_SEED + 710 + streams
    _, xh, yh = synth.vectors(seed, n)
    alphas = [0.75, -0.5, 0.25, -1.0 / 3.0, 0.125, 0.5]
    split = wx.wxpy_variant_encode(vec_bytes=32, unroll=2, threads=256, blocks_per_sm=0,
                                   cache=2, carveout=-1, streams=streams, fp64_offload=1)
    plain = wx.wxpy_variant_encode(vec_bytes=16, unroll=4, threads=512, blocks_per_sm=2,
                                   cache=0, carveout=-1, streams=1, fp64_offload=0)
    x = torch.from_numpy(xh).cuda()
    y = torch.from_numpy(yh).cuda()
    for k, a in enumerate(alphas):
        wx.wxpy_run_variant(split if k % 2 == 0 else plain, a, x, y, x)
    torch.cuda.synchronize()
    want = chain_oracle(alphas, xh, yh)
    assert np.array_equal(x.cpu().numpy().view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("pdl", [1, 0])
def test_dependent_chain_in_a_graph(pdl):
    """The in-place chain captured once into a CUDA graph and replayed twice."""
    wx.wxpy_launch_pdl(pdl)
    n = (1 << 20) + 3
    seed = synth.BASE_SEED + 720
    _, xh, yh = synth.vectors(seed, n)
    alphas = [0.5, -0.75, 0.375, 0.625]
    x = torch.from_numpy(xh).cuda()
    y = torch.from_numpy(yh).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for a in alphas:  # warm-up outside the capture (lazy state)
            wx.wxpy(a, x, y, x, stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for a in alphas:
                wx.wxpy(a, x, y, x, stream=s)
    x.copy_(torch.from_numpy(xh))
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    want = chain_oracle(alphas + alphas, xh, yh)
    assert np.array_equal(x.cpu().numpy().view(np.uint64), want.view(np.uint64))


def test_pdl_switch_validation():
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy_launch_pdl(2)
    assert e.value.status == wx.WXPY_EINVAL
    prev = wx.wxpy_launch_pdl(0)
    assert wx.wxpy_launch_pdl(1) == 0
    assert wx.wxpy_launch_pdl(-1) == 1
    wx.wxpy_launch_pdl(prev)
