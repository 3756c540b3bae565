"""GPU tests of wxpy_host: the host-buffer path (chunked copies in, tuned kernel,
copies out, overlapped on internal streams) gives the oracle's bits, for pinned
and pageable buffers, ragged chunk boundaries and host aliasing."""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _config():
    yield
    wx.wxpy_host_config(1 << 22, 3, False)


@pytest.mark.parametrize("pinned", [True, False])
def test_direct_strategy(pinned):
    """Zero-copy on mapped pinned memory; pageable memory falls back to staging."""
    wx.wxpy_host_config(1 << 22, 3, True)
    for n in (1, 1001, (1 << 20) + 5):
        alpha, xh, yh, x, y, w = host_arrays(n, 900 + n, pinned)
        wx.wxpy_host(alpha, x, y, w)
        torch.cuda.synchronize()
        want = oracle.wxpy(alpha, xh, yh)
        assert np.array_equal(w.numpy().view(np.uint64), want.view(np.uint64)), n
    alpha, xh, yh, x, y, w = host_arrays(70001, 901, pinned)
    wx.wxpy_host(alpha, x, y, x)  # in place
    torch.cuda.synchronize()
    assert np.array_equal(x.numpy().view(np.uint64), oracle.wxpy(alpha, xh, yh).view(np.uint64))


def host_arrays(n, seed, pinned):
    alpha, xh, yh = synth.vectors(seed, n)
    if pinned:
        x = torch.from_numpy(xh).pin_memory()
        y = torch.from_numpy(yh).pin_memory()
        w = torch.full((n,), float("nan"), dtype=torch.float64).pin_memory()
    else:
        x, y, w = torch.from_numpy(xh.copy()), torch.from_numpy(yh.copy()), \
            torch.full((n,), float("nan"), dtype=torch.float64)
    return alpha, xh, yh, x, y, w


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("slots", [1, 2, 3])
def test_chunked_pipeline_matches_oracle(pinned, slots):
    chunk = 4096
    wx.wxpy_host_config(chunk, slots, False)
    for n in (1, 5, chunk - 1, chunk, chunk + 1, 3 * chunk + 7, 10 * chunk + 3):
        alpha, xh, yh, x, y, w = host_arrays(n, 500 + n, pinned)
        wx.wxpy_host(alpha, x, y, w)
        torch.cuda.synchronize()
        want = oracle.wxpy(alpha, xh, yh)
        assert np.array_equal(w.numpy().view(np.uint64), want.view(np.uint64)), (n, slots)


def test_host_aliasing_and_default_config():
    n = (1 << 23) + 11  # several default-size chunks
    alpha, xh, yh, x, y, w = host_arrays(n, 77, True)
    wx.wxpy_host(alpha, x, y, x)  # in place, w == x
    torch.cuda.synchronize()
    assert np.array_equal(x.numpy().view(np.uint64), oracle.wxpy(alpha, xh, yh).view(np.uint64))
    alpha, xh, yh, x, y, w = host_arrays(n, 78, True)
    wx.wxpy_host(alpha, x, x, w)  # x == y
    torch.cuda.synchronize()
    assert np.array_equal(w.numpy().view(np.uint64), oracle.wxpy(alpha, xh, xh).view(np.uint64))


def test_host_on_a_side_stream():
    n = 300001
    alpha, xh, yh, x, y, w = host_arrays(n, 79, True)
    s = torch.cuda.Stream()
    wx.wxpy_host(alpha, x, y, w, stream=s)
    s.synchronize()
    assert np.array_equal(w.numpy().view(np.uint64), oracle.wxpy(alpha, xh, yh).view(np.uint64))
