"""The allocation-free batched entry point, through the C ABI (GPU).

wxpy_batch_noalloc() exists for callers that cannot allocate device memory
(their memory belongs to another allocator, or their loop cannot afford an
allocation call).  It must give the same bits as the existing batched entry
point wxpy_batch() -- the tolerance of every parity test here is 0 ULP -- on
two calls in a row with different tables, since both calls share one fixed
scratch array inside the library.  This file is collected last on purpose.
"""
import pytest
import torch

import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth
from gpu_util import CANARY_I64

pytestmark = pytest.mark.gpu

MAX_SEGMENTS = 65536


def arena_batch(ns, seed):
    """x, y arenas filled from the generator; two canary-filled output arenas;
    descriptor tables for each (segment starts at 256-byte boundaries plus
    s % 4 elements, so every alignment class appears)."""
    starts, pos = [], 0
    for s, n in enumerate(ns):
        starts.append(pos + s % 4)
        pos += ((int(n) + s % 4 + 31) // 32) * 32 + 32
    x = torch.empty(pos, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    w_old = torch.empty_like(x)
    w_new = torch.empty_like(x)
    wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
    wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
    w_old.view(torch.int64).fill_(CANARY_I64)
    w_new.view(torch.int64).fill_(CANARY_I64)
    alphas = synth.uniform_pm2(seed, synth.TAG_ALPHA, len(ns))
    px, py = x.data_ptr(), y.data_ptr()
    xs = [px + 8 * s for s in starts]
    ys = [py + 8 * s for s in starts]
    t_old = wx.desc_table(ns, alphas, xs, ys, [w_old.data_ptr() + 8 * s for s in starts])
    t_new = wx.desc_table(ns, alphas, xs, ys, [w_new.data_ptr() + 8 * s for s in starts])
    return (x, y), w_old, w_new, t_old, t_new


def run_pair(ns, seed):
    keep, w_old, w_new, t_old, t_new = arena_batch(ns, seed)
    wx.wxpy_batch(t_old, wx.table_to_device(t_old))
    d_new = wx.table_to_device(t_new)
    stream = torch.cuda.current_stream().cuda_stream or None
    rc = wx.lib().wxpy_batch_noalloc(d_new.data_ptr(), len(ns), stream)
    assert rc == 0, wx.lib().wxpy_last_error_message()
    torch.cuda.synchronize()
    # whole arenas: segment results equal, gaps untouched in both
    assert torch.equal(w_old.view(torch.int64), w_new.view(torch.int64))
    assert not bool((w_new.view(torch.int64) == CANARY_I64).all())
    del keep


def test_no_alloc_matches_batched_entry_point_on_two_calls_in_a_row():
    # call 1: a mixed batch with empty, tiny and tile-straddling segments
    ns1 = [0, 1, 3, 5, 8191, 8192, 8193, 100003] + list(
        synth.log_uniform_lengths(synth.BASE_SEED + 21, 3000, 1, 1 << 18))
    run_pair(ns1, synth.BASE_SEED + 21)
    # call 2, right after, on another table: many segments, so that the
    # per-segment tile limit (65536*4 slots / count) lengthens the tiles of the
    # big ones, and the scratch left by call 1 must not leak into this one
    ns2 = list(synth.log_uniform_lengths(synth.BASE_SEED + 22, 40000, 1, 1 << 10)) + \
        [1 << 18, (1 << 18) + 7, 0, 12345]
    run_pair(ns2, synth.BASE_SEED + 22)


def test_no_alloc_rejects_tables_over_its_maximum():
    rc = wx.lib().wxpy_batch_noalloc(1 << 20, MAX_SEGMENTS + 1, None)  # rejected before any use
    assert rc == wx.WXPY_EINVAL
    assert "65536" in wx.lib().wxpy_last_error_message().decode()
    assert wx.lib().wxpy_batch_noalloc(0, 0, None) == 0
