"""The allocation-free batched entry point, through the C ABI (GPU).

wxpy_batch_noalloc() exists for callers that cannot allocate device memory:
their memory belongs to another allocator (a framework's caching pool, a
server's fixed arena) that must not see a cudaMalloc it did not make, or their
loop cannot afford an allocation call.  Its results must be the oracle's and
the same bits as the existing batched entry point wxpy_batch() -- the
tolerance of every parity test here is 0 ULP -- on two calls in a row with
different tables, since both calls share one fixed scratch array inside the
library.  Descriptors it must skip (null or misaligned pointers, n <= 0)
leave their memory untouched; in-place problems (w == x, w == y) are exact;
a warm call allocates nothing.

The file is named so that pytest collects it last (a run that stops at the
first failure has then run every other test); it does not depend on running
last and passes alone in a fresh process too.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth
from gpu_util import CANARY_I64

pytestmark = pytest.mark.gpu

MAX_SEGMENTS = 65536


def _stream():
    return torch.cuda.current_stream().cuda_stream or None


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
    return (x, y), w_old, w_new, t_old, t_new, starts, alphas


def check_against_oracle(ns, starts, alphas, x, y, w, limit=None):
    """Every segment (or the first `limit` non-empty ones) of arena w equals
    the oracle on the same inputs, bit for bit."""
    xh, yh, wh = x.cpu().numpy(), y.cpu().numpy(), w.cpu().numpy()
    done = 0
    for n, st, a in zip(ns, starts, alphas):
        n = int(n)
        if n == 0:
            continue
        want = oracle.wxpy(float(a), xh[st:st + n], yh[st:st + n])
        got = wh[st:st + n]
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (n, st)
        done += 1
        if limit and done >= limit:
            break


def run_pair(ns, seed, oracle_limit=None):
    (x, y), w_old, w_new, t_old, t_new, starts, alphas = arena_batch(ns, seed)
    wx.wxpy_batch(t_old, wx.table_to_device(t_old))
    d_new = wx.table_to_device(t_new)
    rc = wx.lib().wxpy_batch_noalloc(d_new.data_ptr(), len(ns), _stream())
    assert rc == 0, wx.lib().wxpy_last_error_message()
    torch.cuda.synchronize()
    # whole arenas: segment results equal, gaps untouched in both
    assert torch.equal(w_old.view(torch.int64), w_new.view(torch.int64))
    assert not bool((w_new.view(torch.int64) == CANARY_I64).all())
    # and the oracle, directly
    check_against_oracle(ns, starts, alphas, x, y, w_new, oracle_limit)


def test_no_alloc_matches_oracle_and_batched_entry_point_on_two_calls_in_a_row():
    # call 1: a mixed batch with empty, tiny and tile-straddling segments
    ns1 = [0, 1, 3, 5, 8191, 8192, 8193, 100003] + list(
        synth.log_uniform_lengths(synth.BASE_SEED + 21, 3000, 1, 1 << 18))
    run_pair(ns1, synth.BASE_SEED + 21)
    # call 2, right after, on another table: many segments, so that the
    # per-segment tile limit (65536*4 slots / count) lengthens the tiles of the
    # big ones, and the scratch left by call 1 must not leak into this one
    ns2 = list(synth.log_uniform_lengths(synth.BASE_SEED + 22, 40000, 1, 1 << 10)) + \
        [1 << 18, (1 << 18) + 7, 0, 12345]
    run_pair(ns2, synth.BASE_SEED + 22, oracle_limit=2000)


def test_no_alloc_in_place_skipped_descriptors_and_no_allocation():
    """In-place segments (w == x, w == y) against the oracle; descriptors with a
    null or 4-byte-misaligned pointer or n <= 0 leave their canary-filled
    targets untouched; a warm call changes neither torch's allocator counters
    nor the device's free memory."""
    n_each = [4099, 70001, 1, 8192]
    seed = synth.BASE_SEED + 23
    bufs, descs, expect = [], [], []
    for k, n in enumerate(n_each):
        xh = synth.uniform_pm1(seed + k, synth.TAG_X, n)
        yh = synth.uniform_pm1(seed + k, synth.TAG_Y, n)
        a = float(synth.alpha_scalar(seed + k))
        x = torch.from_numpy(xh).cuda()
        y = torch.from_numpy(yh).cuda()
        bufs += [x, y]
        if k % 2 == 0:  # w == x
            descs.append((n, a, x.data_ptr(), y.data_ptr(), x.data_ptr()))
            expect.append((x, oracle.wxpy(a, xh, yh)))
        else:           # w == y
            descs.append((n, a, x.data_ptr(), y.data_ptr(), y.data_ptr()))
            expect.append((y, oracle.wxpy(a, xh, yh)))
    # descriptors to skip, each aimed at canary memory
    canary = torch.empty(4096, dtype=torch.float64, device="cuda")
    canary.view(torch.int64).fill_(CANARY_I64)
    src = torch.ones(4096, dtype=torch.float64, device="cuda")
    c0, s0 = canary.data_ptr(), src.data_ptr()
    skipped = [(1000, 2.0, 0, s0, c0),                  # null x
               (1000, 2.0, s0, 0, c0),                  # null y
               (1000, 2.0, s0, s0, 0),                  # null w
               (1000, 2.0, s0, s0, c0 + 4),             # w misaligned by 4 bytes
               (1000, 2.0, s0 + 4, s0, c0 + 8 * 1024),  # x misaligned by 4 bytes
               (0, 2.0, s0, s0, c0 + 8 * 2048),         # empty
               (-5, 2.0, s0, s0, c0 + 8 * 3072)]        # negative n
    allds = descs[:2] + skipped + descs[2:]
    table = wx.desc_table([d[0] for d in allds], [d[1] for d in allds], [d[2] for d in allds],
                          [d[3] for d in allds], [d[4] for d in allds])
    dt = wx.table_to_device(table)
    torch.cuda.synchronize()
    rc = wx.lib().wxpy_batch_noalloc(dt.data_ptr(), len(allds), _stream())
    assert rc == 0, wx.lib().wxpy_last_error_message()
    torch.cuda.synchronize()
    for t, want in expect:
        got = t.cpu().numpy()
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    assert bool((canary.view(torch.int64) == CANARY_I64).all())
    assert bool((src == 1.0).all())

    # a warm call on a table of copies allocates nothing
    xs = [torch.from_numpy(synth.uniform_pm1(seed + 9, synth.TAG_X, 50000)).cuda()
          for _ in range(2)]
    w2 = torch.empty_like(xs[0])
    t2 = wx.desc_table([50000], [0.5], [xs[0].data_ptr()], [xs[1].data_ptr()], [w2.data_ptr()])
    d2 = wx.table_to_device(t2)
    rc = wx.lib().wxpy_batch_noalloc(d2.data_ptr(), 1, _stream())  # warm
    assert rc == 0
    torch.cuda.synchronize()
    stats0 = torch.cuda.memory_stats()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert wx.lib().wxpy_batch_noalloc(d2.data_ptr(), 1, _stream()) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated",
                "reserved_bytes.all.current"):
        assert stats1.get(key) == stats0.get(key), key
    want = oracle.wxpy(0.5, xs[0].cpu().numpy(), xs[1].cpu().numpy())
    assert np.array_equal(w2.cpu().numpy().view(np.uint64), want.view(np.uint64))


def test_no_alloc_rejects_tables_over_its_maximum():
    rc = wx.lib().wxpy_batch_noalloc(1 << 20, MAX_SEGMENTS + 1, None)  # rejected before any use
    assert rc == wx.WXPY_EINVAL
    assert "65536" in wx.lib().wxpy_last_error_message().decode()
    assert wx.lib().wxpy_batch_noalloc(0, 0, None) == 0
