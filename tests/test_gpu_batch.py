"""GPU parity of the batched, segmented launch through the C ABI.

Every segment of a batch must equal, bit for bit, the oracle on that segment
(w_s = RN(RN(alpha_s*x_s)+y_s), paper Sec. 3 / Fig. 1 vecwxpy) and the
single-call wxpy() on the same inputs; the gaps between segments must stay
untouched.  Covers empty and one-element segments, segments that straddle
tiles, mixed alignments, in-place segments, graph replay and re-targeting, the
one-shot call, the short-table guard, the batch search, and the full-size
4096-segment workload (sampled).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth
from gpu_util import CANARY_I64, bits_equal

pytestmark = pytest.mark.gpu


class Batch:
    """Segments laid out in three arenas (x, y, w) with 32-element gaps.

    Segment s starts at an offset of (s % 4) elements past a 256-byte boundary
    in all three arenas; every 7th segment has w shifted by one more element,
    so its pointers share only 8-byte alignment."""

    def __init__(self, ns, seed, host_inputs=True, in_place=()):
        self.ns = [int(n) for n in ns]
        self.seed = seed
        self.starts, self.wstarts = [], []
        pos = 0
        for s, n in enumerate(self.ns):
            o = s % 4
            self.starts.append(pos + o)
            self.wstarts.append(pos + o + (1 if s % 7 == 6 else 0))
            pos += ((n + o + 1 + 31) // 32) * 32 + 32
        self.total = pos
        self.x = torch.empty(self.total, dtype=torch.float64, device="cuda")
        self.y = torch.empty_like(self.x)
        self.w = torch.empty_like(self.x)
        wx.wxpy_fill_uniform(self.x, seed, synth.TAG_X)
        wx.wxpy_fill_uniform(self.y, seed, synth.TAG_Y)
        self.alphas = synth.uniform_pm2(seed, synth.TAG_ALPHA, len(self.ns))
        self.in_place = set(in_place)
        self.xh = synth.uniform_pm1(seed, synth.TAG_X, self.total) if host_inputs else None
        self.yh = synth.uniform_pm1(seed, synth.TAG_Y, self.total) if host_inputs else None
        self.reset_w()

    def reset_w(self):
        self.w.view(torch.int64).fill_(CANARY_I64)
        if self.in_place:
            wx.wxpy_fill_uniform(self.x, self.seed, synth.TAG_X)

    def table(self, alphas=None):
        a = self.alphas if alphas is None else alphas
        px, py, pw = self.x.data_ptr(), self.y.data_ptr(), self.w.data_ptr()
        xs = [px + 8 * st for st in self.starts]
        ys = [py + 8 * st for st in self.starts]
        ws = [(px + 8 * st) if s in self.in_place else (pw + 8 * wst)
              for s, (st, wst) in enumerate(zip(self.starts, self.wstarts))]
        return wx.desc_table(self.ns, a, xs, ys, ws)

    def out_of(self, s):
        n, st = self.ns[s], self.starts[s]
        if s in self.in_place:
            return self.x[st:st + n]
        return self.w[self.wstarts[s]:self.wstarts[s] + n]

    def check_oracle(self, alphas=None):
        a = self.alphas if alphas is None else alphas
        for s, n in enumerate(self.ns):
            st = self.starts[s]
            want = oracle.wxpy(float(a[s]), self.xh[st:st + n], self.yh[st:st + n])
            ok, msg = bits_equal(self.out_of(s), want)
            assert ok, f"segment {s} (n={n}): {msg}"
        self.check_gaps()

    def check_gaps(self):
        mask = torch.ones(self.total, dtype=torch.bool, device="cuda")
        for s, n in enumerate(self.ns):
            if s not in self.in_place:
                mask[self.wstarts[s]:self.wstarts[s] + n] = False
        assert bool((self.w.view(torch.int64)[mask] == CANARY_I64).all()), \
            "the batched launch wrote outside its segments"


def edge_lengths():
    return [0, 1, 2, 3, 4, 5, 31, 32, 33, 255, 1000, 8191, 8192, 8193, 16385, 65543, 0, 1]


@pytest.fixture(autouse=True)
def _shapes():
    wx.wxpy_batch_shape_reset()
    yield
    wx.wxpy_batch_shape_reset()


@pytest.mark.parametrize("offload", [0, 1, 3])
@pytest.mark.parametrize("mode", ["launch", "graph", "oneshot"])
def test_batch_matches_oracle(mode, offload):
    wx.wxpy_batch_launch_set(4, offload)
    ns = edge_lengths() + list(synth.log_uniform_lengths(synth.BASE_SEED + 11, 300, 1, 1 << 17))
    b = Batch(ns, synth.BASE_SEED + 11)
    t = b.table()
    dt = wx.table_to_device(t)
    if mode == "oneshot":
        wx.wxpy_batch(t, dt)
    else:
        plan = wx.wxpy_batch_plan_create(t)
        info = plan.info()
        assert info["segments"] == len(ns) and info["elements"] == sum(ns)
        (plan.launch if mode == "launch" else plan.graph_launch)(dt)
        torch.cuda.synchronize()
        assert plan.status() == 0
        plan.close()
    torch.cuda.synchronize()
    b.check_oracle()


def test_batch_equals_single_calls():
    ns = list(synth.log_uniform_lengths(synth.BASE_SEED + 12, 200, 1, 1 << 16))
    b = Batch(ns, synth.BASE_SEED + 12, host_inputs=False)
    t = b.table()
    plan = wx.wxpy_batch_plan_create(t)
    plan.launch(wx.table_to_device(t))
    torch.cuda.synchronize()
    batched = [b.out_of(s).clone() for s in range(len(ns))]
    b.reset_w()
    for s, n in enumerate(ns):
        st = b.starts[s]
        wx.wxpy(float(b.alphas[s]), b.x[st:st + n], b.y[st:st + n], b.out_of(s))
    torch.cuda.synchronize()
    for s in range(len(ns)):
        assert torch.equal(batched[s].view(torch.int64), b.out_of(s).view(torch.int64)), s


def test_graph_replay_and_retarget():
    ns = list(synth.log_uniform_lengths(synth.BASE_SEED + 13, 150, 1, 1 << 15)) + edge_lengths()
    b = Batch(ns, synth.BASE_SEED + 13)
    t1 = b.table()
    plan = wx.wxpy_batch_plan_create(t1)
    d1 = wx.table_to_device(t1)
    for _ in range(3):
        b.reset_w()
        plan.graph_launch(d1)
        torch.cuda.synchronize()
        b.check_oracle()
    alphas2 = synth.uniform_pm2(synth.BASE_SEED + 99, synth.TAG_ALPHA, len(ns))
    d2 = wx.table_to_device(b.table(alphas2))
    b.reset_w()
    plan.graph_launch(d2)
    torch.cuda.synchronize()
    b.check_oracle(alphas2)
    plan.close()


def test_in_place_segments():
    ns = [5, 1000, 8200, 77, 33000, 1, 4096]
    b = Batch(ns, synth.BASE_SEED + 14, in_place={1, 2, 5})
    t = b.table()
    plan = wx.wxpy_batch_plan_create(t)
    plan.launch(wx.table_to_device(t))
    torch.cuda.synchronize()
    b.check_oracle()
    plan.close()


def test_short_device_table_is_guarded():
    """A device table with smaller n than the plan's: tiles past n are skipped
    and flagged, nothing is written beyond the device table's n."""
    ns = [40000, 30000, 20000]
    b = Batch(ns, synth.BASE_SEED + 15, host_inputs=False)
    t = b.table()
    plan = wx.wxpy_batch_plan_create(t)
    short = t.copy()
    short["n"] = [100, 30000, 9000]
    plan.launch(wx.table_to_device(short))
    torch.cuda.synchronize()
    assert plan.status(clear=True) & 1
    assert plan.status() == 0
    for s, n_short in enumerate(short["n"]):
        tail = b.out_of(s)[int(n_short):]
        assert bool((tail.view(torch.int64) == CANARY_I64).all()), f"segment {s} written past n"
    plan.close()


def test_batch_search_then_parity():
    r = wx.wxpy_batch_tune(0, 14, wx.TUNE_QUICK)
    assert r["rejected"] == 0 and r["candidates"] > 0
    for row in r["buckets"]:
        assert wx.wxpy_batch_shape_get(row["bucket"]) == (row["tile_elems"], row["unroll"])
    ns = edge_lengths() + list(synth.log_uniform_lengths(synth.BASE_SEED + 16, 200, 1, 1 << 14))
    b = Batch(ns, synth.BASE_SEED + 16)
    t = b.table()
    wx.wxpy_batch(t, wx.table_to_device(t))
    torch.cuda.synchronize()
    b.check_oracle()


def test_full_size_4096_segments_sampled():
    """4096 segments, n log-uniform in [1, 2^20] (about 3.1e8 elements), graph
    replay in the launch configuration the benchmark times; every segment is
    checked at its ends and at random interior points."""
    seed = synth.BASE_SEED + 3
    ns = synth.log_uniform_lengths(seed, 4096, 1, 1 << 20)
    b = Batch(ns, seed, host_inputs=False)
    t = b.table()
    plan = wx.wxpy_batch_plan_create(t)
    plan.graph_launch(wx.table_to_device(t))
    torch.cuda.synchronize()
    assert plan.status() == 0
    rng = np.random.default_rng(0)
    idx_all, want_all, got_pos = [], [], []
    for s, n in enumerate(b.ns):
        if n == 0:
            continue
        loc = np.unique(np.concatenate([np.arange(min(n, 8)), np.arange(max(0, n - 8), n),
                                        rng.integers(0, n, 16)]))
        st = b.starts[s]
        xs = synth.uniform_pm1_at(seed, synth.TAG_X, st + loc)
        ys = synth.uniform_pm1_at(seed, synth.TAG_Y, st + loc)
        want_all.append(oracle.wxpy(float(b.alphas[s]), xs, ys))
        got_pos.append(b.wstarts[s] + loc)
    pos = torch.from_numpy(np.concatenate(got_pos)).cuda()
    got = b.w[pos].cpu().numpy()
    want = np.concatenate(want_all)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    plan.close()
