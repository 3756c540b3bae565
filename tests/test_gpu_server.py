"""GPU tests of the continuous-batching server through the C ABI.

Each request's result must be the same bits alone and in the mix (0 ULP):
equal to a standalone wxpy() on the same seeded inputs, and to the oracle --
for seeded requests and for requests on the caller's own data (device or
host memory), in the batched mode (inputs step, then one segmented launch
that reads x and y from the resident buffers), the serial baseline and the
fused option.  The server's admission (budget, slots, queue limit), failure
reporting and built-in Poisson client are checked too.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import synth
from paper_1309_1894_gb300.server import Server, SERVE_BATCHED, SERVE_SERIAL, SERVE_FUSED, \
    REQ_DONE, REQ_QUEUED, REQ_FAILED

pytestmark = pytest.mark.gpu


def _from_ptr(ptr, n):
    """A float64 CUDA tensor aliasing n elements at a device pointer."""
    class _Holder:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Holder(), device="cuda")


def alone(n, alpha, seed):
    """The request computed by itself: generator inputs, one wxpy() call."""
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    wx.wxpy_fill_uniform(x, seed, synth.TAG_X)
    wx.wxpy_fill_uniform(y, seed, synth.TAG_Y)
    return wx.wxpy(alpha, x, y)


def request_mix(seed, count, hi):
    ns = [1, 3, 8191, 8192, 8193, (1 << 20) + 3] + list(
        synth.log_uniform_lengths(seed, count, 1, hi))
    alphas = synth.uniform_pm2(seed, synth.TAG_ALPHA, len(ns))
    seeds = [seed * 1000 + i for i in range(len(ns))]
    return [(int(n), float(a), s) for n, a, s in zip(ns, alphas, seeds)]


def run_requests(mode, reqs, **kw):
    out = {}
    with Server(budget_bytes=2 << 30, mode=mode, **kw) as sv:
        tickets = [sv.submit(n, a, s) for (n, a, s) in reqs]
        for t in tickets:
            lat = sv.wait(t, 60.0)
            assert lat > 0
        torch.cuda.synchronize()
        for t, (n, a, s) in zip(tickets, reqs):
            m, px, py, pw = sv.result(t)
            assert m == n
            out[s] = _from_ptr(pw, n).clone()
            sv.release(t)
        st = sv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0 and st["resident_now"] == 0
        assert st["arena_used"] == 0
    return out, st


def test_batched_results_equal_alone_and_oracle():
    reqs = request_mix(31, 250, 1 << 18)
    out, st = run_requests(SERVE_BATCHED, reqs, n_streams=2, max_batch=64)
    assert st["batches"] < len(reqs)  # requests were coalesced
    for (n, a, s) in reqs:
        w_alone = alone(n, a, s)
        assert torch.equal(out[s].view(torch.int64), w_alone.view(torch.int64)), (n, s)
    for (n, a, s) in reqs[:40]:  # oracle on the host for a subset
        xh = synth.uniform_pm1(s, synth.TAG_X, n)
        yh = synth.uniform_pm1(s, synth.TAG_Y, n)
        want = oracle.wxpy(a, xh, yh)
        got = out[s].cpu().numpy()
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (n, s)


def test_serial_batched_and_fused_modes_agree():
    reqs = request_mix(32, 80, 1 << 16)
    a, st_a = run_requests(SERVE_BATCHED, reqs, n_streams=3, max_batch=16)
    b, st_b = run_requests(SERVE_SERIAL, reqs, n_streams=1, max_batch=1)
    c, st_c = run_requests(SERVE_SERIAL, reqs, n_streams=2, max_batch=32)
    f, st_f = run_requests(SERVE_FUSED, reqs, n_streams=2, max_batch=16)
    assert st_b["batches"] == len(reqs) and st_b["mean_batch"] == 1.0
    # serial: fill x, fill y, wxpy() per request
    assert st_b["launches"] == 3 * len(reqs) == st_c["launches"]
    # batched: one fill launch and one segmented launch per batch
    assert st_a["launches"] == 2 * st_a["batches"] and st_a["batches"] < len(reqs)
    assert st_f["launches"] == st_f["batches"]  # fused: one launch per batch
    for (_, _, s) in reqs:
        assert torch.equal(a[s].view(torch.int64), b[s].view(torch.int64))
        assert torch.equal(a[s].view(torch.int64), c[s].view(torch.int64))
        assert torch.equal(a[s].view(torch.int64), f[s].view(torch.int64))


@pytest.mark.parametrize("mode", [SERVE_BATCHED, SERVE_SERIAL])
def test_caller_data_requests_in_a_mix(mode):
    """Requests on the caller's data -- device tensors, pinned and pageable host
    tensors -- mixed with seeded requests in the same batches: every result is
    the oracle's on its own inputs, the caller's buffers are untouched, and the
    resident x and y hold exactly the caller's values."""
    rng = np.random.default_rng(41)
    lens = [1, 5, 4099, 8192, 70001, (1 << 18) + 3, 300000]
    data = []
    for i, n in enumerate(lens):
        xh = synth.uniform_pm1(900 + i, synth.TAG_X, n)
        yh = synth.uniform_pm1(900 + i, synth.TAG_Y, n)
        # special values in the caller's data: signed zeros, a subnormal, an infinity
        if n > 8:
            xh[:4] = [0.0, -0.0, 5e-324, np.inf]
            yh[:4] = [-0.0, 0.0, -5e-324, 1.0]
        alpha = float(rng.uniform(-2, 2))
        if i % 3 == 0:
            x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        elif i % 3 == 1:
            x = torch.from_numpy(xh).pin_memory()
            y = torch.from_numpy(yh).pin_memory()
        else:  # pageable host memory: copied synchronously, still exact
            x, y = torch.from_numpy(xh.copy()), torch.from_numpy(yh.copy())
        data.append((n, alpha, xh, yh, x, y))
    seeded = request_mix(43, 30, 1 << 17)
    with Server(budget_bytes=1 << 30, mode=mode, n_streams=2, max_batch=16) as sv:
        tickets = []
        for k in range(max(len(data), len(seeded))):
            if k < len(data):
                n, a, _, _, x, y = data[k]
                tickets.append(("d", k, sv.submit_data(a, x, y)))
            if k < len(seeded):
                n, a, sd = seeded[k]
                tickets.append(("s", k, sv.submit(n, a, sd)))
        for _, _, t in tickets:
            sv.wait(t, 60.0)
        torch.cuda.synchronize()
        for kind, k, t in tickets:
            m, px, py, pw = sv.result(t)
            if kind == "d":
                n, a, xh, yh, x, y = data[k]
                assert m == n
                got = _from_ptr(pw, n).cpu().numpy()
                want = oracle.wxpy(a, xh, yh)
                assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (n, k)
                assert np.array_equal(_from_ptr(px, n).cpu().numpy().view(np.uint64),
                                      xh.view(np.uint64))
                assert np.array_equal(_from_ptr(py, n).cpu().numpy().view(np.uint64),
                                      yh.view(np.uint64))
                assert np.array_equal(x.cpu().numpy().view(np.uint64), xh.view(np.uint64))
            else:
                n, a, sd = seeded[k]
                assert m == n
                assert torch.equal(_from_ptr(pw, n).view(torch.int64),
                                   alone(n, a, sd).view(torch.int64)), (n, sd)
            sv.release(t)
        st = sv.stats()
        assert st["completed"] == len(tickets) and st["failed"] == 0
        assert st["arena_used"] == 0
        if mode == SERVE_BATCHED:
            assert st["batches"] < len(tickets)


def test_caller_data_refused_where_invalid():
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    with Server(budget_bytes=64 << 20, mode=SERVE_FUSED) as sv:
        with pytest.raises(wx.WxpyError) as e:
            sv.submit_data(1.0, x, x)
        assert e.value.status == wx.WXPY_EINVAL
    with Server(budget_bytes=64 << 20) as sv:
        import ctypes
        t = ctypes.c_uint64()
        lib = wx.lib()
        p = x.data_ptr()
        assert lib.wxpy_server_submit_data(sv.handle, 16, 1.0, p + 4, p, 0, ctypes.byref(t)) \
            == wx.WXPY_EINVAL
        assert lib.wxpy_server_submit_data(sv.handle, 16, 1.0, p, p, 2, ctypes.byref(t)) \
            == wx.WXPY_EINVAL
        assert lib.wxpy_server_submit_data(sv.handle, 16, 1.0, None, p, 0, ctypes.byref(t)) \
            == wx.WXPY_EINVAL
        assert lib.wxpy_server_submit_data(sv.handle, 3 << 20, 1.0, p, p, 0, ctypes.byref(t)) \
            == wx.WXPY_EBUDGET


def test_budget_slots_and_queue_limit():
    n = 1 << 16  # 3 * 512 KiB per request
    per = 3 * 8 * n
    with Server(budget_bytes=2 * per, max_slots=2, n_streams=2, max_batch=8, max_queue=3) as sv:
        with pytest.raises(wx.WxpyError) as e:
            sv.submit(n * 3, 1.0, 1)  # can never fit the budget
        assert e.value.status == wx.WXPY_EBUDGET
        t = [sv.submit(n, 0.5, 100 + i) for i in range(2)]
        for ti in t:
            sv.wait(ti, 30.0)
        # both slots held (results not released): new requests wait in the queue
        q = [sv.submit(n, 0.5, 200 + i) for i in range(3)]
        with pytest.raises(wx.WxpyError) as e:
            sv.submit(n, 0.5, 299)  # queue of 3 is full
        assert e.value.status == wx.WXPY_EBUSY
        import time
        time.sleep(0.05)
        assert sv.poll(q[0])[0] == REQ_QUEUED
        sv.release(t[0])
        sv.wait(q[0], 30.0)
        assert sv.poll(q[0])[0] == REQ_DONE
        assert sv.poll(q[1])[0] == REQ_QUEUED
        for ti in (t[1], q[0]):
            sv.release(ti)
        for ti in q[1:]:
            sv.wait(ti, 30.0)
            sv.release(ti)
        st = sv.stats()
        assert st["rejected"] == 1 and st["completed"] == 5 and st["resident_now"] == 0
        with pytest.raises(wx.WxpyError) as e:
            sv.poll(t[0])
        assert e.value.status == wx.WXPY_ENOTFOUND


def test_injected_launch_failure_fails_only_that_batch():
    with Server(budget_bytes=256 << 20, n_streams=1, max_batch=4) as sv:
        wx.wxpy_debug_inject_launch_error(719, 1)
        t1 = sv.submit(5000, 1.5, 7)
        with pytest.raises(wx.WxpyError) as e:
            sv.wait(t1, 30.0)
        assert e.value.status == wx.WXPY_ECUDA
        assert sv.poll(t1)[0] == REQ_FAILED
        sv.release(t1)
        wx.wxpy_debug_inject_launch_error(0, 0)
        t2 = sv.submit(5000, 1.5, 7)
        sv.wait(t2, 30.0)
        _, _, _, pw = sv.result(t2)
        assert torch.equal(_from_ptr(pw, 5000).view(torch.int64),
                           alone(5000, 1.5, 7).view(torch.int64))
        sv.release(t2)
        assert sv.stats()["failed"] == 1


def test_poisson_loadgen_short():
    with Server(budget_bytes=2 << 30, n_streams=2, max_batch=256) as sv:
        r = sv.loadgen(rate=3000.0, duration_s=0.5, n_min=256, n_max=1 << 16, seed=5,
                       drain_timeout_s=30.0)
        assert r["drained"] == 1
        assert r["completed"] == r["submitted"] > 500 and r["failed"] == 0
        assert 0 < r["p50_s"] <= r["p99_s"] <= r["max_s"]
        assert r["elem_per_s"] > 0
        st = sv.stats()
        assert st["resident_now"] == 0 and st["arena_used"] == 0
        # the batch timing record: some host time to queue each batch, and no
        # batch took longer from queueing to completion than the slowest request
        assert 0 < st["max_launch_host_s"] <= st["max_batch_s"] <= r["max_s"]


def test_batches_overlap_under_load():
    """Continuous batching, not a queue drained batch by batch: with two streams
    and a steady stream of large requests, two batches are on the device at once
    while new requests keep being admitted."""
    with Server(budget_bytes=4 << 30, n_streams=2, max_batch=64) as sv:
        r = sv.loadgen(rate=20000.0, duration_s=0.5, n_min=1 << 18, n_max=1 << 22, seed=11,
                       drain_timeout_s=30.0)
        st = sv.stats()
        assert r["drained"] == 1 and r["failed"] == 0
        assert st["max_inflight"] == 2
        assert st["batches"] > 2 and st["completed"] == r["completed"]


@pytest.mark.parametrize("admission_us", [0, 10_000_000])
def test_backfill_admission(admission_us):
    """A resident request A (not released) leaves room for small requests but
    not for the large B queued behind it.  Strict order: the small C and D
    wait behind B.  Backfill: C and D are admitted past B and complete while
    B waits; B runs once A is released.  Every result is the oracle's."""
    big = 1 << 22
    per_big = 3 * 8 * big
    with Server(budget_bytes=per_big + per_big // 2, max_slots=16, n_streams=2, max_batch=8,
                max_queue=16, admission_us=admission_us) as sv:
        a = sv.submit(big, 0.5, 11)
        sv.wait(a)
        b = sv.submit(big, -1.5, 12)
        c = sv.submit(4099, 0.25, 13)
        d = sv.submit(70001, 2.0, 14)
        import time
        time.sleep(0.2)
        states = {t: sv.poll(t)[0] for t in (b, c, d)}
        assert states[b] == REQ_QUEUED
        if admission_us:
            assert states[c] == REQ_DONE and states[d] == REQ_DONE
            assert sv.stats()["backfilled"] >= 2
        else:
            assert states[c] == REQ_QUEUED and states[d] == REQ_QUEUED
            assert sv.stats()["backfilled"] == 0
        sv.release(a)
        for t in (b, c, d):
            sv.wait(t)
        for t, (n, alpha, seed) in ((b, (big, -1.5, 12)), (c, (4099, 0.25, 13)),
                                   (d, (70001, 2.0, 14))):
            m, px, py, pw = sv.result(t)
            assert m == n
            w = _from_ptr(pw, n).cpu().numpy()
            want = oracle.wxpy(alpha, synth.uniform_pm1(seed, synth.TAG_X, n),
                               synth.uniform_pm1(seed, synth.TAG_Y, n))
            assert np.array_equal(w.view(np.uint64), want.view(np.uint64))
            sv.release(t)
        st = sv.stats()
        assert st["head_wait_frag_s"] + st["head_wait_full_s"] > 0.1


def test_tile_list_grows_for_a_batch_of_short_tiles():
    """A batch shape with 32-element tiles makes one batch need far more tile
    records than a stream's list was sized for (its share of the budget at
    8192-element tiles): the scheduler reallocates the idle slot's staging
    region before queueing the batch, and every result is still exact."""
    try:
        for b in range(13, 23):
            wx.wxpy_batch_shape_set(b, 32, 1)
        reqs = [(int(n), float(a), 7000 + i) for i, (n, a) in enumerate(zip(
            [(1 << 22) + 5, (1 << 21) + 3, 1 << 20, 123457, 8193, 1, 77],
            synth.uniform_pm2(71, synth.TAG_ALPHA, 7)))]
        # 2 GiB budget, 2 streams: a stream's list starts at 1 GiB / (24 x 8192) + 16,
        # about 5.5k records; the first request alone is 131k tiles of 32 elements
        out, st = run_requests(SERVE_BATCHED, reqs, n_streams=2, max_batch=16)
        for (n, a, s) in reqs:
            assert torch.equal(out[s].view(torch.int64), alone(n, a, s).view(torch.int64)), n
    finally:
        wx.wxpy_batch_shape_reset()
