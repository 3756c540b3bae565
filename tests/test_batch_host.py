"""Host-side logic of the batched launch (no GPU): descriptor validation runs
before any CUDA call, and the batch shape table."""
import pytest

import paper_1309_1894_gb300 as wx

B = 1 << 40  # pointer values only; never dereferenced


def table(rows):
    return wx.desc_table([r[0] for r in rows], [1.0] * len(rows), [r[1] for r in rows],
                         [r[2] for r in rows], [r[3] for r in rows])


@pytest.mark.parametrize("rows,status", [
    ([(-1, B, B + 4096, B + 8192)], wx.WXPY_EINVAL),
    ([(8, 0, B + 4096, B + 8192)], wx.WXPY_EINVAL),
    ([(8, B + 4, B + 4096, B + 8192)], wx.WXPY_EINVAL),
    ([(8, B, B + 4096, B + 8)], wx.WXPY_EOVERLAP),                        # within a segment
    ([(8, B, B + 4096, B + 8192), (8, B + 65536, B + 65600, B + 8192)], wx.WXPY_EOVERLAP),  # same w
    ([(8, B, B + 4096, B + 8192), (8, B + 65536, B + 65600, B + 8192 + 56)], wx.WXPY_EOVERLAP),
    ([(8, B, B + 4096, B + 8192), (8, B + 8192, B + 65600, B + 70000)], wx.WXPY_EOVERLAP),  # reads another's w
    ([(8, B, B + 4096, B + 8192), (8, B + 65536, B + 8192 + 32, B + 70000)], wx.WXPY_EOVERLAP),
])
def test_validation_before_cuda(rows, status):
    t = table(rows)
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy_batch_plan_create(t)
    assert e.value.status == status
    dev_dummy = B  # never reached: validation fails first
    rc = wx.lib().wxpy_batch(t.ctypes.data, dev_dummy, len(t), None)
    assert rc == status


def test_independent_segments_pass_validation_and_reads_may_share():
    """x and y may be shared between segments (both only read)."""
    t = table([(8, B, B + 4096, B + 8192), (8, B, B + 4096, B + 16384), (0, 0, 0, 0)])
    # validation passes; the plan then needs a device, so only check that the
    # error (if any) is not a validation error
    rc = wx.lib().wxpy_batch(t.ctypes.data, 0, 0, None)  # count 0: no-op
    assert rc == 0


def test_shape_table():
    wx.wxpy_batch_shape_reset()
    t0, u0 = wx.wxpy_batch_shape_get(20)
    assert t0 % 32 == 0 and u0 in (1, 2, 4, 8)
    wx.wxpy_batch_shape_set(20, 4096, 4)
    assert wx.wxpy_batch_shape_get(20) == (4096, 4)
    wx.wxpy_batch_shape_set(3, 0, 1)
    assert wx.wxpy_batch_shape_get(3) == (0, 1)
    for bad in ((20, 100, 4), (20, 4096, 3), (20, 4096, 8), (64, 0, 1), (-1, 0, 1)):
        with pytest.raises(wx.WxpyError):
            wx.wxpy_batch_shape_set(*bad)
    wx.wxpy_batch_shape_reset()
    assert wx.wxpy_batch_shape_get(20) == (t0, u0)


def test_cache_file_with_batch_shapes(tmp_path):
    import json
    wx.wxpy_batch_shape_reset()
    doc = {"format": "wxpy-tune-1", "device": "X",
           "batch_launch": {"threads": 256, "blocks_per_sm": 8},
           "batch": [{"bucket": 5, "tile": 0, "unroll_log2": 1},
                     {"bucket": 18, "tile": 16384, "unroll_log2": 2}],
           "entries": [{"key": 100, "variant": 42}]}
    p = tmp_path / "c.json"
    p.write_text(json.dumps(doc))
    wx.wxpy_tune_clear()
    wx.wxpy_tune_cache_load(str(p), check_device=False)
    assert wx.wxpy_batch_shape_get(18) == (16384, 4)
    assert wx.wxpy_batch_shape_get(5) == (0, 2)
    assert wx.wxpy_tune_get(100) == 42
    doc["batch"][0]["tile"] = 33  # not a multiple of 32: whole file refused
    p.write_text(json.dumps(doc))
    wx.wxpy_batch_shape_reset()
    wx.wxpy_tune_clear()
    with pytest.raises(wx.WxpyError):
        wx.wxpy_tune_cache_load(str(p), check_device=False)
    assert wx.wxpy_tune_get(100) == -1
    wx.wxpy_batch_shape_reset()
    wx.wxpy_tune_clear()


def test_batch_launch_knobs():
    wx.wxpy_batch_shape_reset()
    bps, of = wx.wxpy_batch_launch_get()
    assert 1 <= bps <= 32 and of in (0, 1, 3)
    wx.wxpy_batch_launch_set(8, 0)
    assert wx.wxpy_batch_launch_get() == (8, 0)
    wx.wxpy_batch_launch_set(2, 3)  # every product in the integer pipelines
    assert wx.wxpy_batch_launch_get() == (2, 3)
    for bad in ((0, 0), (33, 0), (4, 2), (4, -1), (4, 4)):
        with pytest.raises(wx.WxpyError):
            wx.wxpy_batch_launch_set(*bad)
    wx.wxpy_batch_shape_reset()
    assert wx.wxpy_batch_launch_get() == (bps, of)
