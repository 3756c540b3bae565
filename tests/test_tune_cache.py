"""The tuning table and its JSON file on the host (no GPU): set/get/clear and
loading without a device check, including malformed files that must store nothing."""
import json

import pytest

import paper_1309_1894_gb300 as wx


@pytest.fixture(autouse=True)
def _clean():
    wx.lib()
    wx.wxpy_tune_clear()
    yield
    wx.wxpy_tune_clear()


def write(path, entries, fmt="wxpy-tune-1", device="X|cc10.3|sm152|cudart13000"):
    path.write_text(json.dumps({"format": fmt, "device": device, "entries": entries}, indent=1))
    return str(path)


def test_set_get_clear():
    wx.wxpy_tune_set(5, 1234)
    assert wx.wxpy_tune_get(5) == 1234
    wx.wxpy_tune_set(5, -1)
    assert wx.wxpy_tune_get(5) == -1
    wx.wxpy_tune_set(7, 3)
    wx.wxpy_tune_clear()
    assert wx.wxpy_tune_get(7) == -1
    with pytest.raises(wx.WxpyError):
        wx.wxpy_tune_set(64 * 12, 1)
    with pytest.raises(wx.WxpyError):
        wx.wxpy_tune_set(1, wx.wxpy_variant_count())


def test_load_without_device_check(tmp_path):
    p = write(tmp_path / "a.json", [{"key": 12 * 20, "variant": 9856},
                                    {"key": 12 * 28 + 1, "variant": 77}])
    wx.wxpy_tune_cache_load(p, check_device=False)
    assert wx.wxpy_tune_get(12 * 20) == 9856
    assert wx.wxpy_tune_get(12 * 28 + 1) == 77


@pytest.mark.parametrize("entries,fmt", [
    ([{"key": 3, "variant": 99999999}], "wxpy-tune-1"),
    ([{"key": -1, "variant": 5}], "wxpy-tune-1"),
    ([{"key": 3}], "wxpy-tune-1"),
    ([{"key": 3, "variant": 5}], "something-else"),
])
def test_malformed_file_stores_nothing(tmp_path, entries, fmt):
    p = write(tmp_path / "bad.json", [{"key": 1, "variant": 2}] + entries, fmt=fmt)
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy_tune_cache_load(p, check_device=False)
    assert e.value.status == wx.WXPY_EINVAL
    assert wx.wxpy_tune_get(1) == -1


def test_missing_file(tmp_path):
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy_tune_cache_load(str(tmp_path / "nope.json"), check_device=False)
    assert e.value.status == wx.WXPY_ENOTFOUND
