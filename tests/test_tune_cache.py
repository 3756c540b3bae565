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


def test_load_launch_bound_flag(tmp_path):
    """Cells the search found launch-bound carry "launch_bound": 1 (optional;
    0 when absent); any other value makes the file malformed."""
    p = write(tmp_path / "lb.json", [{"key": 12 * 10, "variant": 240, "launch_bound": 1},
                                     {"key": 12 * 24, "variant": 19920, "launch_bound": 0},
                                     {"key": 12 * 25, "variant": 19696}])
    wx.wxpy_tune_cache_load(p, check_device=False)
    assert wx.wxpy_tune_get(12 * 10) == 240 and wx.wxpy_tune_get(12 * 25) == 19696
    bad = write(tmp_path / "lb2.json", [{"key": 12 * 11, "variant": 240, "launch_bound": 2}])
    with pytest.raises(wx.WxpyError):
        wx.wxpy_tune_cache_load(bad, check_device=False)
    assert wx.wxpy_tune_get(12 * 11) == -1


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


def test_vecops_split_set_get_clear():
    assert wx.wxpy_vecops_tuned_get(wx.VEC_AXPBYPCZ) == (-1, -1)
    wx.wxpy_vecops_tuned_set(wx.VEC_AXPBYPCZ, 0, 12)
    assert wx.wxpy_vecops_tuned_get(wx.VEC_AXPBYPCZ) == (0, 12)
    wx.wxpy_vecops_tuned_set(wx.VEC_AXPBYPCZ, -1, -1)
    assert wx.wxpy_vecops_tuned_get(wx.VEC_AXPBYPCZ) == (-1, -1)
    wx.wxpy_vecops_tuned_set(3, 2, 16)
    wx.wxpy_tune_clear()  # drops the searched splits too
    assert wx.wxpy_vecops_tuned_get(3) == (-1, -1)
    for bad in ((wx.VEC_CLASSES, 0, 4), (-1, 0, 4), (0, 3, 4), (0, 0, 17), (0, -1, 4),
                (wx.VEC_PMULT, 1, 4)):  # pointwise_mult has no sums to offload
        with pytest.raises(wx.WxpyError) as e:
            wx.wxpy_vecops_tuned_set(*bad)
        assert e.value.status == wx.WXPY_EINVAL


def test_load_vecops_section(tmp_path):
    path = tmp_path / "v.json"
    path.write_text(json.dumps({"format": "wxpy-tune-1", "device": "X",
                                "vecops": [{"class": 3, "add_offload": 1, "mul_sixteenths": 10},
                                           {"class": 8, "add_offload": 0, "mul_sixteenths": 2}],
                                "entries": [{"key": 4, "variant": 11}]}))
    wx.wxpy_tune_cache_load(str(path), check_device=False)
    assert wx.wxpy_vecops_tuned_get(3) == (1, 10)
    assert wx.wxpy_vecops_tuned_get(8) == (0, 2)
    assert wx.wxpy_vecops_tuned_get(0) == (-1, -1)
    assert wx.wxpy_tune_get(4) == 11


@pytest.mark.parametrize("entry", [{"class": wx.VEC_CLASSES, "add_offload": 0, "mul_sixteenths": 2},
                                   {"class": 1, "add_offload": 3, "mul_sixteenths": 2},
                                   {"class": 1, "add_offload": 0, "mul_sixteenths": 17},
                                   {"class": 1, "add_offload": 0}])
def test_malformed_vecops_entry_stores_nothing(tmp_path, entry):
    path = tmp_path / "bad.json"
    path.write_text(json.dumps({"format": "wxpy-tune-1", "device": "X",
                                "vecops": [{"class": 2, "add_offload": 0, "mul_sixteenths": 6},
                                           entry],
                                "entries": [{"key": 1, "variant": 2}]}))
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy_tune_cache_load(str(path), check_device=False)
    assert e.value.status == wx.WXPY_EINVAL
    assert wx.wxpy_vecops_tuned_get(2) == (-1, -1)
    assert wx.wxpy_tune_get(1) == -1


def test_reduce_config_set_get_clear():
    assert wx.wxpy_reduce_tuned_get(0) == (-1, -1, -1)
    wx.wxpy_reduce_tuned_set(0, 2, 12, 1)
    assert wx.wxpy_reduce_tuned_get(0) == (2, 12, 1)
    wx.wxpy_reduce_tuned_set(0, -1, -1, -1)
    assert wx.wxpy_reduce_tuned_get(0) == (-1, -1, -1)
    wx.wxpy_reduce_tuned_set(1, 0, 16, 0)
    wx.wxpy_tune_clear()  # drops the searched configurations too
    assert wx.wxpy_reduce_tuned_get(1) == (-1, -1, -1)
    wx.wxpy_reduce_tuned_set(0, 5, 16, 6)  # warp-tiled: six levels inside a thread
    assert wx.wxpy_reduce_tuned_get(0) == (5, 16, 6)
    wx.wxpy_reduce_tuned_set(0, -1, -1, -1)
    for bad in ((2, 0, 16, 0), (-1, 0, 16, 0), (0, 7, 16, 0), (0, 0, 17, 0), (0, 0, 16, 7),
                (1, 0, 16, 1)):  # dot's terms can be negative: no integer tree sums
        with pytest.raises(wx.WxpyError) as e:
            wx.wxpy_reduce_tuned_set(*bad)
        assert e.value.status == wx.WXPY_EINVAL


def test_load_reduce_section(tmp_path):
    path = tmp_path / "r.json"
    path.write_text(json.dumps({"format": "wxpy-tune-1", "device": "X",
                                "vecops": [{"class": 3, "add_offload": 1, "mul_sixteenths": 10}],
                                "reduce": [{"kind": 0, "variant": 0, "mul_sixteenths": 8,
                                            "sum_levels": 2},
                                           {"kind": 1, "variant": 3, "mul_sixteenths": 16,
                                            "sum_levels": 0}],
                                "entries": [{"key": 4, "variant": 11}]}))
    wx.wxpy_tune_cache_load(str(path), check_device=False)
    assert wx.wxpy_reduce_tuned_get(0) == (0, 8, 2)
    assert wx.wxpy_reduce_tuned_get(1) == (3, 16, 0)
    assert wx.wxpy_vecops_tuned_get(3) == (1, 10)
    assert wx.wxpy_tune_get(4) == 11


@pytest.mark.parametrize("entry", [{"kind": 2, "variant": 0, "mul_sixteenths": 2, "sum_levels": 0},
                                   {"kind": 1, "variant": 0, "mul_sixteenths": 2, "sum_levels": 1},
                                   {"kind": 0, "variant": 7, "mul_sixteenths": 2, "sum_levels": 0},
                                   {"kind": 0, "variant": 4, "mul_sixteenths": 2, "sum_levels": 7},
                                   {"kind": 0, "variant": 0, "mul_sixteenths": 2}])
def test_malformed_reduce_entry_stores_nothing(tmp_path, entry):
    path = tmp_path / "bad.json"
    path.write_text(json.dumps({"format": "wxpy-tune-1", "device": "X",
                                "reduce": [{"kind": 0, "variant": 0, "mul_sixteenths": 6,
                                            "sum_levels": 0}, entry],
                                "entries": [{"key": 1, "variant": 2}]}))
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy_tune_cache_load(str(path), check_device=False)
    assert e.value.status == wx.WXPY_EINVAL
    assert wx.wxpy_reduce_tuned_get(0) == (-1, -1, -1)
    assert wx.wxpy_tune_get(1) == -1
