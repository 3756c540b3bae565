"""paper_1309_1894_gb300.tune_all: arguments are checked before any GPU call
(CPU), and a small run on the GPU writes a tune cache whose searched entries a
fresh table loads back."""
import json

import pytest

from paper_1309_1894_gb300 import tune_all as ta


def test_arguments_checked_first():
    with pytest.raises(ValueError):
        ta.tune_all(None, kmin=12, kmax=10)
    with pytest.raises(ValueError):
        ta.tune_all(None, classes=("aligned", "sideways"))


@pytest.mark.gpu
def test_small_run_writes_a_loadable_cache(tmp_path):
    import paper_1309_1894_gb300 as wx
    path = str(tmp_path / "tune.json")
    try:
        s = ta.tune_all(path, kmin=10, kmax=12, classes=("aligned", "xy"), quick=True,
                        batch=False, vecops_n=1 << 18, reduce_n=1 << 18)
        assert len(s["buckets"]) == 6 and all(b["rejected"] == 0 for b in s["buckets"])
        assert len(s["vecops"]["classes"]) == wx.VEC_CLASSES and len(s["reduce"]["kinds"]) == 2
        saved = json.load(open(path))
        assert saved["entries"] and saved["vecops"] and saved["reduce"]
        wx.wxpy_tune_clear()
        wx.wxpy_tune_cache_load(path, check_device=True)
        assert wx.wxpy_reduce_tuned_get(0)[0] >= 0
        assert wx.wxpy_vecops_tuned_get(0)[1] >= 0
    finally:
        wx.wxpy_tune_clear()
