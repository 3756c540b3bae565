"""The C ABI library (no GPU): it builds, loads, exports every declared symbol,
and its host-side logic (validation, classification, variant space) is right.
No call here launches a kernel."""
import ctypes
import os
import subprocess

import pytest

import abi
import paper_1309_1894_gb300 as wx
from paper_1309_1894_gb300 import binding
from paper_1309_1894_gb300 import build as wbuild


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(wbuild.LIBRARY):
        wbuild.build()
    return wx.lib()


def test_every_declared_symbol_is_exported(lib):
    names = abi.declared_functions()
    assert "wxpy" in names and len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", wbuild.LIBRARY],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in names:
        getattr(lib, n)  # resolvable through dlsym too


def test_binding_covers_every_symbol():
    names = set(abi.declared_functions())
    bound = set(binding.SIGNATURES)
    assert names <= bound, f"not bound in Python: {sorted(names - bound)}"


def test_strerror(lib):
    for s in range(10):
        assert wx.strerror(s) and wx.strerror(s) != "unknown status"
    assert wx.strerror(99) == "unknown status"


def test_variant_space_roundtrip(lib):
    count = wx.wxpy_variant_count()
    per = 3 * 4 * 4 * 5 * 3 * 4 * 4
    assert count == per * 4
    # ids without the FP64 offload knob keep their meaning (offload is the top digit),
    # and so do those of the earlier offload values 1 and 2
    assert wx.wxpy_variant_describe(per - 1)["fp64_offload"] == 0
    assert wx.wxpy_variant_describe(per)["fp64_offload"] == 1
    assert wx.wxpy_variant_describe(3 * per - 1)["fp64_offload"] == 2
    assert wx.wxpy_variant_describe(3 * per)["fp64_offload"] == 3
    seen = set()
    for vid in range(0, count, 7):
        d = wx.wxpy_variant_describe(vid)
        assert d["id"] == vid
        fields = {k: v for k, v in d.items() if k != "id"}
        assert wx.wxpy_variant_encode(**fields) == vid
        seen.add(tuple(fields.values()))
    assert len(seen) == len(range(0, count, 7))
    with pytest.raises(wx.WxpyError):
        wx.wxpy_variant_describe(count)
    with pytest.raises(wx.WxpyError):
        wx.wxpy_variant_describe(-1)
    with pytest.raises(wx.WxpyError):
        wx.wxpy_variant_encode(vec_bytes=24, unroll=1, threads=128, blocks_per_sm=0,
                               cache=0, carveout=-1, streams=1)


BASE = 1 << 40  # a pointer value; never dereferenced by wxpy_classify


@pytest.mark.parametrize("off", [0, 8, 16, 24])
def test_classify_coaligned(lib, off):
    n = 1000
    c = wx.wxpy_classify(n, BASE + off, BASE + 65536 + off, BASE + 2 * 65536 + off)
    assert c["align"] == 32 and c["alias"] == 0
    assert c["head"] == ((32 - off) % 32) // 8
    assert c["bucket"] == 9


def test_classify_mixed_alignment(lib):
    n = 100
    assert wx.wxpy_classify(n, BASE + 0, BASE + 65536 + 16, BASE + 2 * 65536)["align"] == 16
    assert wx.wxpy_classify(n, BASE + 0, BASE + 65536 + 8, BASE + 2 * 65536 + 24)["align"] == 8
    assert wx.wxpy_classify(n, BASE + 8, BASE + 65536 + 8, BASE + 2 * 65536 + 24)["align"] == 16


def test_classify_aliasing(lib):
    n = 64
    x, y, w = BASE, BASE + 4096, BASE + 8192
    assert wx.wxpy_classify(n, x, y, x)["alias"] == wx.ALIAS_WX
    assert wx.wxpy_classify(n, x, y, y)["alias"] == wx.ALIAS_WY
    assert wx.wxpy_classify(n, x, x, w)["alias"] == wx.ALIAS_XY
    assert wx.wxpy_classify(n, x, x, x)["alias"] == wx.ALIAS_XY | wx.ALIAS_WX | wx.ALIAS_WY
    # x and y may overlap partially: both are only read
    assert wx.wxpy_classify(n, x, x + 8, w)["alias"] == 0


def test_classify_buckets(lib):
    for k in range(0, 40):
        for n in (1 << k, (1 << k) + 3):
            if n >= (1 << (k + 1)):
                continue
            assert wx.wxpy_classify(n, BASE, BASE + (1 << 44), BASE + (2 << 44))["bucket"] == k
    # 2^k and 2^k + 3 share a bucket (k >= 2)
    assert wx.wxpy_classify(0, 0, 0, 0)["bucket"] == -1


@pytest.mark.parametrize("args,status", [
    ((-1, BASE, BASE + 4096, BASE + 8192), wx.WXPY_EINVAL),
    ((10, 0, BASE + 4096, BASE + 8192), wx.WXPY_EINVAL),
    ((10, BASE, 0, BASE + 8192), wx.WXPY_EINVAL),
    ((10, BASE, BASE + 4096, 0), wx.WXPY_EINVAL),
    ((10, BASE + 4, BASE + 4096, BASE + 8192), wx.WXPY_EINVAL),
    ((10, BASE, BASE + 4096, BASE + 8), wx.WXPY_EOVERLAP),
    ((10, BASE, BASE + 4096, BASE + 4096 - 8), wx.WXPY_EOVERLAP),
    ((10, BASE, BASE + 4096, BASE + 4096 + 72), wx.WXPY_EOVERLAP),
])
def test_validation_errors(lib, args, status):
    with pytest.raises(wx.WxpyError) as e:
        wx.wxpy_classify(*args)
    assert e.value.status == status
    # the launching entry points reject the same arguments before any CUDA call
    n, x, y, w = args
    assert lib.wxpy(n, 1.0, x, y, w, None) == status
    assert lib.wxpy_run_variant(0, n, 1.0, x, y, w, None) == status


def test_empty_call_is_a_noop_without_cuda(lib):
    assert lib.wxpy(0, 1.0, None, None, None, None) == 0
    assert lib.wxpy_run_variant(5, 0, 1.0, None, None, None, None) == 0
    assert lib.wxpy_reference(0, 1.0, None, None, None, None) == 0


def test_error_message_is_thread_local_text(lib):
    assert lib.wxpy(-5, 1.0, None, None, None, None) == wx.WXPY_EINVAL
    msg = lib.wxpy_last_error_message().decode()
    assert "negative" in msg


def test_set_variant_range(lib):
    with pytest.raises(wx.WxpyError):
        wx.wxpy_set_variant(wx.wxpy_variant_count())
    wx.wxpy_set_variant(3)
    wx.wxpy_set_variant(-1)


def test_host_entry_validation_before_cuda(lib):
    assert lib.wxpy_host(-1, 1.0, BASE, BASE + 4096, BASE + 8192, None) == wx.WXPY_EINVAL
    assert lib.wxpy_host(10, 1.0, BASE, BASE + 4096, BASE + 8, None) == wx.WXPY_EOVERLAP
    assert lib.wxpy_host(0, 1.0, None, None, None, None) == 0
    for bad in ((100, 3, 0), (4096 + 8, 3, 0), (4096, 0, 0), (4096, 9, 0), (4096, 3, 2)):
        assert lib.wxpy_host_config(*bad) == wx.WXPY_EINVAL
    assert lib.wxpy_host_config(1 << 22, 3, 1) == 0
    assert lib.wxpy_host_config(1 << 22, 3, 0) == 0


def test_vecops_validation_before_cuda(lib):
    import ctypes
    P = ctypes.c_void_p
    assert lib.wxpy_axpbypcz(-1, 1.0, 1.0, 1.0, BASE, BASE + 4096, BASE + 8192, None) == wx.WXPY_EINVAL
    assert lib.wxpy_axpbypcz(10, 1.0, 1.0, 1.0, BASE, BASE + 4096, BASE + 8, None) == wx.WXPY_EOVERLAP
    assert lib.wxpy_axpbypcz(10, 1.0, 1.0, 1.0, BASE, BASE + 4, BASE + 8192, None) == wx.WXPY_EINVAL
    assert lib.wxpy_pointwise_mult(10, BASE, BASE + 4096, BASE + 4096 + 16, None) == wx.WXPY_EOVERLAP
    assert lib.wxpy_pointwise_mult(0, None, None, None, None) == 0
    al = (ctypes.c_double * 2)(1.0, 2.0)
    xs = (P * 2)(BASE, BASE + 8)  # x[1] overlaps y partially
    assert lib.wxpy_maxpy(10, 2, al, xs, BASE + 16, None) == wx.WXPY_EOVERLAP
    assert lib.wxpy_maxpy(10, -1, al, xs, BASE + 65536, None) == wx.WXPY_EINVAL
    assert lib.wxpy_axpy(-1, 1.0, BASE, BASE + 4096, None) == wx.WXPY_EINVAL
    for bad in ((3, 0), (-2, 0), (0, 17), (0, -2)):
        assert lib.wxpy_vecops_pipes(*bad) == wx.WXPY_EINVAL
    assert lib.wxpy_vecops_pipes(2, 16) == 0
    assert lib.wxpy_vecops_pipes(-1, -1) == 0
    assert lib.wxpy_debug_vecops_drop_tile(-2) == wx.WXPY_EINVAL
    assert lib.wxpy_debug_vecops_drop_tile(-1) == 0
    assert lib.wxpy_debug_reduce_drop_chunk(-2) == wx.WXPY_EINVAL
    assert lib.wxpy_debug_reduce_drop_chunk(-1) == 0
    for bad in (-2, 7):
        assert lib.wxpy_reduce_variant(bad) == wx.WXPY_EINVAL
    assert lib.wxpy_reduce_variant(-1) == 0
    for bad in (-2, 7):
        assert lib.wxpy_reduce_sum_levels(bad) == wx.WXPY_EINVAL
    assert lib.wxpy_reduce_sum_levels(-1) == 0


def test_reduce_validation_before_cuda(lib):
    ws_need = lib.wxpy_reduce_workspace_bytes(100)
    assert ws_need == 256 + 8 and lib.wxpy_reduce_workspace_bytes(8193) == 256 + 16
    assert lib.wxpy_reduce_workspace_bytes(3 * 8192 + 1) == 256 + 8 * 4
    assert lib.wxpy_reduce_workspace_bytes(-1) == -1
    X, Y, W, Z, R, WS = (BASE + k * 65536 for k in range(6))
    args = dict(n=100, x=X, y=Y, w=W, z=Z, r=R, ws=WS, wsb=ws_need)

    def norm2(**kw):
        a = {**args, **kw}
        return lib.wxpy_norm2(a["n"], 1.0, a["x"], a["y"], a["w"], a["r"], a["ws"], a["wsb"], None)

    def dot(**kw):
        a = {**args, **kw}
        return lib.wxpy_dot(a["n"], 1.0, a["x"], a["y"], a["w"], a["z"], a["r"], a["ws"], a["wsb"],
                            None)

    for f in (norm2, dot):
        assert f(n=-1) == wx.WXPY_EINVAL
        assert f(r=0) == wx.WXPY_EINVAL
        assert f(r=R + 4) == wx.WXPY_EINVAL
        assert f(x=X + 4) == wx.WXPY_EINVAL
        assert f(ws=0) == wx.WXPY_EINVAL
        assert f(wsb=ws_need - 8) == wx.WXPY_EINVAL
        assert f(ws=WS + 8) == wx.WXPY_EINVAL
        assert f(w=X + 8) == wx.WXPY_EOVERLAP
        assert f(r=W + 16) == wx.WXPY_EOVERLAP
        assert f(ws=X + 64) == wx.WXPY_EOVERLAP
    assert dot(z=0) == wx.WXPY_EINVAL
    assert dot(w=Z + 8) == wx.WXPY_EOVERLAP
    assert lib.wxpy_reduce_pipes(17) == wx.WXPY_EINVAL
    assert lib.wxpy_reduce_pipes(-2) == wx.WXPY_EINVAL
    assert lib.wxpy_reduce_pipes(-1) == 0


def test_python_surface_names():
    """The Python names of the package's public surface: wxpy(alpha, x, y, out=...),
    tune(n) and Server, with no GPU call."""
    import inspect
    sig = inspect.signature(wx.wxpy)
    assert list(sig.parameters)[:3] == ["alpha", "x", "y"] and "out" in sig.parameters
    assert wx.tune.__doc__ and callable(wx.tune)
    assert inspect.isclass(wx.Server)
    with pytest.raises(ValueError):
        wx.wxpy(1.0, None, None, w=object(), out=object())


@pytest.mark.parametrize("value,forced", [("4112", True), ("-3", False), ("12x", False),
                                          ("99999999", False)])
def test_force_variant_from_environment(value, forced):
    """WXPY_FORCE_VARIANT forces the lookup from the process's start (no GPU
    call: the lookup classifies pointer values); invalid values are ignored,
    and an explicit wxpy_set_variant(-1) still wins."""
    import os
    import subprocess
    import sys
    code = r'''
import ctypes, sys
import paper_1309_1894_gb300 as wx
lib = wx.lib()
info = wx.binding.VariantInfo()
src = ctypes.c_int()
base = 1 << 40
assert lib.wxpy_lookup(1 << 20, base, base + (1 << 24), base + (2 << 24), ctypes.byref(info),
                       ctypes.byref(src)) == 0
first = src.value
assert lib.wxpy_set_variant(-1) == 0
assert lib.wxpy_lookup(1 << 20, base, base + (1 << 24), base + (2 << 24), ctypes.byref(info),
                       ctypes.byref(src)) == 0
print(first, src.value)
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, WXPY_FORCE_VARIANT=value, PYTHONPATH=root)
    env.pop("WXPY_TUNE_CACHE", None)
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    first, after = (int(t) for t in r.stdout.split())
    assert first == (2 if forced else 0)
    assert after == 0
