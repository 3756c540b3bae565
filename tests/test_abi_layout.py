"""Struct layouts of the C ABI (no GPU): every ctypes mirror in the Python
binding has the size and field offsets that a C compiler gives the
declaration in include/wxpy.h."""
import ctypes
import os
import subprocess

import pytest

from paper_1309_1894_gb300 import binding, server

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MIRRORS = {
    "wxpy_device_info": binding.DeviceInfo,
    "wxpy_class_info": binding.ClassInfo,
    "wxpy_variant_info": binding.VariantInfo,
    "wxpy_tune_result": binding.TuneResult,
    "wxpy_batch_info": binding.BatchInfo,
    "wxpy_batch_tune_result": binding.BatchTuneResult,
    "wxpy_server_config": server.ServerConfig,
    "wxpy_server_stats": server.ServerStats,
    "wxpy_loadgen_config": server.LoadgenConfig,
    "wxpy_loadgen_result": server.LoadgenResult,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "wxpy.h"', "int main(void) {"]
    for cname, py in MIRRORS.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append('printf("wxpy_desc sizeof %zu\\n", sizeof(wxpy_desc));')
    for f in ("n", "alpha", "x", "y", "w"):
        lines.append(f'printf("wxpy_desc {f} %zu\\n", offsetof(wxpy_desc, {f}));')
    lines.append("return 0; }")
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines))
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    table = {}
    for line in out.splitlines():
        name, field, value = line.split()
        table[(name, field)] = int(value)
    return table


@pytest.mark.parametrize("cname", sorted(MIRRORS))
def test_ctypes_mirror_matches_c(c_layout, cname):
    py = MIRRORS[cname]
    assert ctypes.sizeof(py) == c_layout[(cname, "sizeof")]
    for f, _ in py._fields_:
        assert getattr(py, f).offset == c_layout[(cname, f)], f


def test_descriptor_matches_numpy_dtype(c_layout):
    import numpy as np
    dt = np.dtype(binding.DESC_DTYPE)
    assert dt.itemsize == c_layout[("wxpy_desc", "sizeof")] == 40
    for f in ("n", "alpha", "x", "y", "w"):
        assert dt.fields[f][1] == c_layout[("wxpy_desc", f)]
