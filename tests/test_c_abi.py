"""The C ABI from a plain C99 program (tests/c_abi_example.c): it compiles
against include/wxpy.h and links libwxpy.so with no C++ or torch (CPU), and on
a GPU its w and squared norm are the oracle's bits."""
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    from paper_1309_1894_gb300 import build as wbuild
    if not os.path.exists(wbuild.LIBRARY):
        wbuild.build()
    pkg = os.path.join(ROOT, "paper_1309_1894_gb300")
    exe = str(tmp_path_factory.mktemp("cabi") / "c_abi_example")
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                    os.path.join(HERE, "c_abi_example.c"), "-o", exe,
                    "-L", pkg, "-lwxpy", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                    "-Wl,-rpath," + pkg], check=True)
    return exe


def test_compiles_and_links(program):
    assert os.access(program, os.X_OK)


@pytest.mark.gpu
@pytest.mark.parametrize("n", [1, 4099, 3 * 8192 + 77])
def test_results_are_the_oracles(program, n):
    r = subprocess.run([program, str(n)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split()
    assert len(lines) == n + 2 and lines[-2] == "norm2"
    got = np.array([int(t, 16) for t in lines[:n]], dtype=np.uint64)
    i = np.arange(n)
    x = (i % 97) / 64.0 - 0.7
    y = (i % 31) / 128.0 - 0.1
    want = oracle.wxpy(0.75, x, y)
    assert np.array_equal(got, want.view(np.uint64))
    _, s = oracle.wxpy_norm2(0.75, x, y)
    assert int(lines[-1], 16) == int(np.float64(s).view(np.uint64))
