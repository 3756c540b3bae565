"""The integer-pipeline sum of two non-negative binary64 values
(csrc/fp64_addpos.cuh, used by the squared 2-norm's tree) against the host's
IEEE addition, on the CPU: random significands over every exponent gap from 0
to 70, exact ties at every gap, carries into the next binade, sums that
reach the top binade, and the operands it must leave to the hardware
instruction."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("addpos") / "libaddpos_check.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-Wall",
                    "-Werror", os.path.join(HERE, "addpos_check.cc"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.addpos_check.restype = ctypes.c_int64
    L.addpos_check.argtypes = [ctypes.c_int64, dp, dp, ctypes.POINTER(ctypes.c_int64)]
    return L


def check(L, a, b):
    a, b = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
    fast = ctypes.c_int64()
    dp = ctypes.POINTER(ctypes.c_double)
    bad = L.addpos_check(len(a), a.ctypes.data_as(dp), b.ctypes.data_as(dp), ctypes.byref(fast))
    return bad, fast.value


def sig(rng, m):
    return 1.0 + rng.integers(0, 1 << 52, m, dtype=np.int64).astype(np.float64) * 2.0 ** -52


def test_random_over_every_gap(lib):
    rng = np.random.default_rng(11)
    m = 200_000
    for gap in range(0, 71):
        e = rng.integers(-900, 900, m)
        a = np.ldexp(sig(rng, m), e)
        b = np.ldexp(sig(rng, m), e - gap)
        bad, fast = check(lib, a, b)
        assert bad == 0, gap
        assert fast == m, gap
        bad, fast = check(lib, b, a)  # either order
        assert bad == 0 and fast == m, gap


def test_ties_and_carries(lib):
    rng = np.random.default_rng(12)
    m = 100_000
    for gap in range(1, 56):
        a = np.ldexp(sig(rng, m), 3)
        # b exactly half an ulp of a times an odd multiple (ties), and just off it
        k = 2 * rng.integers(0, 1 << min(gap, 30), m) + 1
        b = np.ldexp(k.astype(np.float64), 3 - 53)
        b = b[(b > 0) & (b < a)]
        aa = a[: len(b)]
        for bb in (b, np.nextafter(b, 0), np.nextafter(b, np.inf)):
            bad, fast = check(lib, aa, bb)
            assert bad == 0, gap
    # significands of all ones: every rounding carries into the next binade
    a = np.full(m, 2.0 - 2.0 ** -52)
    b = np.ldexp(sig(rng, m), -rng.integers(0, 60, m))
    assert check(lib, a, b)[0] == 0


def test_overflow_and_slow_operands(lib):
    big = np.nextafter(np.inf, 0)  # exponent field 0x7FE: left to the hardware
    rng = np.random.default_rng(13)
    m = 50_000
    # exponent field 0x7FD: sums that carry into the top binade (field 0x7FE)
    a = np.ldexp(sig(rng, m), 1022)
    b = np.ldexp(sig(rng, m), 1022 - rng.integers(0, 3, m))
    bad, fast = check(lib, a, b)
    assert bad == 0 and fast == m
    assert ((a + b).view(np.uint64) >> 52 == 0x7FE).any()
    for x, y in ((big, 1.0), (np.inf, 1.0), (np.nan, 1.0), (1.0, 0.0), (1.0, 5e-324),
                 (0.0, 0.0), (-1.0, 2.0)):
        _, fast = check(lib, np.array([x]), np.array([y]))
        assert fast == 0, (x, y)
