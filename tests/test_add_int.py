"""The integer-pipeline binary64 sum of any two values (csrc/fp64_emu.cuh:
add_rn_core, the sum the single-call kernels may move off the FP64 pipeline)
against the host's IEEE addition, on the CPU: both signs over every exponent
gap from 0 to 70, cancellation down to an exact zero (+0), exact ties at
every gap, carries into the next binade and borrows out of it, and the edges
of the normal range, where the slow flag must match the documented domain:
an operand that is zero, subnormal, infinite or NaN, or a nonzero result that
is subnormal or overflows."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("addint") / "libadd_check.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-Wall",
                    "-Werror", os.path.join(HERE, "add_check.cc"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.add_check.restype = ctypes.c_int64
    L.add_check.argtypes = [ctypes.c_int64, dp, dp, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_uint8)]
    return L


def check(L, a, b):
    """(pairs differing from the host's sum, pairs on the fast path, slow flags)."""
    a, b = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
    fast = ctypes.c_int64()
    slow = np.zeros(len(a), np.uint8)
    dp = ctypes.POINTER(ctypes.c_double)
    bad = L.add_check(len(a), a.ctypes.data_as(dp), b.ctypes.data_as(dp), ctypes.byref(fast),
                      slow.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return bad, fast.value, slow.astype(bool)


def field(v):
    return (np.asarray(v, np.float64).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)


def expected_slow(a, b):
    """An operand outside the normal range, or a nonzero result that is not
    normal.  (Two doubles are multiples of 2^-1074, so a sum below 2^-1022 is
    exact as a subnormal: the unbounded-exponent rounding of the fast path
    and the host's rounding only part where the result leaves the normal
    range.)"""
    with np.errstate(all="ignore"):
        r = a + b
    op = (field(a) == 0) | (field(a) == 0x7FF) | (field(b) == 0) | (field(b) == 0x7FF)
    res = (r != 0) & ((field(r) == 0) | (field(r) == 0x7FF))
    return op | res


def sig(rng, m):
    return 1.0 + rng.integers(0, 1 << 52, m, dtype=np.int64).astype(np.float64) * 2.0 ** -52


def test_every_gap_both_signs(lib):
    rng = np.random.default_rng(31)
    m = 60_000
    for gap in range(0, 71):
        e = rng.integers(-900, 900, m)
        a = np.ldexp(sig(rng, m), e) * rng.choice([-1.0, 1.0], m)
        b = np.ldexp(sig(rng, m), e - gap) * rng.choice([-1.0, 1.0], m)
        for x, y in ((a, b), (b, a)):
            bad, fast, _ = check(lib, x, y)
            assert bad == 0 and fast == m, gap


def test_cancellation(lib):
    rng = np.random.default_rng(32)
    m = 100_000
    a = np.ldexp(sig(rng, m), rng.integers(-900, 900, m))
    # the same value (exact zero, +0 either way round), a neighbour, a few ulps off
    k = rng.integers(0, 1 << 20, m)
    for b in (-a, -np.nextafter(a, 0), -np.nextafter(a, np.inf), -(a + k * np.spacing(a)),
              -(a * (1 - k * 2.0 ** -53))):
        bad, fast, slow = check(lib, a, b)
        assert bad == 0 and fast == m
        bad, fast, slow = check(lib, b, a)
        assert bad == 0 and fast == m
    zero = check(lib, np.array([1.5, -7.25]), np.array([-1.5, 7.25]))
    assert zero[:2] == (0, 2)  # +0 from both signs, bitwise


def test_ties_carries_and_borrows(lib):
    rng = np.random.default_rng(33)
    m = 50_000
    for gap in range(1, 56):
        a = np.ldexp(sig(rng, m), 3)
        k = 2 * rng.integers(0, 1 << min(gap, 30), m) + 1  # odd multiples of half an ulp
        b = np.ldexp(k.astype(np.float64), 3 - 53)
        keep = (b > 0) & (b < a)
        aa, b = a[keep], b[keep]
        for bb in (b, np.nextafter(b, 0), np.nextafter(b, np.inf)):
            for s in (1.0, -1.0):
                bad, fast, _ = check(lib, aa, s * bb)
                assert bad == 0 and fast == len(aa), gap
    # all-ones significands: additions carry into the next binade
    a = np.full(m, 2.0 - 2.0 ** -52) * np.ldexp(1.0, rng.integers(-300, 300, m))
    b = a * np.ldexp(sig(rng, m), -rng.integers(0, 60, m)) / 2
    assert check(lib, a, b)[:2] == (0, m)
    # powers of two minus a little: subtractions borrow out of the binade
    a = np.ldexp(1.0, rng.integers(-300, 300, m))
    b = -a * np.ldexp(sig(rng, m), -rng.integers(1, 60, m))
    assert check(lib, a, b)[:2] == (0, m)


def test_range_edges_and_slow_flags(lib):
    rng = np.random.default_rng(34)
    m = 20_000
    big = np.nextafter(np.inf, 0)
    tiny = 2.0 ** -1022
    cases = [
        # results around the overflow edge
        (np.ldexp(sig(rng, m), 1023), np.ldexp(sig(rng, m), 1023 - rng.integers(0, 3, m))),
        (np.full(m, big), np.ldexp(sig(rng, m), 970 - rng.integers(0, 5, m))),
        # results around the smallest normal, from both sides
        (np.ldexp(sig(rng, m), -1021), -np.ldexp(sig(rng, m), -1021 - rng.integers(0, 2, m))),
        (np.full(m, tiny) * sig(rng, m), -np.full(m, tiny)),
    ]
    a = np.concatenate([c[0] for c in cases])
    b = np.concatenate([c[1] for c in cases])
    bad, fast, slow = check(lib, a, b)
    assert bad == 0
    assert np.array_equal(slow, expected_slow(a, b))
    assert 0 < fast < len(a)
    sv = np.array([0.0, -0.0, 5e-324, -2.5e-310, tiny, np.inf, -np.inf, np.nan, 1.5, -3.0, big])
    a, b = np.repeat(sv, len(sv)), np.tile(sv, len(sv))
    bad, fast, slow = check(lib, a, b)
    assert bad == 0 and np.array_equal(slow, expected_slow(a, b))
