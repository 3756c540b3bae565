"""The integer-pipeline binary64 products (csrc/fp64_mul.cuh: mul_rn_core on
a split coefficient, and sqr_rn_core) against the host's IEEE multiplication,
on the CPU: random operands over the whole exponent range and both signs,
products on either side of 2 (the 2^105 split of the 106-bit product),
rounding carries into the next binade, exact ties at both splits, the edges
of the normal result range, and the operands and results it must leave to the
hardware instruction (flagged slow, by the rule worked out here with exact
integers)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("mulint") / "libmul_check.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-Wall",
                    "-Werror", os.path.join(HERE, "mul_check.cc"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.mul_check.restype = ctypes.c_int64
    L.mul_check.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_uint8)]
    return L


def check(L, a, b=None, want_slow=False):
    """(pairs differing from the host's product, pairs on the fast path[, slow flags])."""
    a = np.ascontiguousarray(a, np.float64)
    square = b is None
    b = a if square else np.ascontiguousarray(b, np.float64)
    fast = ctypes.c_int64()
    slow = np.zeros(len(a), np.uint8)
    dp = ctypes.POINTER(ctypes.c_double)
    bad = L.mul_check(len(a), a.ctypes.data_as(dp), b.ctypes.data_as(dp), int(square),
                      ctypes.byref(fast), slow.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return (bad, fast.value, slow.astype(bool)) if want_slow else (bad, fast.value)


def sig(rng, m):
    return 1.0 + rng.integers(0, 1 << 52, m, dtype=np.int64).astype(np.float64) * 2.0 ** -52


def expected_slow(a, b):
    """The fast path's documented domain, from exact integers: both operands
    normal and finite, and the unrounded result's biased exponent (ea + eb -
    1023 + t, t = 1 when the 106-bit significand product reaches 2^105) in
    [1, 0x7FD]."""
    out = []
    for x, y in zip(a.tolist(), b.tolist()):
        ux = int(np.float64(x).view(np.uint64))
        uy = int(np.float64(y).view(np.uint64))
        ex, ey = (ux >> 52) & 0x7FF, (uy >> 52) & 0x7FF
        if not (1 <= ex <= 0x7FE and 1 <= ey <= 0x7FE):
            out.append(True)
            continue
        p = ((ux & ((1 << 52) - 1)) | (1 << 52)) * ((uy & ((1 << 52) - 1)) | (1 << 52))
        t = int(p >= 1 << 105)
        e = ex + ey - 1023 + t
        out.append(not 1 <= e <= 0x7FD)
    return np.array(out)


def test_random_products_and_squares(lib):
    rng = np.random.default_rng(21)
    m = 400_000
    ea = rng.integers(-500, 500, m)
    eb = rng.integers(-500, 500, m)
    a = np.ldexp(sig(rng, m), ea) * rng.choice([-1.0, 1.0], m)
    b = np.ldexp(sig(rng, m), eb) * rng.choice([-1.0, 1.0], m)
    assert check(lib, a, b) == (0, m)
    assert check(lib, a) == (0, m)


def test_either_side_of_two_and_carries(lib):
    rng = np.random.default_rng(22)
    k = rng.integers(-(1 << 20), 1 << 20, 200_000)
    r2 = np.sqrt(2.0)
    a = r2 * (1 + k * 2.0 ** -52)  # significand products straddle 2
    b = r2 * (1 - rng.integers(-(1 << 20), 1 << 20, len(k)) * 2.0 ** -52)
    assert check(lib, a, b) == (0, len(a))
    assert check(lib, a) == (0, len(a))
    # significands of all ones times values just above 1: every rounding carries
    m = 100_000
    a = np.full(m, 2.0 - 2.0 ** -52) * np.ldexp(1.0, rng.integers(-300, 300, m))
    b = 1 + rng.integers(0, 1 << 12, m) * 2.0 ** -52
    assert check(lib, a, b) == (0, m)


def test_exact_ties_round_to_even(lib):
    """b = 1.5 makes the 106-bit product 3A 2^51: below 2 (A < 4/3 2^52) an
    odd A leaves exactly half an ulp, at or above 2 A = 2 mod 4 does; both
    cases round to even.  A few other short significands add more ties."""
    rng = np.random.default_rng(23)
    m = 100_000
    big = 1 << 52
    lo = big + 2 * rng.integers(0, (big // 3) // 2 - 1, m) + 1            # odd, A < 4/3 2^52
    hi = big + (big // 3) + 4 * rng.integers(1, (2 * big // 3) // 4 - 1, m) + 2  # A = 2 mod 4
    for A in (lo, hi):
        a = A.astype(np.float64) * 2.0 ** -52
        assert np.all(a.astype(np.float64) * 2.0 ** 52 == A)  # exactly representable
        for s in (1.0, -1.0):
            assert check(lib, s * a, np.full(m, 1.5)) == (0, m)
            assert check(lib, np.full(m, 1.5), s * a) == (0, m)  # the coefficient side too
    a = sig(rng, m)
    for short in (1.25, 1.75, 1.125, 1.375, 1.0625, 1.3125, 1.5 + 2.0 ** -52):
        assert check(lib, a, np.full(m, short)) == (0, m)


def _sqrt_mod_pow2(r, k):
    """An odd x with x*x = r (mod 2^k), for r = 1 (mod 8) (Hensel lifting)."""
    x = 1
    for i in range(3, k):
        if ((x * x - r) >> i) & 1:
            x += 1 << (i - 1)
    assert (x * x - r) % (1 << k) == 0
    return x


def test_just_above_a_tie_by_the_lowest_word(lib):
    """Products whose discarded part is one half plus a few units in the lowest
    32 bits of the 106-bit product (bits 32 up to the round bit all zero): only
    those low bits say the product is above the tie, so they must count as
    sticky -- with the kept part even, dropping them would round down.  Made
    from exact integers: B = A^-1 R modulo 2^(52 + t) for a chosen remainder
    R = 2^(51 + t) + d, 0 < d < 2^32; squares from a square root of R modulo
    2^(52 + t)."""
    rng = np.random.default_rng(25)
    big = 1 << 52
    pa, pb, sq = [], [], []
    while len(pa) < 4000 or len(sq) < 2000:
        t = int(rng.integers(0, 2))
        mod = 1 << (52 + t)
        d = int(rng.integers(1, 1 << 32))
        r = (1 << (51 + t)) + d
        if len(pa) < 4000:
            A = big + 2 * int(rng.integers(0, big // 2)) + 1  # odd: invertible modulo 2^k
            B = (pow(A, -1, mod) * r) % mod
            if big <= B < 2 * big and (A * B >= 1 << 105) == bool(t):
                P = A * B
                assert P % mod == r and (P >> (52 + t)) % 2 in (0, 1)
                pa.append(A)
                pb.append(B)
        if len(sq) < 2000 and d % 8 == 1:
            x = _sqrt_mod_pow2(r, 52 + t)
            for A in (x % big + big, (mod - x) % big + big):
                if (A * A >= 1 << 105) == bool(t) and (A * A) % mod == r:
                    sq.append(A)
    kept_even = sum(((A * B) >> 52 >> ((A * B) >> 105)) % 2 == 0 for A, B in zip(pa, pb))
    assert kept_even > 1000  # the case where a lost sticky bit would round the wrong way
    e = rng.integers(-400, 400, len(pa))
    a = np.ldexp(np.array(pa, dtype=np.float64) * 2.0 ** -52, e)
    b = np.ldexp(np.array(pb, dtype=np.float64) * 2.0 ** -52, -e // 2)
    assert all(int(v) == A for v, A in zip(np.array(pa, dtype=np.float64), pa))  # exact
    for s in (1.0, -1.0):
        assert check(lib, s * a, b) == (0, len(a))
    q = np.array(sq, dtype=np.float64) * 2.0 ** -52
    assert check(lib, q) == (0, len(q))
    assert check(lib, -np.ldexp(q, 100)) == (0, len(q))


def test_normal_range_edges_and_slow_flags(lib):
    """Products whose unrounded exponent lands at and around both ends of the
    normal range: the fast path covers exactly the documented domain, and is
    exact wherever it is taken."""
    rng = np.random.default_rng(24)
    m = 4_000
    cases = []
    for esum in (-1024, -1023, -1022, -1021, 1020, 1021, 1022, 1023):
        ea = rng.integers(-600, 600, m)
        ea = np.clip(ea, esum - 1023, esum + 1022)  # both exponents stay in range
        a = np.ldexp(sig(rng, m), ea)
        b = np.ldexp(sig(rng, m), esum - ea)
        cases.append((a, b))
    a = np.concatenate([c[0] for c in cases])
    b = np.concatenate([c[1] for c in cases])
    with np.errstate(over="ignore", under="ignore"):
        bad, fast, slow = check(lib, a, b, want_slow=True)
    assert bad == 0
    assert np.array_equal(slow, expected_slow(a, b))
    assert 0 < fast < len(a)  # both sides of both edges are present
    sq = np.ldexp(sig(rng, m), rng.choice([-512, -511, 510, 511], m))
    with np.errstate(over="ignore", under="ignore"):
        bad, fast, slow = check(lib, sq, want_slow=True)
    assert bad == 0 and np.array_equal(slow, expected_slow(sq, sq)) and 0 < fast < m


def test_special_operands_are_left_to_the_hardware(lib):
    sv = np.array([0.0, -0.0, 5e-324, -2.5e-310, np.inf, -np.inf, np.nan, 1.5, -3.0,
                   np.nextafter(np.inf, 0)])
    a = np.repeat(sv, len(sv))
    b = np.tile(sv, len(sv))
    with np.errstate(all="ignore"):
        bad, fast, slow = check(lib, a, b, want_slow=True)
        assert bad == 0 and np.array_equal(slow, expected_slow(a, b))
        bad, fast, slow = check(lib, sv, want_slow=True)
    assert bad == 0 and np.array_equal(slow, expected_slow(sv, sv))
    assert fast == 2  # 1.5 and -3.0
