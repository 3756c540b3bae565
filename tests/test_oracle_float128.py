"""The oracle against binary128 arithmetic (no GPU): ten million cases.

``float128_pin.c`` computes RN(RN(alpha*x) + y) by another route than the
oracle's double operations: the product exact in _Float128, one rounding to
double, the sum exact in _Float128 when the exponent gap is at most 59, one
rounding to double.  Every checked case must agree bit for bit; the cases it
cannot compute exactly are counted and must stay a small minority.  The
planted mutants of the oracle must fail this pin too.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from test_oracle_mutants import MUTANTS

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("f128") / "libfloat128_pin.so")
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-Wall", "-Werror", os.path.join(HERE, "float128_pin.c"), "-o", so, "-lm"],
                   check=True)
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.pin_check.restype = ctypes.c_int64
    L.pin_check.argtypes = [ctypes.c_int64, ctypes.c_double, dp, dp, dp,
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def check(L, alpha, x, y, w):
    c, s = ctypes.c_int64(), ctypes.c_int64()
    bad = L.pin_check(len(x), alpha, _p(x), _p(y), _p(w), ctypes.byref(c), ctypes.byref(s))
    return bad, c.value, s.value


def cases(seed, m, spread):
    """x, y: random signs and 53-bit significands, exponents in [-spread, spread]."""
    rng = np.random.default_rng(seed)
    def one():
        sig = 1.0 + rng.integers(0, 1 << 52, m, dtype=np.int64).astype(np.float64) * 2.0 ** -52
        return np.ldexp(sig * rng.choice([-1.0, 1.0], m), rng.integers(-spread, spread + 1, m))
    return one(), one()


ALPHAS = [1.0, -1.0, 0.5, 3.0, 1.5, -0.75, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52, 0.1, -1.9999999,
          2.0 ** 30, 2.0 ** -30, 1.4142135623730951, -2.718281828459045, 1e-3, 7.0, 0.0, -0.0,
          1.25 + 2.0 ** -40, 65536.5]


def test_ten_million_cases_agree(checker):
    total = checked = 0
    per = 500_000
    for k, alpha in enumerate(ALPHAS):
        x, y = cases(1000 + k, per, spread=30 if k % 2 else 8)
        w = oracle.wxpy(alpha, x, y)
        bad, c, s = check(checker, alpha, x, y, w)
        assert bad == 0, f"alpha={alpha!r}: {bad} of {c} checked cases differ"
        total += per
        checked += c
    assert total == 10_000_000
    assert checked >= 0.95 * total, checked


def test_ties_and_cancellation(checker):
    # products that land exactly half an ulp from two doubles, sums that tie or cancel
    k = np.arange(1, 200001, dtype=np.float64)
    x = 1.0 + k * 2.0 ** -52
    for alpha in (3.0, 1.5, 0.75, -1.5):
        for y in (np.zeros_like(x), -alpha * x, np.full_like(x, 2.0 ** -53), np.ldexp(x, -53)):
            y = np.ascontiguousarray(y)
            w = oracle.wxpy(alpha, x, y)
            bad, c, _ = check(checker, alpha, x, y, w)
            assert bad == 0 and c == len(x), (alpha, bad, c)


# every single-call mutant (the batch-path one is caught by the batched pins)
@pytest.mark.parametrize("name", sorted(m for m in MUTANTS if m != "batch_first_alpha"))
def test_mutants_fail_the_binary128_pin(checker, tmp_path, name):
    old, new = MUTANTS[name]
    src = open(oracle.SOURCE).read()
    path = tmp_path / f"m_{name}.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"libm_{name}.so")
    oracle.build(force=True, source=str(path), output=so, extra_flags=("-lm", "-Wno-error"))
    lib = oracle.load_library(so)
    x, y = cases(77, 20000, spread=8)
    caught = False
    for alpha in (0.75, 3.0, -1.5):
        w = oracle.wxpy(alpha, x, y, library=lib)
        bad, _, _ = check(checker, alpha, x, y, w)
        caught = caught or bad > 0
    assert caught, f"mutant {name} passed the binary128 pin"


def test_sibling_oracle_against_binary128(checker):
    """The sibling oracle (vecops_oracle.c), two million cases per operation,
    each step recomputed exactly in binary128 and rounded once."""
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    L = checker
    L.pin_axpbypcz.restype = L.pin_maxpy.restype = L.pin_pmult.restype = ctypes.c_int64
    L.pin_axpbypcz.argtypes = [ctypes.c_int64] + [ctypes.c_double] * 3 + [dp] * 4 + [i64p, i64p]
    L.pin_maxpy.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, dp, dp, i64p, i64p]
    L.pin_pmult.argtypes = [ctypes.c_int64, dp, dp, dp, i64p, i64p]
    n = 500_000
    c, s = ctypes.c_int64(), ctypes.c_int64()
    for k, (al, be, ga) in enumerate(((0.75, -1.25, 3.0), (1.0, 1.0, 1.0),
                                     (2.0 ** -20, 2.0 ** 20, -0.5), (1.5, 0.1, -7.0))):
        x, y = cases(3000 + k, n, spread=20)
        z, _ = cases(3100 + k, n, spread=20)
        out = oracle.axpbypcz(al, be, ga, x, y, z)
        bad = L.pin_axpbypcz(n, al, be, ga, _p(x), _p(y), _p(z), _p(out), ctypes.byref(c),
                             ctypes.byref(s))
        # wide coefficient scales (2^-20 against 2^20) leave more exponent gaps
        # beyond binary128's exact range: a lower share is checkable there
        assert bad == 0 and c.value >= 0.8 * n, (k, bad, c.value)
    for m in (1, 3, 8):
        xs = [cases(3200 + 10 * m + j, n, spread=20)[0] for j in range(m)]
        y, _ = cases(3300 + m, n, spread=20)
        a = np.array([0.5, -3.0, 1.0 + 2.0 ** -52, 0.25, 7.0, -0.125, 1.5, 2.0][:m])
        out = oracle.maxpy(a, xs, y)
        packed = np.ascontiguousarray(np.concatenate(xs))
        bad = L.pin_maxpy(n, m, _p(a), _p(packed), _p(y), _p(out), ctypes.byref(c),
                          ctypes.byref(s))
        assert bad == 0 and c.value >= 0.95 * n, (m, bad, c.value)
    L.pin_axpby.restype = ctypes.c_int64
    L.pin_axpby.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                            i64p, i64p]
    for k, (al, be) in enumerate(((0.75, -1.25), (1.0, 1.0), (-3.0, 2.0 ** -30),
                                  (0.1, 1.0 + 2.0 ** -52))):
        x, y = cases(3500 + k, n, spread=20)
        out = oracle.axpby(al, be, x, y)
        bad = L.pin_axpby(n, al, be, _p(x), _p(y), _p(out), ctypes.byref(c), ctypes.byref(s))
        assert bad == 0 and c.value >= 0.9 * n, (k, bad, c.value)
    x, y = cases(3400, 2 * n, spread=200)
    out = oracle.pmult(x, y)
    bad = L.pin_pmult(2 * n, _p(x), _p(y), _p(out), ctypes.byref(c), ctypes.byref(s))
    assert bad == 0 and c.value >= 0.95 * 2 * n, (bad, c.value)
