"""Pins for the WXPY oracle: checks against mathematics, not against the oracle itself.

Each ``pin_*`` function takes a loaded oracle library (``oracle.load_library``)
and returns a list of failure messages (empty = pinned).  They are used both on
the real oracle and on planted mutants of it (``test_oracle_mutants.py``), so
that a plausible mistake anywhere in the oracle -- a dropped term, a wrong sign
or index, a transposed operand, a fused multiply-add, a short loop -- fails at
least one of them.

The operation (paper Sec. 3, Fig. 1, "vecwxpy", read as PETSc's VecWXPY) is
w[i] = RN(RN(alpha*x[i]) + y[i]) in binary64, round-to-nearest-even, no FMA.
``exact_wxpy`` below computes that value from exact rational arithmetic
(``fractions.Fraction``) with a single correctly rounded conversion per
operation, which is a different computation from the oracle's two hardware
roundings and therefore an independent check of it.
"""
from __future__ import annotations

import math
import struct
from fractions import Fraction

import numpy as np

import oracle
from paper_1309_1894_gb300 import synth

DBL_MAX = float.fromhex("0x1.fffffffffffffp+1023")
DBL_TRUE_MIN = float.fromhex("0x0.0000000000001p-1022")
DBL_MIN = float.fromhex("0x1.0p-1022")
# RN overflows to infinity once |exact| reaches DBL_MAX + ulp(DBL_MAX)/2.
OVERFLOW_THRESHOLD = Fraction(2) ** 1024 - Fraction(2) ** 970


def bits_of(v: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def same_bits(a: float, b: float) -> bool:
    """Bitwise equality, except that any NaN equals any NaN (payloads are not fixed)."""
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return bits_of(a) == bits_of(b)


def round_rn(q: Fraction) -> float:
    """Correctly rounded (nearest, ties to even) binary64 of a non-zero rational."""
    mag = abs(q)
    if mag >= OVERFLOW_THRESHOLD:
        v = math.inf
    else:
        # CPython's int / int true division is correctly rounded (ties to even,
        # subnormals included).
        v = mag.numerator / mag.denominator
    return -v if q < 0 else v


def exact_mul(a: float, b: float) -> float:
    """RN(a*b) from the exact product, with IEEE special cases."""
    if math.isnan(a) or math.isnan(b):
        return math.nan
    neg = (math.copysign(1.0, a) < 0) != (math.copysign(1.0, b) < 0)
    if math.isinf(a) or math.isinf(b):
        if a == 0.0 or b == 0.0:
            return math.nan
        return -math.inf if neg else math.inf
    q = Fraction(a) * Fraction(b)
    if q == 0:
        return -0.0 if neg else 0.0
    r = round_rn(q)
    if r == 0.0:  # underflow to zero keeps the sign of the exact product
        return -0.0 if neg else 0.0
    return r


def exact_add(a: float, b: float) -> float:
    """RN(a+b) from the exact sum, with IEEE special cases."""
    if math.isnan(a) or math.isnan(b):
        return math.nan
    if math.isinf(a) or math.isinf(b):
        if math.isinf(a) and math.isinf(b) and (a > 0) != (b > 0):
            return math.nan
        return a if math.isinf(a) else b
    q = Fraction(a) + Fraction(b)
    if q == 0:
        # exact zero sum: -0 only when both operands are -0 (RN rule)
        both_neg_zero = (a == 0.0 and b == 0.0 and math.copysign(1.0, a) < 0
                         and math.copysign(1.0, b) < 0)
        return -0.0 if both_neg_zero else 0.0
    return round_rn(q)


def exact_wxpy(alpha: float, x: float, y: float) -> float:
    """RN(RN(alpha*x) + y), each rounding taken from exact rational arithmetic."""
    return exact_add(exact_mul(alpha, x), y)


def special_values() -> list[float]:
    """Signed zeros, subnormals, extremes, infinities, NaN, powers of two, odd ulps."""
    v = [0.0, -0.0, DBL_TRUE_MIN, -DBL_TRUE_MIN, DBL_MIN, -DBL_MIN,
         DBL_MIN - DBL_TRUE_MIN, DBL_MAX, -DBL_MAX, math.inf, -math.inf, math.nan,
         1.0, -1.0, 0.5, 2.0, 3.0, -3.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53,
         2.0 ** -53, 2.0 ** -1000, 2.0 ** 1000, 0.1, -0.7, 1.5, 1e308, -1e-310]
    return v


def tie_and_fma_cases() -> list[tuple[float, float, float]]:
    """Hand-built (alpha, x, y) whose two roundings are easy to get wrong.

    * product ties: 3*(1+2^-52) is exactly halfway between two doubles;
    * sum ties: 1 + 2^-53 and (1+2^-52) + 2^-53 are halfway cases (even wins);
    * fused-vs-unfused: (1+2^-30)^2 - (1+2^-29) is 2^-60 if fused and 0 if not;
    * cancellation: alpha=1, y=-x gives +0;
    * overflow of the sum and of the product; underflow of the product.
    """
    e = 2.0 ** -30
    return [
        (3.0, 1.0 + 2.0 ** -52, 0.0),
        (3.0, 1.0 + 2.0 ** -52, -0.0),
        (1.0, 1.0, 2.0 ** -53),
        (1.0, 1.0 + 2.0 ** -52, 2.0 ** -53),
        (-1.0, 1.0 + 2.0 ** -52, -(2.0 ** -53)),
        (1.0 + e, 1.0 + e, -(1.0 + 2 * e)),
        (1.0 + e, -(1.0 + e), 1.0 + 2 * e),
        (1.0, 0.3, -0.3),
        (DBL_MAX, 1.0, DBL_MAX),
        (2.0, DBL_MAX, 0.0),
        (2.0 ** -600, 2.0 ** -600, 0.0),
        (-(2.0 ** -600), 2.0 ** -600, -0.0),
        (2.0 ** -537, 2.0 ** -538, 0.0),
        (0.0, math.inf, 1.0),
        (math.inf, 1.0, -math.inf),
        (0.0, 5.0, -0.0),
        (-0.0, 5.0, -0.0),
        (1.0, -0.0, -0.0),
        (1.0, -0.0, 0.0),
    ]


def random_cases(seed: int, count: int) -> tuple[float, np.ndarray, np.ndarray]:
    """One alpha and ``count`` (x, y) pairs with wide exponent spread.

    Values are U(-1,1) scaled by 2^k with k spread over a range that exercises
    cancellation, absorption and subnormal products."""
    a, x, y = synth.vectors(seed, count)
    kx = (synth.bits(seed, 11, 0, count) % np.uint64(121)).astype(np.int64) - 60
    ky = (synth.bits(seed, 12, 0, count) % np.uint64(121)).astype(np.int64) - 60
    return a, np.ldexp(x, kx), np.ldexp(y, ky)


def run_oracle(lib, alpha, x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return oracle.wxpy(alpha, x, y, library=lib)


def pin_exact_rounding(lib) -> list[str]:
    """Every element equals RN(RN(alpha*x)+y) computed exactly (random + special)."""
    fails = []
    sv = special_values()
    # all special pairs (x, y) for several alphas, including special alphas
    xs = np.array([a for a in sv for _ in sv], dtype=np.float64)
    ys = np.array([b for _ in sv for b in sv], dtype=np.float64)
    for alpha in sv + [0.75, -1.25, 1.0 + 2.0 ** -52]:
        w = run_oracle(lib, alpha, xs, ys)
        for i in range(xs.shape[0]):
            want = exact_wxpy(alpha, float(xs[i]), float(ys[i]))
            if not same_bits(float(w[i]), want):
                fails.append(f"special alpha={alpha!r} x={xs[i]!r} y={ys[i]!r}: "
                             f"got {float(w[i]).hex()} want {want.hex()}")
                if len(fails) > 10:
                    return fails
    for (alpha, xv, yv) in tie_and_fma_cases():
        w = run_oracle(lib, alpha, np.array([xv]), np.array([yv]))
        want = exact_wxpy(alpha, xv, yv)
        if not same_bits(float(w[0]), want):
            fails.append(f"tie/fma alpha={alpha!r} x={xv!r} y={yv!r}: "
                         f"got {float(w[0]).hex()} want {want.hex()}")
    for seed in (1, 2, 3):
        alpha, x, y = random_cases(synth.BASE_SEED + seed, 4000)
        w = run_oracle(lib, alpha, x, y)
        for i in range(x.shape[0]):
            want = exact_wxpy(alpha, float(x[i]), float(y[i]))
            if not same_bits(float(w[i]), want):
                fails.append(f"random seed={seed} i={i}: got {float(w[i]).hex()} "
                             f"want {want.hex()}")
                break
    return fails


def pin_closed_forms(lib) -> list[str]:
    """Closed forms that hold for every input of the synthetic distribution.

    alpha=0 gives y; y=+0 gives RN(alpha*x) (here alpha*x is never -0 except
    where x=-0 is excluded); alpha=1, y=-x gives +0; alpha=-1, y=x gives +0;
    alpha=1, y=x gives 2x exactly; alpha=2^k scales exactly."""
    fails = []
    n = 1000
    a, x, y = synth.vectors(synth.BASE_SEED + 77, n)
    x = x[x != 0.0]
    y = y[: x.shape[0]]
    y = np.where(y == 0.0, 0.25, y)

    def check(name, got, want):
        gb = got.view(np.uint64)
        wb = np.asarray(want, dtype=np.float64).view(np.uint64)
        bad = np.nonzero(gb != wb)[0]
        if bad.size:
            i = int(bad[0])
            fails.append(f"{name}: i={i} got {float(got[i]).hex()} "
                         f"want {float(np.asarray(want)[i]).hex()}")

    # alpha = 0: 0*x is +-0 and +-0 + y = y for y != 0
    check("alpha=0 -> y", run_oracle(lib, 0.0, x, y), y)
    # y = +0: RN(alpha*x) + 0 = RN(alpha*x) when alpha*x != -0 (x != 0 here)
    for alpha in (a, 1.0, -3.0, 0.1):
        check(f"y=0 -> alpha*x (alpha={alpha})",
              run_oracle(lib, alpha, x, np.zeros_like(x)),
              np.array([exact_mul(alpha, float(v)) for v in x]))
    # alpha = 1, y = -x: exact cancellation gives +0
    check("alpha=1,y=-x -> +0", run_oracle(lib, 1.0, x, -x), np.zeros_like(x))
    check("alpha=-1,y=x -> +0", run_oracle(lib, -1.0, x, x), np.zeros_like(x))
    # alpha = 1, y = x: x + x = 2x exactly
    check("alpha=1,y=x -> 2x", run_oracle(lib, 1.0, x, x), 2.0 * x)
    # alpha = 2^k, y = 0: exact scaling
    check("alpha=8,y=0 -> 8x", run_oracle(lib, 8.0, x, np.zeros_like(x)), 8.0 * x)
    # alpha = 1, y = 0 -> x (identity)
    check("alpha=1,y=0 -> x", run_oracle(lib, 1.0, x, np.zeros_like(x)), x)
    return fails


def pin_aliasing(lib) -> list[str]:
    """w == x and w == y (in place) give the same bits as the disjoint call."""
    fails = []
    a, x, y = synth.vectors(synth.BASE_SEED + 5, 257)
    want = np.array([exact_wxpy(a, float(p), float(q)) for p, q in zip(x, y)])
    xx = x.copy()
    oracle.wxpy_into(a, xx, y, xx, library=lib)
    if not np.array_equal(xx.view(np.uint64), want.view(np.uint64)):
        fails.append("w==x differs from the exact result")
    yy = y.copy()
    oracle.wxpy_into(a, x, yy, yy, library=lib)
    if not np.array_equal(yy.view(np.uint64), want.view(np.uint64)):
        fails.append("w==y differs from the exact result")
    z = x.copy()
    oracle.wxpy_into(a, z, z, z, library=lib)
    want2 = np.array([exact_wxpy(a, float(p), float(p)) for p in x])
    if not np.array_equal(z.view(np.uint64), want2.view(np.uint64)):
        fails.append("w==x==y differs from the exact result")
    return fails


def pin_bruteforce_tiny(lib) -> list[str]:
    """Every n in 0..67: element-by-element exact check, nothing written past n."""
    fails = []
    for n in range(68):
        a, x, y = synth.vectors(synth.BASE_SEED + 1000 + n, n)
        w = np.full(n + 4, np.nan)
        oracle.wxpy_into(a, x, y, w[:n], library=lib)
        for i in range(n):
            want = exact_wxpy(a, float(x[i]), float(y[i]))
            if not same_bits(float(w[i]), want):
                fails.append(f"tiny n={n} i={i}: got {float(w[i]).hex()} want {want.hex()}")
                break
        if not np.all(np.isnan(w[n:])):
            fails.append(f"tiny n={n}: wrote past the end")
    return fails


def pin_batch(lib) -> list[str]:
    """Batched oracle: segment s equals the exact result with its own alpha_s."""
    fails = []
    ns = [0, 1, 3, 17, 64, 5]
    alphas = synth.uniform_pm2(synth.BASE_SEED + 9, synth.TAG_ALPHA, len(ns))
    xs = [synth.uniform_pm1(synth.BASE_SEED + 9 + s, synth.TAG_X, n) for s, n in enumerate(ns)]
    ys = [synth.uniform_pm1(synth.BASE_SEED + 9 + s, synth.TAG_Y, n) for s, n in enumerate(ns)]
    ws = oracle.wxpy_batch(alphas, xs, ys, library=lib)
    for s, n in enumerate(ns):
        for i in range(n):
            want = exact_wxpy(float(alphas[s]), float(xs[s][i]), float(ys[s][i]))
            if not same_bits(float(ws[s][i]), want):
                fails.append(f"batch segment {s} i={i}")
                break
    return fails


ALL_PINS = [pin_exact_rounding, pin_closed_forms, pin_aliasing, pin_bruteforce_tiny,
            pin_batch]


def run_all(lib) -> dict[str, list[str]]:
    return {p.__name__: p(lib) for p in ALL_PINS}


def first_failure(lib) -> str | None:
    """Run the pins in order and return the first failure message (or None)."""
    for p in ALL_PINS:
        f = p(lib)
        if f:
            return f"{p.__name__}: {f[0]}"
    return None
