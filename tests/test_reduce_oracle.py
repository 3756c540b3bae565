"""Pins of the update-and-reduce oracle (oracle/reduce_oracle.c) to what the
definition of the operation and the mathematics fix, not to the oracle itself:

* worked examples of the tree: values derived by hand from its definition
  (tiles of 8192 indices, halving tree e[i] += e[i + s] for s = T/2 .. 1, tile
  sums by the same tree over a power-of-two padding), chosen so that a
  sequential sum, a contiguous pairwise tree, another tile size, another
  padding or another cross-tile order each gives a different value;
* exact sums: integer-valued terms whose every partial sum is exact, so any
  order gives the exact integer sum;
* the error bound of a tree of depth d: |result - sum t_i| <= gamma_d sum |t_i|
  with gamma_d = d u / (1 - d u), u = 2^-53, against exact rational sums of the
  correctly rounded terms;
* identities between independent pieces: w equals the wxpy oracle, norm2
  equals a dot product with z = w, and special values propagate (NaN, inf);
* planted mutants of the oracle, each failing one of the pins above.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import pins
from paper_1309_1894_gb300 import synth

T = 8192
U = 2.0 ** -53


def same(a, b):
    return pins.same_bits(float(a), float(b))


def dot_of(values, positions, n, L=None):
    """dot form with w = values placed at positions (alpha = 1, y = 0, z = 1)."""
    x = np.zeros(n)
    x[list(positions)] = values
    return oracle.wxpy_dot(1.0, x, np.zeros(n), np.ones(n), library=L)[1]


def check_worked_examples(L):
    b = 2.0 ** 53
    # one tile: e[0] = 2^53, e[1] = -2^53, e[4096] = 1, e[4097] = 1.
    # s = 4096: e[0] = RN(2^53 + 1) = 2^53 (tie, even), e[1] = -2^53 + 1 (exact);
    # zeros elsewhere; s = 1: 2^53 + (-2^53 + 1) = 1.  (Sequential or contiguous
    # pairwise: 2; tiles of 4096: 0 + 2 = 2.)
    if not same(dot_of([b, -b, 1.0, 1.0], [0, 1, 4096, 4097], 4098, L), 1.0):
        return "halving tree within a tile"
    # the same four values across two tiles: tile 0 sums to 0, tile 1 to 2,
    # and the tile sums add to 2.
    if not same(dot_of([b, -b, 1.0, 1.0], [0, 1, T, T + 1], T + 2, L), 2.0):
        return "tile boundary"
    # norm2: w = [2^27, 1, 0, 1, 0, 1, 0, 1] -> terms [2^54, 1, 0, 1, 0, 1, 0, 1];
    # s = 4: indices 1 + 5 and 3 + 7 give 2, 2; s = 2: 4 at index 1; s = 1:
    # 2^54 + 4 (exact).  Sequential: each 1 is lost under half an ulp (2): 2^54.
    w = np.array([2.0 ** 27, 1, 0, 1, 0, 1, 0, 1])
    if not same(oracle.wxpy_norm2(1.0, w, np.zeros(8), library=L)[1], 2.0 ** 54 + 4):
        return "norm2 halving order"
    # five tiles, P' = 8: tile sums [2^53, 1, 1, 0, -2^53] padded with zeros:
    # s = 4: p0 = 2^53 + (-2^53) = 0, p1 = 1 + 0, p2 = 1 + 0, p3 = 0;
    # s = 2: p0 = 0 + 1 = 1, p1 = 1 + 0 = 1; s = 1: 2.  (Sequential over tile
    # sums: RN(2^53 + 1) = 2^53, again, then 0.)
    got = dot_of([b, 1.0, 1.0, -b], [0, T, 2 * T, 4 * T], 4 * T + 1, L)
    if not same(got, 2.0):
        return "cross-tile tree"
    # padding with +0: a dot term -0 alone in its tile gives +0 after
    # RN(-0 + +0) = +0.
    x = np.array([-0.0] + [0.0] * 4)
    if not same(oracle.wxpy_dot(1.0, x, np.array([-0.0] * 5), np.ones(5), library=L)[1], 0.0):
        return "signed zero padding"
    if not same(oracle.wxpy_dot(1.0, np.zeros(0), np.zeros(0), np.zeros(0), library=L)[1], 0.0):
        return "empty"
    return None


def check_exact_integer_sums(L):
    rng = np.random.default_rng(11)
    for n in (1, 7, T - 1, T, T + 1, 3 * T + 5, 50001):
        w = rng.integers(-1000, 1001, n).astype(np.float64)
        z = rng.integers(-1000, 1001, n).astype(np.float64)
        # |terms| < 2^20, n < 2^16: every partial sum is an integer below 2^53
        _, s = oracle.wxpy_norm2(1.0, w, np.zeros(n), library=L)
        if s != float(sum(int(v) * int(v) for v in w)):
            return f"norm2 exact n={n}"
        _, d = oracle.wxpy_dot(1.0, w, np.zeros(n), z, library=L)
        if d != float(sum(int(a) * int(b) for a, b in zip(w, z))):
            return f"dot exact n={n}"
    return None


def depth(n):
    ntiles = max(1, -(-n // T))
    return 13 + math.ceil(math.log2(ntiles)) if ntiles > 1 else 13


def check_error_bound(L):
    for n, seed in ((5, 1), (T + 3, 2), (4 * T + 77, 3), (20000, 4)):
        alpha, x, y = synth.vectors(synth.BASE_SEED + 40 + seed, n)
        z = synth.uniform_pm1(seed, synth.TAG_Y + 7, n)
        w, s = oracle.wxpy_norm2(alpha, x, y, library=L)
        w2, d = oracle.wxpy_dot(alpha, x, y, z, library=L)
        if not np.array_equal(w.view(np.uint64), w2.view(np.uint64)):
            return "w differs between norm2 and dot"
        for terms, got in (([pins.exact_mul(float(v), float(v)) for v in w], s),
                           ([pins.exact_mul(float(a), float(b)) for a, b in zip(w, z)], d)):
            exact = sum((Fraction(t) for t in terms), Fraction(0))
            mag = sum((abs(Fraction(t)) for t in terms), Fraction(0))
            k = depth(n)
            gamma = Fraction(k) * Fraction(U) / (1 - Fraction(k) * Fraction(U))
            if abs(Fraction(got) - exact) > gamma * mag:
                return f"error bound n={n}"
    return None


def check_update_and_identities(L):
    for n in (0, 1, 67, T + 1):
        alpha, x, y = synth.vectors(synth.BASE_SEED + 60 + n, n)
        w, s = oracle.wxpy_norm2(alpha, x, y, library=L)
        if not np.array_equal(w.view(np.uint64), oracle.wxpy(alpha, x, y).view(np.uint64)):
            return f"w vs wxpy n={n}"
        _, d = oracle.wxpy_dot(alpha, x, y, w, library=L)  # z holds the values of w
        if not same(s, d):
            return f"norm2 vs dot(w, w) n={n}"
    # special values: NaN anywhere gives NaN; +inf terms give +inf; inf - inf NaN
    n = 100
    x = np.ones(n)
    x[37] = math.nan
    if not math.isnan(oracle.wxpy_norm2(1.0, x, np.zeros(n), library=L)[1]):
        return "NaN propagation"
    x[37] = math.inf
    if oracle.wxpy_norm2(1.0, x, np.zeros(n), library=L)[1] != math.inf:
        return "inf"
    z = np.ones(n)
    z[5] = -math.inf
    if not math.isnan(oracle.wxpy_dot(1.0, x, np.zeros(n), z, library=L)[1]):
        return "inf - inf"
    # overflow of a square
    if oracle.wxpy_norm2(1.0, np.array([1e200]), np.zeros(1), library=L)[1] != math.inf:
        return "square overflow"
    return None


CHECKS = [check_worked_examples, check_exact_integer_sums, check_error_bound,
          check_update_and_identities]


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_reduce_oracle(check):
    assert check(oracle.reduce_lib()) is None


MUTANTS = {
    "sequential_tile": ("    for (s = len / 2; s >= 1; s /= 2)\n        for (i = 0; i < s; ++i)\n"
                        "            e[i] = e[i] + e[i + s];\n    return e[0];",
                        "    for (i = 1; i < len; ++i)\n        e[0] = e[0] + e[i];\n"
                        "    (void)s;\n    return e[0];"),
    "contiguous_pairwise": ("            e[i] = e[i] + e[i + s];",
                            "            e[i] = e[2 * i] + e[2 * i + 1];"),
    "tile_4096": ("#define TILE 8192", "#define TILE 4096"),
    "pad_with_last": ("            tile[i] = g < n ? t[g] : 0.0;",
                      "            tile[i] = g < n ? t[g] : t[n - 1];"),
    "fused_update": ("        double sum = prod + y[i];\n        w[i] = sum;\n        t[i] = sum * sum;",
                     "        double sum = __builtin_fma(alpha, x[i], y[i]);\n        w[i] = sum;\n"
                     "        t[i] = sum * sum; (void)prod;"),
    "square_of_x": ("        t[i] = sum * sum;", "        t[i] = x[i] * x[i];"),
    "cross_tile_sequential": ("    *result = halving_sum(partial, padded);",
                              "    for (k = 1; k < padded; ++k)\n        partial[0] = partial[0] + partial[k];\n"
                              "    *result = partial[0];"),
    "drops_last_tile": ("    ntiles = (n + TILE - 1) / TILE;", "    ntiles = n / TILE > 0 ? n / TILE : 1;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_reduce_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(oracle.REDUCE_SOURCE).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"lib{name}.so")
    oracle.build(force=True, source=str(path), output=so, extra_flags=("-lm", "-Wno-error"))
    L = oracle.load_reduce_library(so)
    assert any(c(L) is not None for c in CHECKS), f"mutant {name} passed every pin"
