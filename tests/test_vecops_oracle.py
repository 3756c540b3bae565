"""The sibling-kernel oracle (VecAXPY, VecAYPX, VecAXPBYPCZ, VecMAXPY,
VecPointwiseMult) pinned to mathematics (no GPU): every product and sum equals
the exact rational value rounded once; closed forms; planted mistakes caught."""
import numpy as np
import pytest

import oracle
import pins
from paper_1309_1894_gb300 import synth

E = pins.exact_mul
A = pins.exact_add


def wide(seed, n):
    """Values U(-1,1) * 2^k, k in [-60, 60], plus the special values."""
    v = synth.uniform_pm1(seed, synth.TAG_X, n)
    k = (synth.bits(seed, 13, 0, n) % np.uint64(121)).astype(np.int64) - 60
    return np.concatenate([np.ldexp(v, k), np.array(pins.special_values())])


def inputs(seed, count):
    xs = [wide(seed + i, count) for i in range(4)]
    n = min(len(x) for x in xs)
    return [x[:n] for x in xs]


def same(got, want):
    return all(pins.same_bits(float(a), float(b)) for a, b in zip(got, want))


def check_axpy(L):
    x, y, _, _ = inputs(1, 400)
    for alpha in (0.75, -1.5, pins.DBL_MAX, 2.0 ** -600, 0.0):
        want = [A(E(alpha, float(a)), float(b)) for a, b in zip(x, y)]
        if not same(oracle.axpy(alpha, x, y, library=L), want):
            return f"axpy alpha={alpha}"
    return None


def check_aypx(L):
    x, y, _, _ = inputs(2, 400)
    for alpha in (0.75, -1.5, 3.0):
        want = [A(float(a), E(alpha, float(b))) for a, b in zip(x, y)]
        if not same(oracle.aypx(alpha, x, y, library=L), want):
            return f"aypx alpha={alpha}"
    return None


def check_axpby(L):
    x, y, _, _ = inputs(7, 400)
    for (a, b) in ((0.75, -1.25), (1.0, 1.0), (2.0 ** -40, 2.0 ** 40), (-3.0, 0.5)):
        want = [A(E(a, float(p)), E(b, float(q))) for p, q in zip(x, y)]
        if not same(oracle.axpby(a, b, x, y, library=L), want):
            return f"axpby {a},{b}"
    return None


def check_axpbypcz(L):
    x, y, z, _ = inputs(3, 400)
    for (a, b, c) in ((0.75, -1.25, 3.0), (1.0, 1.0, 1.0), (2.0 ** -40, 2.0 ** 40, -0.5)):
        want = [A(A(E(a, float(p)), E(b, float(q))), E(c, float(r))) for p, q, r in zip(x, y, z)]
        if not same(oracle.axpbypcz(a, b, c, x, y, z, library=L), want):
            return f"axpbypcz {a},{b},{c}"
    return None


def check_maxpy(L):
    x0, x1, x2, y = inputs(4, 300)
    al = [0.5, -3.0, 1.0 + 2.0 ** -52]
    for m in (0, 1, 2, 3):
        want = []
        for i in range(len(y)):
            acc = float(y[i])
            for j, xj in enumerate((x0, x1, x2)[:m]):
                acc = A(acc, E(al[j], float(xj[i])))
            want.append(acc)
        if not same(oracle.maxpy(al[:m], [x0, x1, x2][:m], y, library=L), want):
            return f"maxpy m={m}"
    return None


def check_pmult(L):
    x, y, _, _ = inputs(5, 400)
    want = [E(float(a), float(b)) for a, b in zip(x, y)]
    return None if same(oracle.pmult(x, y, library=L), want) else "pmult"


def check_closed_forms(L):
    x, y, z, _ = [v[:300] for v in inputs(6, 300)]
    x, y, z = (np.where(v == 0.0, 0.5, v) for v in (x, y, z))
    finite = np.isfinite(x) & np.isfinite(y) & np.isfinite(z)
    x, y, z = x[finite], y[finite], z[finite]
    # beta = gamma = 0 leaves RN(alpha*x) when that product is not zero
    got = oracle.axpbypcz(3.0, 0.0, 0.0, x, y, z, library=L)
    want = np.array([E(3.0, float(v)) for v in x])
    keep = want != 0.0
    if not np.array_equal(got[keep].view(np.uint64), want[keep].view(np.uint64)):
        return "axpbypcz beta=gamma=0"
    # maxpy with all alphas 0 leaves y (y != 0)
    if not np.array_equal(oracle.maxpy([0.0, 0.0], [x, z], y, library=L).view(np.uint64),
                          y.view(np.uint64)):
        return "maxpy zeros"
    # pmult by one is the identity
    if not np.array_equal(oracle.pmult(x, np.ones_like(x), library=L).view(np.uint64),
                          x.view(np.uint64)):
        return "pmult by 1"
    # maxpy is m successive axpy calls (the left-to-right reading, y the running sum)
    al = [0.5, -3.0, 1.0 + 2.0 ** -52]
    xs = [x, z, np.ldexp(y, -3)]
    acc = y
    for a_j, x_j in zip(al, xs):
        acc = oracle.axpy(a_j, x_j, acc, library=L)
    if not np.array_equal(oracle.maxpy(al, xs, y, library=L).view(np.uint64), acc.view(np.uint64)):
        return "maxpy vs successive axpy"
    # axpby with beta = 1 is axpy (RN(1*y) = y); axpby with alpha = 0 is RN(beta*y) for
    # nonzero products
    if not np.array_equal(oracle.axpby(0.75, 1.0, x, y, library=L).view(np.uint64),
                          oracle.axpy(0.75, x, y, library=L).view(np.uint64)):
        return "axpby beta=1 vs axpy"
    got = oracle.axpby(0.0, -2.5, x, y, library=L)
    want = np.array([E(-2.5, float(v)) for v in y])
    keep = want != 0.0
    if not np.array_equal(got[keep].view(np.uint64), want[keep].view(np.uint64)):
        return "axpby alpha=0"
    # axpy agrees with the wxpy oracle (two independent implementations)
    if not np.array_equal(oracle.axpy(0.75, x, y, library=L).view(np.uint64),
                          oracle.wxpy(0.75, x, y).view(np.uint64)):
        return "axpy vs wxpy"
    return None


CHECKS = [check_axpy, check_aypx, check_axpby, check_axpbypcz, check_maxpy, check_pmult,
          check_closed_forms]


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_vecops_oracle(check):
    assert check(oracle.vec_lib()) is None


MUTANTS = {
    "axpbypcz_right_to_left": ("double s1 = ax + by;\n        double s2 = s1 + cz;",
                               "double s1 = by + cz;\n        double s2 = ax + s1;"),
    "maxpy_fused": ("            acc = acc + prod;",
                    "            acc = __builtin_fma(alpha[j], x[j][i], acc); (void)prod;"),
    "aypx_swapped": ("double prod = alpha * y[i];\n        double sum = x[i] + prod;",
                     "double prod = alpha * x[i];\n        double sum = y[i] + prod;"),
    "pmult_square": ("double prod = x[i] * y[i];", "double prod = x[i] * x[i];"),
    "axpby_beta_on_x": ("        double by = beta * y[i];\n        double sum = ax + by;",
                        "        double by = beta * x[i];\n        double sum = ax + by;"),
    "maxpy_alpha0": ("double prod = alpha[j] * x[j][i];", "double prod = alpha[0] * x[j][i];"),
    "maxpy_drops_last": ("        for (j = 0; j < m; ++j) {\n            double prod",
                         "        for (j = 0; j + 1 < m; ++j) {\n            double prod"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_vecops_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(oracle.VEC_SOURCE).read()
    assert src.count(old) == 1
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"lib{name}.so")
    oracle.build(force=True, source=str(path), output=so, extra_flags=("-lm", "-Wno-error"))
    L = oracle.load_vec_library(so)
    assert any(c(L) is not None for c in CHECKS), f"mutant {name} passed every pin"
