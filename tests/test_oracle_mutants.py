"""Planted mistakes in the oracle must be caught by the pins (no GPU).

Each mutant is a one-token change to ``oracle/wxpy_oracle.c`` -- the kinds of
mistakes a reader would look for when checking the oracle against the paper's
definition -- compiled on the CPU into a temporary library.  The pins of
``tests/pins.py`` must reject every one of them, and accept the real oracle.
"""

import pytest

import oracle
import pins

MUTANTS = {
    "fused_multiply_add": ("double sum = prod + yi;",
                           "double sum = __builtin_fma(alpha, xi, yi); (void)prod;"),
    "dropped_y_term": ("double sum = prod + yi;", "double sum = prod; (void)yi;"),
    "wrong_sign": ("double sum = prod + yi;", "double sum = prod - yi;"),
    "transposed_operand": ("double prod = alpha * xi;", "double prod = alpha * yi;"),
    "wrong_index": ("double yi = y[i];", "double yi = y[n - 1 - i];"),
    "short_loop": ("for (i = 0; i < n; ++i)", "for (i = 0; i + 1 < n; ++i)"),
    "batch_first_alpha": ("oracle_wxpy(n[s], alpha[s],", "oracle_wxpy(n[s], alpha[0],"),
    "add_then_multiply": ("double sum = prod + yi;", "double sum = alpha * (xi + yi);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    with open(oracle.SOURCE) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"mutant_{name}.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"libmutant_{name}.so")
    oracle.build(force=True, source=str(path), output=so, extra_flags=("-lm", "-Wno-error"))
    lib = oracle.load_library(so)
    assert pins.first_failure(lib) is not None, f"mutant {name} passed every pin"


def test_real_oracle_passes_every_pin():
    assert pins.first_failure(oracle.lib()) is None
