"""The oracle checked against mathematics (no GPU).

Paper Sec. 2: variants are judged against the outputs of the plain reference
code, so that reference code (``oracle/wxpy_oracle.c``) must itself be pinned to
something other than itself: exact rational arithmetic, closed forms, aliasing
identities and brute force on tiny inputs (see ``tests/pins.py``).
"""
import ctypes

import numpy as np
import pytest

import oracle
import pins


@pytest.fixture(scope="module")
def lib():
    return oracle.lib()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(lib, pin):
    fails = pin(lib)
    assert not fails, "\n".join(fails[:10])


def test_rejects_bad_arguments(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    x = np.zeros(4)
    p = x.ctypes.data_as(dp)
    assert lib.oracle_wxpy(-1, 1.0, p, p, p) == 1
    assert lib.oracle_wxpy(4, 1.0, None, p, p) == 1
    assert lib.oracle_wxpy(4, 1.0, p, None, p) == 1
    assert lib.oracle_wxpy(4, 1.0, p, p, None) == 1
    assert lib.oracle_wxpy(0, 1.0, None, None, None) == 0


def test_exact_helper_against_known_roundings():
    """The exact-arithmetic helper itself, on cases whose answers are textbook facts."""
    # 0.1 + 0.2 rounds to 0x1.3333333333334p-2 (the well-known 0.30000000000000004)
    assert pins.exact_add(0.1, 0.2) == 0.30000000000000004
    # 1 + 2^-53 is a tie and rounds to even (1.0); 1 + 2^-53 + 2^-105 rounds up
    assert pins.exact_add(1.0, 2.0 ** -53) == 1.0
    assert pins.exact_add(1.0 + 2.0 ** -52, 2.0 ** -53) == 1.0 + 2.0 ** -51
    # 3 * (1 + 2^-52) = 3 + 3*2^-52 is halfway between 3+2^-51 and 3+2^-50: even wins
    assert pins.exact_mul(3.0, 1.0 + 2.0 ** -52) == 3.0 + 2.0 ** -50
    # signed zeros
    assert str(pins.exact_add(-0.0, -0.0)) == "-0.0"
    assert str(pins.exact_add(-0.0, 0.0)) == "0.0"
    assert str(pins.exact_add(1.5, -1.5)) == "0.0"
    assert str(pins.exact_mul(-(2.0 ** -600), 2.0 ** -600)) == "-0.0"
    # overflow and the smallest subnormal
    assert pins.exact_add(pins.DBL_MAX, pins.DBL_MAX) == float("inf")
    assert pins.exact_mul(2.0 ** -537, 2.0 ** -537) == pins.DBL_TRUE_MIN
    assert pins.exact_mul(2.0 ** -538, 2.0 ** -537) == 0.0  # tie at half of min -> 0
