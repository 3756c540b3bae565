"""The stored special-value fixture (no GPU).

``tests/golden/special_cases.txt`` was written by ``make_special_cases.py`` from
the oracle; here every row is re-derived from exact rational arithmetic, and the
oracle must still reproduce it."""
import os

import numpy as np

import oracle
import pins

PATH = os.path.join(os.path.dirname(__file__), "golden", "special_cases.txt")


def load_rows():
    rows = []
    with open(PATH) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, x, y, w, label = line.split()
            rows.append((float.fromhex(a), float.fromhex(x), float.fromhex(y),
                         float.fromhex(w), label))
    return rows


def test_fixture_matches_exact_arithmetic():
    rows = load_rows()
    assert len(rows) > 500
    for (a, x, y, w, label) in rows:
        assert pins.same_bits(w, pins.exact_wxpy(a, x, y)), (label, a, x, y, w)


def test_oracle_reproduces_fixture():
    for (a, x, y, w, label) in load_rows():
        got = oracle.wxpy(a, np.array([x]), np.array([y]))[0]
        assert pins.same_bits(float(got), w), (label, a, x, y)
