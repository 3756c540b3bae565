"""Write ``special_cases.txt``: special-value WXPY cases with the oracle's outputs.

The paper prints no worked example (its only result, Fig. 1, is a timing plot
whose image is missing), so the stored expected values are written by this
script, which calls only ``oracle/``.  ``tests/test_golden.py`` re-derives each
row from exact rational arithmetic, so the file is pinned to mathematics and
not only to the oracle.  Run from the repository root:

    python tests/golden/make_special_cases.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import pins  # noqa: E402


def rows():
    sv = pins.special_values()
    out = []
    for (a, x, y) in pins.tie_and_fma_cases():
        out.append((a, x, y, "tie_or_fma"))
    for a in (0.0, -0.0, 1.0, -1.0, 3.0, 2.0 ** -1074, float("inf")):
        for x in sv:
            for y in (0.0, -0.0, 1.0, -(2.0 ** -1074), float("-inf")):
                out.append((a, x, y, "special"))
    return out


def main():
    rs = rows()
    path = os.path.join(HERE, "special_cases.txt")
    with open(path, "w") as f:
        f.write("# WXPY special cases: alpha x y w (binary64 hex), label.\n")
        f.write("# w = RN(RN(alpha*x) + y) (paper Sec. 3, Fig. 1 'vecwxpy', read as\n")
        f.write("# PETSc VecWXPY; Sec. 2 reference results), written by\n")
        f.write("# make_special_cases.py from the CPU oracle.\n")
        for (a, x, y, label) in rs:
            w = oracle.wxpy(a, np.array([x]), np.array([y]))[0]
            f.write(f"{float(a).hex()} {float(x).hex()} {float(y).hex()} "
                    f"{float(w).hex()} {label}\n")
    print(f"wrote {len(rs)} rows to {path}")


if __name__ == "__main__":
    main()
