"""CPU oracle for VecWXPY, w = alpha*x + y in FP64 (paper Sec. 2 and Sec. 3, Fig. 1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
library under ``paper_1309_1894_gb300/`` never imports it and shares no code
with it.

The paper's method (Sec. 2) compares every generated code variant with the
outputs of the plain reference code; ``wxpy_oracle.c`` is that reference code,
compiled with ``-O2 -ffp-contract=off -fno-fast-math`` so that the product and
the sum are rounded separately (no fused multiply-add).  This module builds it
with gcc and exposes it to numpy through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "wxpy_oracle.c")
LIBRARY = os.path.join(HERE, "liboracle.so")

# -ffp-contract=off: the product and the sum are two separate roundings.
# -fno-fast-math: subnormals kept, IEEE semantics kept.
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-std=c99", "-Wall", "-Wextra", "-Werror"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False, source: str = SOURCE, output: str = LIBRARY,
          extra_flags: tuple = ()) -> str:
    """Compile ``source`` into the shared library ``output`` with gcc."""
    if (not force and os.path.exists(output)
            and os.path.getmtime(output) >= os.path.getmtime(source)):
        return output
    tmp = output + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, *extra_flags, source, "-o", tmp]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, output)
    return output


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_wxpy.restype = ctypes.c_int
    lib.oracle_wxpy.argtypes = [ctypes.c_int64, ctypes.c_double, dp, dp, dp]
    lib.oracle_wxpy_batch.restype = ctypes.c_int
    lib.oracle_wxpy_batch.argtypes = [
        ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), dp,
        ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(dp)]
    return lib


def load_library(path: str) -> ctypes.CDLL:
    """Load an oracle shared library built from ``wxpy_oracle.c`` (or a copy)."""
    return _bind(ctypes.CDLL(path))


def lib() -> ctypes.CDLL:
    """The oracle library, built on first use."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(a: np.ndarray, name: str) -> None:
    if a.dtype != np.float64 or a.ndim != 1 or not a.flags.c_contiguous:
        raise ValueError(f"{name} must be a contiguous 1-D float64 array")


def wxpy_into(alpha: float, x: np.ndarray, y: np.ndarray, w: np.ndarray,
              library: ctypes.CDLL | None = None) -> np.ndarray:
    """w[i] = RN(RN(alpha*x[i]) + y[i]) in place; w may be x or y itself."""
    for a, nm in ((x, "x"), (y, "y"), (w, "w")):
        _check(a, nm)
    n = x.shape[0]
    if y.shape[0] != n or w.shape[0] != n:
        raise ValueError("x, y and w must have the same length")
    L = library if library is not None else lib()
    rc = L.oracle_wxpy(n, float(alpha), _dptr(x), _dptr(y), _dptr(w))
    if rc != 0:
        raise RuntimeError(f"oracle_wxpy returned {rc}")
    return w


def wxpy(alpha: float, x: np.ndarray, y: np.ndarray,
         library: ctypes.CDLL | None = None) -> np.ndarray:
    """A new array w with w[i] = RN(RN(alpha*x[i]) + y[i])."""
    w = np.empty_like(x)
    return wxpy_into(alpha, x, y, w, library)


def wxpy_batch(alphas, xs, ys, library: ctypes.CDLL | None = None):
    """Batched oracle: one output array per segment (a list)."""
    count = len(xs)
    ws = [np.empty_like(x) for x in xs]
    for a in (*xs, *ys, *ws):
        _check(a, "segment")
    n = np.array([x.shape[0] for x in xs], dtype=np.int64)
    al = np.ascontiguousarray(alphas, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    xp = (dp * max(count, 1))(*[_dptr(a) for a in xs])
    yp = (dp * max(count, 1))(*[_dptr(a) for a in ys])
    wp = (dp * max(count, 1))(*[_dptr(a) for a in ws])
    L = library if library is not None else lib()
    rc = L.oracle_wxpy_batch(count, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             _dptr(al), xp, yp, wp)
    if rc != 0:
        raise RuntimeError(f"oracle_wxpy_batch returned {rc}")
    return ws
