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


# ---------------------------------------------------------------- sibling kernels
VEC_SOURCE = os.path.join(HERE, "vecops_oracle.c")
VEC_LIBRARY = os.path.join(HERE, "liboracle_vecops.so")
_vec_lib = None


def load_vec_library(path: str) -> ctypes.CDLL:
    """Load an oracle library built from ``vecops_oracle.c`` (or a copy)."""
    dp = ctypes.POINTER(ctypes.c_double)
    L = ctypes.CDLL(path)
    i64, d = ctypes.c_int64, ctypes.c_double
    for name, args in (("oracle_axpy", [i64, d, dp, dp]), ("oracle_aypx", [i64, d, dp, dp]),
                       ("oracle_axpby", [i64, d, d, dp, dp]),
                       ("oracle_axpbypcz", [i64, d, d, d, dp, dp, dp]),
                       ("oracle_maxpy", [i64, ctypes.c_int, dp, ctypes.POINTER(dp), dp]),
                       ("oracle_pmult", [i64, dp, dp, dp])):
        fn = getattr(L, name)
        fn.restype = ctypes.c_int
        fn.argtypes = args
    return L


def vec_lib() -> ctypes.CDLL:
    """The sibling-kernel oracle library, built on first use."""
    global _vec_lib
    with _lock:
        if _vec_lib is None:
            _vec_lib = load_vec_library(build(source=VEC_SOURCE, output=VEC_LIBRARY))
        return _vec_lib


def _vcheck(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} returned {rc}")


def axpy(alpha, x, y, library=None):
    """A new array: RN(RN(alpha*x) + y) (PETSc VecAXPY on a copy of y)."""
    out = np.array(y, dtype=np.float64, copy=True)
    _check(np.ascontiguousarray(x), "x")
    L = library or vec_lib()
    _vcheck(L.oracle_axpy(out.shape[0], float(alpha), _dptr(np.ascontiguousarray(x)), _dptr(out)),
            "oracle_axpy")
    return out


def aypx(alpha, x, y, library=None):
    """A new array: RN(x + RN(alpha*y)) (PETSc VecAYPX on a copy of y)."""
    out = np.array(y, dtype=np.float64, copy=True)
    L = library or vec_lib()
    _vcheck(L.oracle_aypx(out.shape[0], float(alpha), _dptr(np.ascontiguousarray(x)), _dptr(out)),
            "oracle_aypx")
    return out


def axpby(alpha, beta, x, y, library=None):
    """A new array: RN(RN(alpha*x) + RN(beta*y)) (PETSc VecAXPBY on a copy of y)."""
    out = np.array(y, dtype=np.float64, copy=True)
    L = library or vec_lib()
    _vcheck(L.oracle_axpby(out.shape[0], float(alpha), float(beta),
                           _dptr(np.ascontiguousarray(x)), _dptr(out)), "oracle_axpby")
    return out


def axpbypcz(alpha, beta, gamma, x, y, z, library=None):
    """A new array: RN(RN(RN(alpha*x) + RN(beta*y)) + RN(gamma*z)) (VecAXPBYPCZ on a copy of z)."""
    out = np.array(z, dtype=np.float64, copy=True)
    L = library or vec_lib()
    _vcheck(L.oracle_axpbypcz(out.shape[0], float(alpha), float(beta), float(gamma),
                              _dptr(np.ascontiguousarray(x)), _dptr(np.ascontiguousarray(y)),
                              _dptr(out)), "oracle_axpbypcz")
    return out


def maxpy(alphas, xs, y, library=None):
    """A new array: y + sum_j alpha_j x_j, each product and each sum rounded, j in order."""
    out = np.array(y, dtype=np.float64, copy=True)
    xs = [np.ascontiguousarray(x, dtype=np.float64) for x in xs]
    al = np.ascontiguousarray(alphas, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    ptrs = (dp * max(1, len(xs)))(*[_dptr(x) for x in xs])
    L = library or vec_lib()
    _vcheck(L.oracle_maxpy(out.shape[0], len(xs), _dptr(al), ptrs, _dptr(out)), "oracle_maxpy")
    return out


def pmult(x, y, library=None):
    """A new array: RN(x*y) element-wise (PETSc VecPointwiseMult)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    L = library or vec_lib()
    _vcheck(L.oracle_pmult(x.shape[0], _dptr(x), _dptr(np.ascontiguousarray(y)), _dptr(out)),
            "oracle_pmult")
    return out


REDUCE_SOURCE = os.path.join(HERE, "reduce_oracle.c")
REDUCE_LIBRARY = os.path.join(HERE, "liboracle_reduce.so")
REDUCE_TILE = 8192
_reduce_lib = None


def load_reduce_library(path: str) -> ctypes.CDLL:
    """Load an oracle library built from ``reduce_oracle.c`` (or a copy)."""
    dp = ctypes.POINTER(ctypes.c_double)
    L = ctypes.CDLL(path)
    i64, d = ctypes.c_int64, ctypes.c_double
    for name, args in (("oracle_wxpy_norm2", [i64, d, dp, dp, dp, dp]),
                       ("oracle_wxpy_dot", [i64, d, dp, dp, dp, dp, dp])):
        fn = getattr(L, name)
        fn.restype = ctypes.c_int
        fn.argtypes = args
    return L


def reduce_lib() -> ctypes.CDLL:
    """The update-and-reduce oracle library, built on first use."""
    global _reduce_lib
    with _lock:
        if _reduce_lib is None:
            _reduce_lib = load_reduce_library(build(source=REDUCE_SOURCE, output=REDUCE_LIBRARY))
        return _reduce_lib


def wxpy_norm2(alpha, x, y, library=None):
    """(w, s): w = RN(RN(alpha*x) + y) and s = TREE(RN(w*w)) (see reduce_oracle.c)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.empty_like(x)
    res = np.zeros(1)
    L = library or reduce_lib()
    _vcheck(L.oracle_wxpy_norm2(x.shape[0], float(alpha), _dptr(x), _dptr(y), _dptr(w),
                                _dptr(res)), "oracle_wxpy_norm2")
    return w, float(res[0])


def wxpy_dot(alpha, x, y, z, library=None):
    """(w, s): w = RN(RN(alpha*x) + y) and s = TREE(RN(w*z)) (see reduce_oracle.c)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    w = np.empty_like(x)
    res = np.zeros(1)
    L = library or reduce_lib()
    _vcheck(L.oracle_wxpy_dot(x.shape[0], float(alpha), _dptr(x), _dptr(y), _dptr(w), _dptr(z),
                              _dptr(res)), "oracle_wxpy_dot")
    return w, float(res[0])


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
