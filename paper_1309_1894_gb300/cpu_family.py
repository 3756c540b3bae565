"""ctypes binding of ``libwxpy_cpu.so``: the host VecWXPY family and its search
(the paper's own CPU experiment, Sec. 3, Fig. 1, on this machine's cores).

Argument marshalling only; every loop runs in the C library.  Arrays are 1-D
contiguous float64 numpy arrays (host memory).  The library is separate from
the GPU one and never touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .binding import WxpyError

HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY = os.path.join(HERE, "libwxpy_cpu.so")

TUNE_SINGLE = 1
TUNE_WARM = 2

_lock = threading.Lock()
_lib = None


class CpuVariantInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int32), ("flavour", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("vec", ctypes.c_int32), ("unroll", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("flags", ctypes.c_char_p)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["flags"] = self.flags.decode()
        return d


class CpuTuneResult(ctypes.Structure):
    _fields_ = [("best", ctypes.c_int32), ("best_single", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("rejected", ctypes.c_int32),
                ("bucket", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("best_us", ctypes.c_double), ("best_single_us", ctypes.c_double),
                ("baseline_us", ctypes.c_double), ("reference_us", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_INT = ctypes.c_int

SIGNATURES = {
    "wxpy_cpu": (_INT, [_I64, _D, _P, _P, _P]),
    "wxpy_cpu_run_variant": (_INT, [_INT, _I64, _D, _P, _P, _P]),
    "wxpy_cpu_variant_count": (_INT, []),
    "wxpy_cpu_variant_describe": (_INT, [_INT, ctypes.POINTER(CpuVariantInfo)]),
    "wxpy_cpu_baseline_variant": (_INT, []),
    "wxpy_cpu_reference_variant": (_INT, []),
    "wxpy_cpu_tune": (_INT, [_I64, ctypes.c_uint, ctypes.POINTER(CpuTuneResult)]),
    "wxpy_cpu_tune_get": (_INT, [_INT, ctypes.POINTER(_INT)]),
    "wxpy_cpu_tune_set": (_INT, [_INT, _INT]),
    "wxpy_cpu_tune_clear": (_INT, []),
    "wxpy_cpu_last_error": (ctypes.c_char_p, []),
    "wxpy_cpu_tune_cache_save": (_INT, [ctypes.c_char_p]),
    "wxpy_cpu_tune_cache_load": (_INT, [ctypes.c_char_p, _INT]),
}


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIBRARY):
                raise RuntimeError(f"{LIBRARY} is not built; build it with "
                                   "paper_1309_1894_gb300.build.build_cpu()")
            h = ctypes.CDLL(LIBRARY)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(h, name)
                f.restype, f.argtypes = res, args
            _lib = h
        return _lib


def _check(status: int, what: str) -> None:
    if status != 0:
        raise WxpyError(status, what, lib().wxpy_cpu_last_error().decode())


def _vec(a, name: str):
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or a.ndim != 1 \
            or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a 1-D contiguous float64 numpy array")
    return a.size, a.ctypes.data


def wxpy_cpu(alpha: float, x, y, w=None, variant: int | None = None):
    """w = RN(RN(alpha*x) + y) on host arrays (the tuned variant, else the
    baseline; or `variant`); returns w."""
    import numpy as np
    n, px = _vec(x, "x")
    ny, py = _vec(y, "y")
    if w is None:
        w = np.empty_like(x)
    nw, pw = _vec(w, "w")
    if not (n == ny == nw):
        raise ValueError("length mismatch")
    if variant is None:
        _check(lib().wxpy_cpu(n, alpha, px, py, pw), "wxpy_cpu")
    else:
        _check(lib().wxpy_cpu_run_variant(variant, n, alpha, px, py, pw), "wxpy_cpu_run_variant")
    return w


def variant_count() -> int:
    return lib().wxpy_cpu_variant_count()


def describe(variant: int) -> dict:
    info = CpuVariantInfo()
    _check(lib().wxpy_cpu_variant_describe(variant, ctypes.byref(info)), "describe")
    return info.as_dict()


def baseline_variant() -> int:
    return lib().wxpy_cpu_baseline_variant()


def reference_variant() -> int:
    return lib().wxpy_cpu_reference_variant()


def tune(n: int, single_thread: bool = False, warm: bool = False) -> dict:
    res = CpuTuneResult()
    flags = (TUNE_SINGLE if single_thread else 0) | (TUNE_WARM if warm else 0)
    _check(lib().wxpy_cpu_tune(n, flags, ctypes.byref(res)), "wxpy_cpu_tune")
    d = res.as_dict()
    d["best_variant"] = describe(res.best)
    d["best_single_variant"] = describe(res.best_single)
    return d


def tune_get(bucket: int) -> int:
    v = _INT()
    _check(lib().wxpy_cpu_tune_get(bucket, ctypes.byref(v)), "tune_get")
    return v.value


def tune_set(bucket: int, variant: int) -> None:
    _check(lib().wxpy_cpu_tune_set(bucket, variant), "tune_set")


def tune_clear() -> None:
    _check(lib().wxpy_cpu_tune_clear(), "tune_clear")


def tune_cache_save(path: str) -> None:
    _check(lib().wxpy_cpu_tune_cache_save(path.encode()), "tune_cache_save")


def tune_cache_load(path: str, check_machine: bool = True) -> None:
    _check(lib().wxpy_cpu_tune_cache_load(path.encode(), int(check_machine)), "tune_cache_load")
