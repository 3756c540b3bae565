"""ctypes binding of ``libwxpy.so`` (declared in ``include/wxpy.h``).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY = os.path.join(HERE, "libwxpy.so")

WXPY_OK = 0
WXPY_EINVAL = 1
WXPY_EOVERLAP = 2
WXPY_ENOMEM = 3
WXPY_EBUDGET = 4
WXPY_ECUDA = 5
WXPY_ETIMEOUT = 6
WXPY_ENOTFOUND = 7
WXPY_EBUSY = 8
WXPY_EMISMATCH = 9

ALIAS_XY, ALIAS_WX, ALIAS_WY = 1, 2, 4


class WxpyError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({strerror(status)}){': ' + detail if detail else ''}")


class DeviceInfo(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 128), ("device", ctypes.c_int32),
                ("sm_count", ctypes.c_int32), ("cc_major", ctypes.c_int32),
                ("cc_minor", ctypes.c_int32), ("l2_bytes", ctypes.c_int64),
                ("global_bytes", ctypes.c_int64), ("runtime_version", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ClassInfo(ctypes.Structure):
    _fields_ = [("alias", ctypes.c_int32), ("align", ctypes.c_int32), ("head", ctypes.c_int32),
                ("bucket", ctypes.c_int32), ("tune_key", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class VariantInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int32), ("vec_bytes", ctypes.c_int32), ("unroll", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("cache", ctypes.c_int32), ("carveout", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("fp64_offload", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("best", VariantInfo), ("best_us", ctypes.c_double),
                ("default_us", ctypes.c_double), ("reference_us", ctypes.c_double),
                ("best_gbs", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("rejected", ctypes.c_int32), ("bucket", ctypes.c_int32),
                ("tune_key", ctypes.c_int32), ("ties", ctypes.c_int32),
                ("launch_bound", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "best"}
        d["best"] = self.best.as_dict()
        return d


TUNE_ALIGN16, TUNE_ALIGN8, TUNE_XY, TUNE_WALIAS, TUNE_QUICK, TUNE_RESIDENT = 1, 2, 4, 8, 16, 32

# sibling-kernel classes of the pipe-split search (1 .. 7: maxpy groups of 2 .. 8 terms)
VEC_AXPBYPCZ, VEC_PMULT, VEC_AXPBY, VEC_CLASSES = 0, 8, 9, 10
VEC_CLASS_NAMES = ["axpbypcz"] + [f"maxpy{m}" for m in range(2, 9)] + ["pointwise_mult", "axpby"]


class VecopsTuneResult(ctypes.Structure):
    _fields_ = [("op_class", ctypes.c_int32), ("add_offload", ctypes.c_int32),
                ("mul_sixteenths", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("rejected", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("best_us", ctypes.c_double), ("default_us", ctypes.c_double),
                ("gbs", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}
        d["op"] = VEC_CLASS_NAMES[self.op_class]
        return d


class ReduceTuneResult(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("mul_sixteenths", ctypes.c_int32), ("sum_levels", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("rejected", ctypes.c_int32),
                ("best_us", ctypes.c_double), ("default_us", ctypes.c_double),
                ("gbs", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["op"] = ("norm2", "dot")[self.kind]
        return d


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_INT = ctypes.c_int

# name -> (restype, argtypes)
SIGNATURES = {
    "wxpy_strerror": (ctypes.c_char_p, [_INT]),
    "wxpy_last_cuda_error": (_INT, []),
    "wxpy_last_error_message": (ctypes.c_char_p, []),
    "wxpy_version": (_INT, []),
    "wxpy_device_query": (_INT, [ctypes.POINTER(DeviceInfo)]),
    "wxpy_classify": (_INT, [_I64, _P, _P, _P, ctypes.POINTER(ClassInfo)]),
    "wxpy_variant_count": (_INT, []),
    "wxpy_variant_describe": (_INT, [_INT, ctypes.POINTER(VariantInfo)]),
    "wxpy_variant_encode": (_INT, [ctypes.POINTER(VariantInfo), ctypes.POINTER(_INT)]),
    "wxpy_set_variant": (_INT, [_INT]),
    "wxpy_lookup": (_INT, [_I64, _P, _P, _P, ctypes.POINTER(VariantInfo), ctypes.POINTER(_INT)]),
    "wxpy": (_INT, [_I64, _D, _P, _P, _P, _P]),
    "wxpy_run_variant": (_INT, [_INT, _I64, _D, _P, _P, _P, _P]),
    "wxpy_reference": (_INT, [_I64, _D, _P, _P, _P, _P]),
    "wxpy_debug_inject_launch_error": (_INT, [_INT, _INT]),
    "wxpy_launch_pdl": (_INT, [_INT, ctypes.POINTER(_INT)]),
    "wxpy_tune": (_INT, [_I64, ctypes.c_uint, ctypes.POINTER(TuneResult)]),
    "wxpy_tune_get": (_INT, [_INT, ctypes.POINTER(_INT)]),
    "wxpy_tune_set": (_INT, [_INT, _INT]),
    "wxpy_tune_clear": (_INT, []),
    "wxpy_tune_cache_save": (_INT, [ctypes.c_char_p]),
    "wxpy_tune_cache_load": (_INT, [ctypes.c_char_p, _INT]),
    "wxpy_fill_uniform": (_INT, [_I64, ctypes.c_uint64, ctypes.c_uint32, _I64, _D, _D, _P, _P]),
    "wxpy_batch_plan_create": (_INT, [_P, _I64, ctypes.POINTER(_P)]),
    "wxpy_batch_launch": (_INT, [_P, _P, _P]),
    "wxpy_batch_graph_launch": (_INT, [_P, _P, _P]),
    "wxpy_batch_plan_info": (_INT, [_P, _P]),
    "wxpy_batch_status": (_INT, [_P, ctypes.POINTER(ctypes.c_uint), _INT]),
    "wxpy_batch_plan_destroy": (_INT, [_P]),
    "wxpy_batch": (_INT, [_P, _P, _I64, _P]),
    "wxpy_batch_tune": (_INT, [_INT, _INT, ctypes.c_uint, _P]),
    "wxpy_batch_shape_get": (_INT, [_INT, ctypes.POINTER(_INT), ctypes.POINTER(_INT)]),
    "wxpy_batch_shape_set": (_INT, [_INT, _INT, _INT]),
    "wxpy_batch_shape_reset": (_INT, []),
    "wxpy_axpy": (_INT, [_I64, _D, _P, _P, _P]),
    "wxpy_aypx": (_INT, [_I64, _D, _P, _P, _P]),
    "wxpy_axpbypcz": (_INT, [_I64, _D, _D, _D, _P, _P, _P, _P]),
    "wxpy_maxpy": (_INT, [_I64, _INT, ctypes.POINTER(_D), ctypes.POINTER(_P), _P, _P]),
    "wxpy_pointwise_mult": (_INT, [_I64, _P, _P, _P, _P]),
    "wxpy_vecops_pipes": (_INT, [_INT, _INT]),
    "wxpy_axpby": (_INT, [_I64, _D, _D, _P, _P, _P]),
    "wxpy_vecops_status": (_INT, []),
    "wxpy_reduce_workspace_bytes": (_I64, [_I64]),
    "wxpy_norm2": (_INT, [_I64, _D, _P, _P, _P, _P, _P, _I64, _P]),
    "wxpy_dot": (_INT, [_I64, _D, _P, _P, _P, _P, _P, _P, _I64, _P]),
    "wxpy_reduce_pipes": (_INT, [_INT]),
    "wxpy_reduce_status": (_INT, []),
    "wxpy_reduce_variant": (_INT, [_INT]),
    "wxpy_reduce_sum_levels": (_INT, [_INT]),
    "wxpy_reduce_tune": (_INT, [_I64, ctypes.c_void_p]),
    "wxpy_reduce_tuned_get": (_INT, [_INT, ctypes.POINTER(_INT), ctypes.POINTER(_INT),
                                     ctypes.POINTER(_INT)]),
    "wxpy_reduce_tuned_set": (_INT, [_INT, _INT, _INT, _INT]),
    "wxpy_debug_reduce_drop_chunk": (_INT, [_I64]),
    "wxpy_vecops_tune": (_INT, [_I64, ctypes.POINTER(VecopsTuneResult)]),
    "wxpy_vecops_tuned_get": (_INT, [_INT, ctypes.POINTER(_INT), ctypes.POINTER(_INT)]),
    "wxpy_vecops_tuned_set": (_INT, [_INT, _INT, _INT]),
    "wxpy_debug_vecops_drop_tile": (_INT, [_I64]),
    "wxpy_host": (_INT, [_I64, _D, _P, _P, _P, _P]),
    "wxpy_host_config": (_INT, [_I64, _INT, _INT]),
    "wxpy_batch_launch_get": (_INT, [ctypes.POINTER(_INT), ctypes.POINTER(_INT)]),
    "wxpy_batch_launch_set": (_INT, [_INT, _INT]),
    "wxpy_batch_noalloc": (_INT, [_P, _I64, _P]),
    "wxpy_server_create": (_INT, [_P, ctypes.POINTER(_P)]),
    "wxpy_server_submit": (_INT, [_P, _I64, _D, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "wxpy_server_submit_data": (_INT, [_P, _I64, _D, _P, _P, _INT,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "wxpy_server_poll": (_INT, [_P, ctypes.c_uint64, ctypes.POINTER(_INT), ctypes.POINTER(_D)]),
    "wxpy_server_wait": (_INT, [_P, ctypes.c_uint64, _D, ctypes.POINTER(_D)]),
    "wxpy_server_result": (_INT, [_P, ctypes.c_uint64, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                  ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "wxpy_server_release": (_INT, [_P, ctypes.c_uint64]),
    "wxpy_server_get_stats": (_INT, [_P, _INT, _P]),
    "wxpy_server_destroy": (_INT, [_P]),
    "wxpy_server_loadgen": (_INT, [_P, _P, _P]),
}

_lock = threading.Lock()
_lib_handle = None


def lib() -> ctypes.CDLL:
    """The loaded ``libwxpy.so``; raises if it has not been built."""
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            if not os.path.exists(LIBRARY):
                raise RuntimeError(
                    f"{LIBRARY} is not built; build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
            h = ctypes.CDLL(LIBRARY)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib_handle = h
        return _lib_handle


def strerror(status: int) -> str:
    try:
        return lib().wxpy_strerror(status).decode()
    except Exception:  # the library may be the thing that is missing
        return "?"


def check(status: int, where: str) -> None:
    if status != WXPY_OK:
        detail = lib().wxpy_last_error_message().decode(errors="replace")
        raise WxpyError(status, where, detail)


# ---------------------------------------------------------------- marshalling
def _stream_handle(stream) -> int | None:
    """cudaStream_t of ``stream`` (torch.cuda.Stream, int or None = torch's current)."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _vec(t, name: str):
    """(n, device pointer) of a contiguous 1-D float64 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dim() != 1 or (t.numel() > 1 and t.stride(0) != 1):
        raise ValueError(f"{name} must be a contiguous 1-D tensor")
    return t.numel(), t.data_ptr()


# ---------------------------------------------------------------- API
def version() -> int:
    return lib().wxpy_version()


def wxpy_device_query() -> dict:
    info = DeviceInfo()
    check(lib().wxpy_device_query(ctypes.byref(info)), "wxpy_device_query")
    d = {f: getattr(info, f) for f, _ in info._fields_ if f != "reserved"}
    d["name"] = info.name.decode()
    return d


def wxpy_classify(n: int, x: int, y: int, w: int) -> dict:
    """Classification of a call from raw pointer values (host only)."""
    info = ClassInfo()
    check(lib().wxpy_classify(n, x, y, w, ctypes.byref(info)), "wxpy_classify")
    return {f: getattr(info, f) for f, _ in info._fields_ if f != "reserved"}


def wxpy_variant_count() -> int:
    return lib().wxpy_variant_count()


def wxpy_variant_describe(vid: int) -> dict:
    info = VariantInfo()
    check(lib().wxpy_variant_describe(vid, ctypes.byref(info)), "wxpy_variant_describe")
    return info.as_dict()


def wxpy_variant_encode(**fields) -> int:
    info = VariantInfo(id=-1, **fields)
    out = _INT()
    check(lib().wxpy_variant_encode(ctypes.byref(info), ctypes.byref(out)), "wxpy_variant_encode")
    return out.value


def wxpy_set_variant(vid: int) -> None:
    check(lib().wxpy_set_variant(vid), "wxpy_set_variant")


def wxpy_lookup(x, y, w) -> tuple[dict, int]:
    """(variant, source) that wxpy(., x, y, w) would run; source 0 default, 1 tuned, 2 forced."""
    n, px = _vec(x, "x")
    _, py = _vec(y, "y")
    _, pw = _vec(w, "w")
    info = VariantInfo()
    src = _INT()
    check(lib().wxpy_lookup(n, px, py, pw, ctypes.byref(info), ctypes.byref(src)), "wxpy_lookup")
    return info.as_dict(), src.value


def _prepare(alpha, x, y, w):
    import torch
    n, px = _vec(x, "x")
    ny, py = _vec(y, "y")
    if w is None:
        w = torch.empty_like(x)
    nw, pw = _vec(w, "w")
    if not (n == ny == nw):
        raise ValueError(f"length mismatch: x {n}, y {ny}, w {nw}")
    return n, float(alpha), px, py, pw, w


def wxpy(alpha: float, x, y, w=None, stream=None, *, out=None):
    """w = alpha*x + y (FP64, no FMA) on ``stream``; returns w (allocated if
    None).  ``out`` is another name for ``w``."""
    if out is not None:
        if w is not None and w is not out:
            raise ValueError("give w or out, not both")
        w = out
    n, a, px, py, pw, w = _prepare(alpha, x, y, w)
    check(lib().wxpy(n, a, px, py, pw, _stream_handle(stream)), "wxpy")
    return w


def wxpy_axpy(alpha: float, x, y, stream=None):
    """y <- alpha*x + y in place (VecAXPY)."""
    n, px = _vec(x, "x")
    ny, py = _vec(y, "y")
    if n != ny:
        raise ValueError("length mismatch")
    check(lib().wxpy_axpy(n, float(alpha), px, py, _stream_handle(stream)), "wxpy_axpy")
    return y


def wxpy_aypx(alpha: float, x, y, stream=None):
    """y <- x + alpha*y in place (VecAYPX)."""
    n, px = _vec(x, "x")
    ny, py = _vec(y, "y")
    if n != ny:
        raise ValueError("length mismatch")
    check(lib().wxpy_aypx(n, float(alpha), px, py, _stream_handle(stream)), "wxpy_aypx")
    return y


def wxpy_axpby(alpha: float, beta: float, x, y, stream=None):
    """y <- alpha*x + beta*y in place (VecAXPBY)."""
    n, px = _vec(x, "x")
    ny, py = _vec(y, "y")
    if n != ny:
        raise ValueError("length mismatch")
    check(lib().wxpy_axpby(n, alpha, beta, px, py, _stream_handle(stream)), "wxpy_axpby")
    return y


def wxpy_axpbypcz(alpha: float, beta: float, gamma: float, x, y, z, stream=None):
    """z <- alpha*x + beta*y + gamma*z in place (VecAXPBYPCZ)."""
    n, px = _vec(x, "x")
    _, py = _vec(y, "y")
    nz, pz = _vec(z, "z")
    if not (n == y.numel() == nz):
        raise ValueError("length mismatch")
    check(lib().wxpy_axpbypcz(n, float(alpha), float(beta), float(gamma), px, py, pz,
                              _stream_handle(stream)), "wxpy_axpbypcz")
    return z


def wxpy_maxpy(alphas, xs, y, stream=None):
    """y <- y + sum_j alphas[j]*xs[j] in place, terms in order (VecMAXPY)."""
    n, py = _vec(y, "y")
    ptrs = []
    for j, x in enumerate(xs):
        m, p = _vec(x, f"x[{j}]")
        if m != n:
            raise ValueError("length mismatch")
        ptrs.append(p)
    m = len(ptrs)
    al = (_D * max(1, m))(*[float(a) for a in alphas])
    pp = (_P * max(1, m))(*ptrs)
    check(lib().wxpy_maxpy(n, m, al, pp, py, _stream_handle(stream)), "wxpy_maxpy")
    return y


def wxpy_pointwise_mult(x, y, w=None, stream=None):
    """w <- x .* y (VecPointwiseMult)."""
    import torch
    n, px = _vec(x, "x")
    _, py = _vec(y, "y")
    if w is None:
        w = torch.empty_like(x)
    nw, pw = _vec(w, "w")
    if not (n == y.numel() == nw):
        raise ValueError("length mismatch")
    check(lib().wxpy_pointwise_mult(n, px, py, pw, _stream_handle(stream)), "wxpy_pointwise_mult")
    return w


def reduce_workspace(n: int, device=None):
    """A workspace tensor (uint8, on the device) for wxpy_norm2 / wxpy_dot of length n."""
    import torch
    return torch.empty(max(16, lib().wxpy_reduce_workspace_bytes(n)), dtype=torch.uint8,
                       device=device or "cuda")


def _reduce_args(x, y, w, result, workspace):
    import torch
    n, px = _vec(x, "x")
    ny, py = _vec(y, "y")
    if w is None:
        w = torch.empty_like(x)
    nw, pw = _vec(w, "w")
    if not (n == ny == nw):
        raise ValueError("length mismatch")
    if result is None:
        result = torch.empty(1, dtype=torch.float64, device=x.device)
    _, pr = _vec(result, "result")
    if workspace is None:
        workspace = reduce_workspace(n, x.device)
    return n, px, py, w, pw, result, pr, workspace


def wxpy_norm2(alpha: float, x, y, w=None, result=None, workspace=None, stream=None):
    """w <- RN(RN(alpha*x) + y) and result <- the fixed-tree sum of RN(w*w); returns (w, result)."""
    n, px, py, w, pw, result, pr, ws = _reduce_args(x, y, w, result, workspace)
    check(lib().wxpy_norm2(n, alpha, px, py, pw, pr, ws.data_ptr(), ws.numel(),
                           _stream_handle(stream)), "wxpy_norm2")
    return w, result


def wxpy_dot(alpha: float, x, y, z, w=None, result=None, workspace=None, stream=None):
    """w <- RN(RN(alpha*x) + y) and result <- the fixed-tree sum of RN(w*z); returns (w, result)."""
    n, px, py, w, pw, result, pr, ws = _reduce_args(x, y, w, result, workspace)
    nz, pz = _vec(z, "z")
    if nz != n:
        raise ValueError("length mismatch")
    check(lib().wxpy_dot(n, alpha, px, py, pw, pz, pr, ws.data_ptr(), ws.numel(),
                         _stream_handle(stream)), "wxpy_dot")
    return w, result


def wxpy_reduce_pipes(mul_sixteenths: int = -1) -> None:
    check(lib().wxpy_reduce_pipes(mul_sixteenths), "wxpy_reduce_pipes")


def wxpy_reduce_variant(variant: int = -1) -> None:
    """Kernel of the fused reductions for co-aligned pointers: 0 register-
    loaded, 1..3 staged shapes, -1 the default (same bits for all)."""
    check(lib().wxpy_reduce_variant(variant), "wxpy_reduce_variant")


def wxpy_reduce_sum_levels(levels: int = -1) -> None:
    """norm2: in-thread tree levels summed in the integer pipelines (0..3, -1 default)."""
    check(lib().wxpy_reduce_sum_levels(levels), "wxpy_reduce_sum_levels")


def wxpy_reduce_tune(n: int) -> list[dict]:
    """The configuration search of wxpy_norm2 and wxpy_dot on n-element vectors."""
    res = (ReduceTuneResult * 2)()
    check(lib().wxpy_reduce_tune(n, res), "wxpy_reduce_tune")
    return [r.as_dict() for r in res]


def wxpy_reduce_tuned_get(kind: int) -> tuple[int, int, int]:
    v, m, l = _INT(), _INT(), _INT()
    check(lib().wxpy_reduce_tuned_get(kind, ctypes.byref(v), ctypes.byref(m), ctypes.byref(l)),
          "wxpy_reduce_tuned_get")
    return v.value, m.value, l.value


def wxpy_reduce_tuned_set(kind: int, variant: int, mul_sixteenths: int, sum_levels: int) -> None:
    check(lib().wxpy_reduce_tuned_set(kind, variant, mul_sixteenths, sum_levels),
          "wxpy_reduce_tuned_set")


def wxpy_reduce_status() -> None:
    """Raises WxpyError(WXPY_ETIMEOUT) if a staged reduction's bounded wait ran out."""
    check(lib().wxpy_reduce_status(), "wxpy_reduce_status")


def wxpy_debug_reduce_drop_chunk(chunk: int) -> None:
    check(lib().wxpy_debug_reduce_drop_chunk(chunk), "wxpy_debug_reduce_drop_chunk")


def wxpy_vecops_pipes(add_offload: int = -1, mul_sixteenths: int = -1) -> None:
    """Pipe split of axpbypcz / maxpy / pointwise_mult (-1: the operation's default)."""
    check(lib().wxpy_vecops_pipes(add_offload, mul_sixteenths), "wxpy_vecops_pipes")


def wxpy_vecops_tune(n: int) -> list[dict]:
    """The pipe-split search of every sibling-kernel class on n-element vectors."""
    res = (VecopsTuneResult * VEC_CLASSES)()
    check(lib().wxpy_vecops_tune(n, res), "wxpy_vecops_tune")
    return [r.as_dict() for r in res]


def wxpy_vecops_tuned_get(op_class: int) -> tuple[int, int]:
    a, m = _INT(), _INT()
    check(lib().wxpy_vecops_tuned_get(op_class, ctypes.byref(a), ctypes.byref(m)),
          "wxpy_vecops_tuned_get")
    return a.value, m.value


def wxpy_vecops_tuned_set(op_class: int, add_offload: int, mul_sixteenths: int) -> None:
    check(lib().wxpy_vecops_tuned_set(op_class, add_offload, mul_sixteenths),
          "wxpy_vecops_tuned_set")


def wxpy_vecops_status() -> None:
    """Raises WxpyError(WXPY_ETIMEOUT) when a staged vector kernel's bounded wait ran out."""
    check(lib().wxpy_vecops_status(), "wxpy_vecops_status")


def wxpy_debug_vecops_drop_tile(tile: int) -> None:
    check(lib().wxpy_debug_vecops_drop_tile(tile), "wxpy_debug_vecops_drop_tile")


def _host_vec(t, name: str):
    """(n, host pointer) of a contiguous 1-D float64 CPU tensor or numpy array."""
    import numpy as np
    if isinstance(t, np.ndarray):
        if t.dtype != np.float64 or t.ndim != 1 or not t.flags.c_contiguous:
            raise ValueError(f"{name} must be a contiguous 1-D float64 array")
        return t.shape[0], t.ctypes.data
    if t.dtype.__str__() != "torch.float64" or t.is_cuda or t.dim() != 1 or (
            t.numel() > 1 and t.stride(0) != 1):
        raise ValueError(f"{name} must be a contiguous 1-D float64 CPU tensor")
    return t.numel(), t.data_ptr()


def wxpy_host(alpha: float, x, y, w, stream=None):
    """w = alpha*x + y on host vectors (pinned for overlap), asynchronous on ``stream``."""
    n, px = _host_vec(x, "x")
    ny, py = _host_vec(y, "y")
    nw, pw = _host_vec(w, "w")
    if not (n == ny == nw):
        raise ValueError(f"length mismatch: x {n}, y {ny}, w {nw}")
    check(lib().wxpy_host(n, float(alpha), px, py, pw, _stream_handle(stream)), "wxpy_host")
    return w


def wxpy_host_config(chunk_elems: int = 1 << 22, slots: int = 3, direct: bool = False) -> None:
    check(lib().wxpy_host_config(chunk_elems, slots, int(direct)), "wxpy_host_config")


def wxpy_run_variant(vid: int, alpha: float, x, y, w=None, stream=None):
    n, a, px, py, pw, w = _prepare(alpha, x, y, w)
    check(lib().wxpy_run_variant(vid, n, a, px, py, pw, _stream_handle(stream)),
          "wxpy_run_variant")
    return w


def wxpy_reference(alpha: float, x, y, w=None, stream=None):
    n, a, px, py, pw, w = _prepare(alpha, x, y, w)
    check(lib().wxpy_reference(n, a, px, py, pw, _stream_handle(stream)), "wxpy_reference")
    return w


def wxpy_fill_uniform(dst, seed: int, tag: int, lo: float = -1.0, hi: float = 1.0,
                      start: int = 0, stream=None):
    """Fill the float64 CUDA tensor ``dst`` from stream (seed, tag) starting at ``start``."""
    n, p = _vec(dst, "dst")
    check(lib().wxpy_fill_uniform(n, seed & ((1 << 64) - 1), tag, start, lo, hi, p,
                                  _stream_handle(stream)), "wxpy_fill_uniform")
    return dst


def wxpy_launch_pdl(enable: int = -1) -> int:
    """Programmatic dependent launch of the single-call kernels: 1 on, 0 off,
    -1 unchanged; returns the setting before the call."""
    prev = _INT()
    check(lib().wxpy_launch_pdl(int(enable), ctypes.byref(prev)), "wxpy_launch_pdl")
    return prev.value


def wxpy_debug_inject_launch_error(cuda_error: int, count: int) -> None:
    check(lib().wxpy_debug_inject_launch_error(cuda_error, count),
          "wxpy_debug_inject_launch_error")


def wxpy_tune(n: int, flags: int = 0) -> dict:
    """Run the empirical search for the cell of n (and the class in ``flags``)."""
    r = TuneResult()
    check(lib().wxpy_tune(n, flags, ctypes.byref(r)), "wxpy_tune")
    return r.as_dict()


def tune(n: int, flags: int = 0) -> dict:
    """The Sec. 2 search for the size bucket of n (see wxpy_tune)."""
    return wxpy_tune(n, flags)


def wxpy_tune_get(tune_key: int) -> int:
    v = _INT()
    check(lib().wxpy_tune_get(tune_key, ctypes.byref(v)), "wxpy_tune_get")
    return v.value


def wxpy_tune_set(tune_key: int, variant_id: int) -> None:
    check(lib().wxpy_tune_set(tune_key, variant_id), "wxpy_tune_set")


def wxpy_tune_clear() -> None:
    check(lib().wxpy_tune_clear(), "wxpy_tune_clear")


def wxpy_tune_cache_save(path: str) -> None:
    check(lib().wxpy_tune_cache_save(os.fsencode(path)), "wxpy_tune_cache_save")


def wxpy_tune_cache_load(path: str, check_device: bool = True) -> None:
    check(lib().wxpy_tune_cache_load(os.fsencode(path), int(check_device)),
          "wxpy_tune_cache_load")


# ---------------------------------------------------------------- batched launch
# numpy layout of wxpy_desc (40 bytes): n, alpha, x, y, w
DESC_DTYPE = [("n", "<i8"), ("alpha", "<f8"), ("x", "<u8"), ("y", "<u8"), ("w", "<u8")]


class BatchInfo(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("elements", ctypes.c_int64), ("bytes", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("threads", ctypes.c_int32)]


class BatchTuneResult(ctypes.Structure):
    _fields_ = [("tile_elems", ctypes.c_int32 * 64), ("unroll", ctypes.c_int32 * 64),
                ("us", ctypes.c_double * 64), ("gbs", ctypes.c_double * 64),
                ("mixed_us", ctypes.c_double), ("mixed_gbs", ctypes.c_double),
                ("blocks_per_sm", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("rejected", ctypes.c_int32),
                ("fp64_offload", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def desc_table(ns, alphas, xptrs, yptrs, wptrs):
    """Host descriptor table (numpy structured array with the wxpy_desc layout)."""
    import numpy as np
    t = np.zeros(len(ns), dtype=DESC_DTYPE)
    t["n"], t["alpha"], t["x"], t["y"], t["w"] = ns, alphas, xptrs, yptrs, wptrs
    assert t.itemsize == 40
    return t


def table_to_device(table, device="cuda"):
    """A device copy of a host descriptor table (torch uint8 tensor)."""
    import numpy as np
    import torch
    raw = np.ascontiguousarray(table).view(np.uint8)
    return torch.from_numpy(raw.copy()).to(device)


def _tptr(table) -> int:
    return table.ctypes.data if len(table) else 0


class BatchPlan:
    """Owns a wxpy_batch_plan (freed on close/del)."""

    def __init__(self, host_table):
        self.table = host_table
        h = _P()
        check(lib().wxpy_batch_plan_create(_tptr(host_table), len(host_table), ctypes.byref(h)),
              "wxpy_batch_plan_create")
        self.handle = h.value

    def launch(self, dev_table, stream=None):
        check(lib().wxpy_batch_launch(self.handle, dev_table.data_ptr(), _stream_handle(stream)),
              "wxpy_batch_launch")

    def graph_launch(self, dev_table, stream=None):
        check(lib().wxpy_batch_graph_launch(self.handle, dev_table.data_ptr(),
                                            _stream_handle(stream)), "wxpy_batch_graph_launch")

    def info(self) -> dict:
        i = BatchInfo()
        check(lib().wxpy_batch_plan_info(self.handle, ctypes.byref(i)), "wxpy_batch_plan_info")
        return {f: getattr(i, f) for f, _ in i._fields_}

    def status(self, clear: bool = False) -> int:
        s = ctypes.c_uint()
        check(lib().wxpy_batch_status(self.handle, ctypes.byref(s), int(clear)), "wxpy_batch_status")
        return s.value

    def close(self):
        if getattr(self, "handle", None):
            lib().wxpy_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wxpy_batch_plan_create(host_table) -> BatchPlan:
    return BatchPlan(host_table)


def wxpy_batch(host_table, dev_table, stream=None) -> None:
    check(lib().wxpy_batch(_tptr(host_table), dev_table.data_ptr() if len(host_table) else 0,
                           len(host_table), _stream_handle(stream)), "wxpy_batch")


def wxpy_batch_noalloc(dev_table, count: int, stream=None) -> None:
    """The batched launch without any allocation (fixed library scratch; see wxpy.h)."""
    check(lib().wxpy_batch_noalloc(dev_table.data_ptr() if count else 0, count,
                                   _stream_handle(stream)), "wxpy_batch_noalloc")


def wxpy_batch_tune(bucket_min: int, bucket_max: int, flags: int = 0) -> dict:
    r = BatchTuneResult()
    check(lib().wxpy_batch_tune(bucket_min, bucket_max, flags, ctypes.byref(r)), "wxpy_batch_tune")
    per = [{"bucket": b, "tile_elems": r.tile_elems[b], "unroll": r.unroll[b], "us": r.us[b],
            "gbs": r.gbs[b]} for b in range(bucket_min, bucket_max + 1)]
    return {"buckets": per, "mixed_us": r.mixed_us, "mixed_gbs": r.mixed_gbs,
            "blocks_per_sm": r.blocks_per_sm, "threads": r.threads,
            "fp64_offload": r.fp64_offload, "candidates": r.candidates, "rejected": r.rejected}


def wxpy_batch_shape_get(bucket: int) -> tuple[int, int]:
    t, u = _INT(), _INT()
    check(lib().wxpy_batch_shape_get(bucket, ctypes.byref(t), ctypes.byref(u)),
          "wxpy_batch_shape_get")
    return t.value, u.value


def wxpy_batch_shape_set(bucket: int, tile_elems: int, unroll: int) -> None:
    check(lib().wxpy_batch_shape_set(bucket, tile_elems, unroll), "wxpy_batch_shape_set")


def wxpy_batch_shape_reset() -> None:
    check(lib().wxpy_batch_shape_reset(), "wxpy_batch_shape_reset")


def wxpy_batch_launch_get() -> tuple[int, int]:
    b, o = _INT(), _INT()
    check(lib().wxpy_batch_launch_get(ctypes.byref(b), ctypes.byref(o)), "wxpy_batch_launch_get")
    return b.value, o.value


def wxpy_batch_launch_set(blocks_per_sm: int, fp64_offload: int) -> None:
    check(lib().wxpy_batch_launch_set(blocks_per_sm, fp64_offload), "wxpy_batch_launch_set")
