"""ctypes binding of the continuous-batching server (``wxpy_server_*`` in wxpy.h).

Argument marshalling only: admission, batching, launches and completion
tracking run in the library's scheduler thread and CUDA kernels.
"""
from __future__ import annotations

import ctypes

from .binding import _D, _I64, _P, check, lib

SERVE_BATCHED, SERVE_SERIAL, SERVE_FUSED = 0, 1, 2
DATA_DEVICE, DATA_HOST = 0, 1
REQ_QUEUED, REQ_ADMITTED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3, 4


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("admission", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "submitted", "rejected", "completed", "failed", "queued_now", "resident_now",
        "max_queue", "batches", "launches", "elements_done", "arena_used", "max_inflight")] + \
        [(f, ctypes.c_double) for f in ("mean_batch", "window_s", "p50_s", "p99_s", "mean_s",
                                        "max_s", "head_wait_frag_s", "head_wait_full_s")] + \
        [("backfilled", ctypes.c_int64), ("reserved", ctypes.c_int64),
         ("max_launch_host_s", ctypes.c_double), ("max_batch_s", ctypes.c_double)]


class LoadgenConfig(ctypes.Structure):
    _fields_ = [("rate", ctypes.c_double), ("duration_s", ctypes.c_double),
                ("n_min", ctypes.c_int64), ("n_max", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("drain_timeout_s", ctypes.c_double)]


class LoadgenResult(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "offered", "submitted", "rejected", "completed", "failed", "max_queue",
        "backlog_at_end", "launches")] + \
        [(f, ctypes.c_double) for f in ("p50_s", "p99_s", "mean_s", "max_s", "wall_s",
                                        "arrivals_s", "elem_per_s", "gbs", "mean_batch")] + \
        [("drained", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _as_dict(s) -> dict:
    return {f: getattr(s, f) for f, _ in s._fields_ if f != "reserved"}


class Server:
    """A running wxpy server (wxpy_server_create ... wxpy_server_destroy)."""

    def __init__(self, budget_bytes: int = 16 << 30, max_slots: int = 4096, n_streams: int = 2,
                 max_batch: int = 1024, max_queue: int = 65536, mode: int = SERVE_BATCHED,
                 admission_us: int = 0):
        """admission_us: 0 strict arrival order; > 0 backfill with that aging bound (us)."""
        cfg = ServerConfig(budget_bytes, max_slots, n_streams, max_batch, max_queue, mode,
                           admission_us)
        h = _P()
        check(lib().wxpy_server_create(ctypes.byref(cfg), ctypes.byref(h)), "wxpy_server_create")
        self.handle = h.value

    def submit(self, n: int, alpha: float, seed: int) -> int:
        t = ctypes.c_uint64()
        check(lib().wxpy_server_submit(self.handle, n, float(alpha), seed & ((1 << 64) - 1),
                                       ctypes.byref(t)), "wxpy_server_submit")
        return t.value

    def submit_data(self, alpha: float, x, y) -> int:
        """Queue a request on the caller's data: float64 1-D contiguous tensors
        x and y (same length), both on the GPU or both in host memory.  They
        must stay alive and unchanged until the request is done or failed."""
        if x.dtype != y.dtype or str(x.dtype) != "torch.float64":
            raise TypeError("x and y must be float64 tensors")
        if x.dim() != 1 or y.dim() != 1 or not x.is_contiguous() or not y.is_contiguous():
            raise ValueError("x and y must be contiguous 1-D tensors")
        if x.numel() != y.numel():
            raise ValueError("x and y must have the same length")
        if x.is_cuda != y.is_cuda:
            raise ValueError("x and y must both be device or both be host tensors")
        kind = DATA_DEVICE if x.is_cuda else DATA_HOST
        t = ctypes.c_uint64()
        check(lib().wxpy_server_submit_data(self.handle, x.numel(), float(alpha), x.data_ptr(),
                                            y.data_ptr(), kind, ctypes.byref(t)),
              "wxpy_server_submit_data")
        return t.value

    def poll(self, ticket: int) -> tuple[int, float]:
        st, lat = ctypes.c_int(), _D()
        check(lib().wxpy_server_poll(self.handle, ticket, ctypes.byref(st), ctypes.byref(lat)),
              "wxpy_server_poll")
        return st.value, lat.value

    def wait(self, ticket: int, timeout_s: float = 30.0) -> float:
        lat = _D()
        check(lib().wxpy_server_wait(self.handle, ticket, timeout_s, ctypes.byref(lat)),
              "wxpy_server_wait")
        return lat.value

    def result(self, ticket: int) -> tuple[int, int, int, int]:
        """(n, x, y, w) device pointers of a done request."""
        x, y, w, n = _P(), _P(), _P(), _I64()
        check(lib().wxpy_server_result(self.handle, ticket, ctypes.byref(x), ctypes.byref(y),
                                       ctypes.byref(w), ctypes.byref(n)), "wxpy_server_result")
        return n.value, x.value, y.value, w.value

    def release(self, ticket: int) -> None:
        check(lib().wxpy_server_release(self.handle, ticket), "wxpy_server_release")

    def stats(self, reset: bool = False) -> dict:
        s = ServerStats()
        check(lib().wxpy_server_get_stats(self.handle, int(reset), ctypes.byref(s)),
              "wxpy_server_get_stats")
        return _as_dict(s)

    def loadgen(self, rate: float, duration_s: float, n_min: int = 256, n_max: int = 1 << 24,
                seed: int = 20130907, drain_timeout_s: float = 120.0, check_drain=True) -> dict:
        cfg = LoadgenConfig(rate, duration_s, n_min, n_max, seed, drain_timeout_s)
        r = LoadgenResult()
        rc = lib().wxpy_server_loadgen(self.handle, ctypes.byref(cfg), ctypes.byref(r))
        if check_drain:
            check(rc, "wxpy_server_loadgen")
        d = _as_dict(r)
        d["status"] = rc
        return d

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().wxpy_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
