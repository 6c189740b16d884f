"""Python front end of the continuous-batching server (``pa_server_*``).

The scheduler, admission control, plan cache and all CUDA work live in the
native library; this module only marshals arguments.
"""

from __future__ import annotations

import ctypes

from ._native import PA_OK, PA_STAGE_LOG, PlanDesc, check, load


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("device_budget_bytes", ctypes.c_size_t),
        ("slots", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("max_plans", ctypes.c_int32),
        ("stages", ctypes.c_uint32),
    ]


class RequestResult(ctypes.Structure):
    _fields_ = [
        ("ticket", ctypes.c_uint64),
        ("status", ctypes.c_int),
        ("arrival_s", ctypes.c_double),
        ("start_s", ctypes.c_double),
        ("done_s", ctypes.c_double),
        ("latency_ms", ctypes.c_double),
        ("batch_frames", ctypes.c_int32),
        ("device_ms", ctypes.c_float),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("failed", ctypes.c_uint64),
        ("batches", ctypes.c_uint64),
        ("bytes_in_use", ctypes.c_size_t),
        ("bytes_peak", ctypes.c_size_t),
        ("plans_resident", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def _bind(L):
    if getattr(L, "_pa_server_bound", False):
        return
    vp = ctypes.c_void_p
    L.pa_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.pa_server_create.restype = ctypes.c_int
    L.pa_server_now.argtypes = [vp]
    L.pa_server_now.restype = ctypes.c_double
    L.pa_server_submit.argtypes = [vp, ctypes.POINTER(PlanDesc), vp, vp, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_uint64)]
    L.pa_server_submit.restype = ctypes.c_int
    L.pa_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(RequestResult)]
    L.pa_server_wait.restype = ctypes.c_int
    L.pa_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.pa_server_get_stats.restype = ctypes.c_int
    L.pa_server_destroy.argtypes = [vp]
    L.pa_server_destroy.restype = ctypes.c_int
    L._pa_server_bound = True


class Server:
    """Requests in, images out; batching and admission happen natively."""

    def __init__(self, budget_bytes: int, slots: int = 4, max_batch: int = 8,
                 max_plans: int = 512, stages: int = PA_STAGE_LOG, checked: bool = False):
        self._L = load(checked)
        _bind(self._L)
        self.cfg = ServerConfig(int(budget_bytes), int(slots), int(max_batch), int(max_plans),
                                int(stages))
        h = ctypes.c_void_p()
        check(self._L, self._L.pa_server_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self._h = h

    def now(self) -> float:
        return float(self._L.pa_server_now(self._h))

    def submit(self, desc: PlanDesc, rf_host_ptr: int, out_host_ptr: int,
               arrival_s: float = 0.0) -> int:
        t = ctypes.c_uint64()
        check(self._L, self._L.pa_server_submit(self._h, ctypes.byref(desc), rf_host_ptr,
                                                out_host_ptr, float(arrival_s), ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        r = RequestResult()
        check(self._L, self._L.pa_server_wait(self._h, int(ticket), int(timeout_ms),
                                              ctypes.byref(r)))
        return r.as_dict()

    def try_wait(self, ticket: int, timeout_ms: int):
        """Like wait(), but returns the status code instead of raising."""
        r = RequestResult()
        st = self._L.pa_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(r))
        return st, (r.as_dict() if st == PA_OK else None)

    def stats(self) -> dict:
        s = ServerStats()
        check(self._L, self._L.pa_server_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.pa_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def percentiles(values, qs=(50, 99)):
    import numpy as np

    v = np.asarray(values, dtype=float)
    return {f"p{q}": float(np.percentile(v, q)) for q in qs} if v.size else {}
