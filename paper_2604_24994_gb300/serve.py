"""Python binding of the serving entry points (pf_serve_*): argument
marshalling only; the queue, batching, graphs and kernels run in the
library."""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import check, lib


class ServeOpts(C.Structure):
    _fields_ = [("max_batch_views", C.c_int32), ("slots", C.c_int32), ("use_graphs", C.c_int32),
                ("max_queue", C.c_int32)]


class ServeReport(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("submitted", "completed", "rejected", "batches", "graph_replays",
                                           "requeued")] + \
               [(k, C.c_double) for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "elapsed_s", "requests_per_s",
                                          "mpix_per_s", "mean_batch_views")] + [("graph_updates", C.c_uint64)]


def _sig():
    l = lib()
    if getattr(l, "_serve_sig", False):
        return l
    P, V = C.POINTER, C.c_void_p
    l.pf_serve_create.argtypes = [P(_lib.Scene), V, C.c_uint64, P(ServeOpts), P(V)]
    l.pf_serve_create.restype = C.c_int
    l.pf_serve_submit.argtypes = [V, P(_lib.Camera), V, V, P(C.c_uint64)]
    l.pf_serve_submit.restype = C.c_int
    l.pf_serve_poll.argtypes = [V, C.c_uint64, C.c_int32, P(C.c_int32)]
    l.pf_serve_poll.restype = C.c_int
    l.pf_serve_stats.argtypes = [V, P(ServeReport)]
    l.pf_serve_stats.restype = C.c_int
    l.pf_serve_reset_stats.argtypes = [V]
    l.pf_serve_reset_stats.restype = C.c_int
    l.pf_serve_destroy.argtypes = [V]
    l.pf_serve_destroy.restype = None
    l._serve_sig = True
    return l


class Server:
    """A render server over a resident DeviceScene with a device pool of
    `budget_bytes` (allocated here with torch and handed to the library)."""

    def __init__(self, scene, budget_bytes: int, max_batch_views: int = 8, slots: int = 2,
                 use_graphs: bool = True, max_queue: int = 4096, device="cuda"):
        l = _sig()
        self.scene = scene
        self.pool = torch.empty(int(budget_bytes), dtype=torch.uint8, device=device)
        self._s = scene.struct()
        o = ServeOpts(int(max_batch_views), int(slots), 1 if use_graphs else 0, int(max_queue))
        self.h = C.c_void_p()
        check(l.pf_serve_create(C.byref(self._s), self.pool.data_ptr(), int(budget_bytes), C.byref(o),
                                C.byref(self.h)), "pf_serve_create")

    def submit(self, cam, rgb: torch.Tensor, T: torch.Tensor) -> int:
        """Queue a view; rgb [H*W,3] and T [H*W] device float32 outputs.
        Returns the request id; raises PFError (status PF_ERR_BUSY when the
        queue is full)."""
        rid = C.c_uint64()
        check(lib().pf_serve_submit(self.h, C.byref(_lib.camera_struct(cam)), rgb.data_ptr(), T.data_ptr(),
                                    C.byref(rid)), "pf_serve_submit")
        return int(rid.value)

    def try_submit(self, cam, rgb, T):
        rid = C.c_uint64()
        st = lib().pf_serve_submit(self.h, C.byref(_lib.camera_struct(cam)), rgb.data_ptr(), T.data_ptr(),
                                   C.byref(rid))
        return st, int(rid.value)

    def poll(self, rid: int, timeout_ms: int = 0) -> int:
        """1 when the outputs are written, 0 if not yet; raises on failure."""
        d = C.c_int32()
        st = lib().pf_serve_poll(self.h, rid, int(timeout_ms), C.byref(d))
        if st == _lib.PF_ERR_TIMEOUT:
            return 0
        check(st, "pf_serve_poll")
        return int(d.value)

    def wait(self, rid: int, timeout_ms: int = 60000) -> None:
        if not self.poll(rid, timeout_ms):
            raise TimeoutError(f"request {rid} not done after {timeout_ms} ms")

    def report(self) -> dict:
        r = ServeReport()
        check(lib().pf_serve_stats(self.h, C.byref(r)), "pf_serve_stats")
        return {f: getattr(r, f) for f, _ in ServeReport._fields_}

    def reset_stats(self):
        check(lib().pf_serve_reset_stats(self.h), "pf_serve_reset_stats")

    def close(self):
        if self.h:
            lib().pf_serve_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
