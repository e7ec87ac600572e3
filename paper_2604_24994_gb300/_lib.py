"""ctypes binding of libpowerfoam.so (argument marshalling only).

Every step of rendering runs in the library's CUDA kernels; this module
only converts Python/torch objects into the C structs of include/powerfoam.h.
It raises if the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpowerfoam.so")

PF_OK, PF_ERR_INVALID_ARG, PF_ERR_CAPACITY, PF_ERR_CUDA, PF_ERR_TIMEOUT, PF_ERR_BUSY, PF_ERR_NOT_FOUND = range(7)

_lock = threading.Lock()
_lib = None


class PFError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({detail})")


class Scene(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex", "nbr")] + [
        ("n_cells", C.c_int32), ("k_nbr", C.c_int32), ("disp", C.c_void_p), ("sites", C.c_void_p),
        ("sv", C.c_void_p), ("n_sites", C.c_int32)]


class Camera(C.Structure):
    _fields_ = [("rot", C.c_double * 9), ("origin", C.c_double * 3), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int32), ("height", C.c_int32),
                ("model", C.c_int32)]


class SceneGrad(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex", "disp", "sites",
                                          "sv")]


class Stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("instances", "candidates", "hits", "planes", "refined", "sphere_pass",
                                                     "warp_candidates", "warp_passes", "warp_hits", "wait_errors")]


def _sig(lib):
    P, V, U64, I32 = C.POINTER, C.c_void_p, C.c_uint64, C.c_int32
    st = C.c_int
    spec = {
        "pf_status_string": ([st], C.c_char_p),
        "pf_last_error_message": ([], C.c_char_p),
        "pf_plan_create": ([I32, I32, P(Camera), I32, U64, P(V)], st),
        "pf_plan_destroy": ([V], None),
        "pf_plan_workspace_bytes": ([V, P(U64)], st),
        "pf_plan_pixels": ([V, P(U64)], st),
        "pf_plan_set_cameras": ([V, P(Camera), I32], st),
        "pf_plan_enable_stats": ([V, I32], st),
        "pf_plan_set_record_hits": ([V, I32], st),
        "pf_plan_omit_hit_records": ([V], st),
        "pf_plan_store_segments": ([V, I32], st),
        "pf_read_hit_counts": ([V, V, V, V], st),
        "pf_plan_read_stats": ([V, V, P(Stats), V], st),
        "pf_prepare": ([P(Scene), V, V, V], st),
        "pf_project": ([P(Scene), V, V, V], st),
        "pf_bin_sort": ([V, V, P(U64), V], st),
        "pf_render_fwd": ([P(Scene), V, V, V, V, V, V], st),
        "pf_render_fwd_contrib": ([P(Scene), V, V, V, V, V, V, V, V], st),
        "pf_connect": ([P(Scene), V, V, V, V], st),
        "pf_render_bwd": ([P(Scene), V, V, V, V, V, V, P(SceneGrad), V], st),
        "pf_render_bwd_contrib": ([P(Scene), V, V, V, V, V, V, V, V, P(SceneGrad), V], st),
        "pf_read_bins": ([V, V, V, V, V, V, V], st),
        "pf_neighbours_workspace_bytes": ([I32], U64),
        "pf_build_neighbours": ([V, V, V, I32, I32, V, V, V, V, V, U64, V], st),
        "pf_connect_cech_workspace_bytes": ([I32], U64),
        "pf_connect_cech": ([V, V, I32, V, V, V, V, V, U64, V], st),
    }
    for name, (args, res) in spec.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library missing ({LIB_PATH}); build it with "
                                   "paper_2604_24994_gb300.build.build()")
            l = C.CDLL(LIB_PATH)
            _sig(l)
            _lib = l
        return _lib


def check(status: int, where: str):
    if status != PF_OK:
        detail = lib().pf_last_error_message().decode(errors="replace")
        name = lib().pf_status_string(status).decode()
        raise PFError(status, where, f"{name}: {detail}")


def camera_struct(cam) -> Camera:
    c = Camera()
    c.rot[:] = [float(x) for x in np.asarray(cam.rot, np.float64).reshape(9)]
    c.origin[:] = [float(x) for x in np.asarray(cam.origin, np.float64).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.model = int(getattr(cam, "model", 0))
    return c


def camera_array(cams):
    arr = (Camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


def ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def stream_ptr(stream) -> int | None:
    return None if stream is None else stream.cuda_stream
