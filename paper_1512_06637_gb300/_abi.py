"""ctypes binding of ``include/gv.h`` (argument marshalling only).

Every query runs in the CUDA library ``libgvgeo.so``; there is no Python or CPU
fallback.  If the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# GV_DEBUG=1 selects the build with device-side checks (build.py, gv_debug_status)
DEBUG = os.environ.get("GV_DEBUG", "0") not in ("", "0")
LIB_PATH = os.path.join(PKG, "libgvgeo_debug.so" if DEBUG else "libgvgeo.so")

GV_OK, GV_ERR_INVALID_ARG, GV_ERR_UNSUPPORTED, GV_ERR_OUT_OF_MEMORY = 0, 1, 2, 3
GV_ERR_CUDA, GV_ERR_TIMEOUT, GV_ERR_BUSY = 4, 5, 6
GV_FP64, GV_FP32_REFINE = 0, 1
GV_INSIDE, GV_SURFACE, GV_OUTSIDE = 0, 1, 2
GV_MAX_ZPLANES = 32

_p = ctypes.c_void_p
_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64


class Basket(ctypes.Structure):
    _fields_ = [("offset", _i64), ("n", _i64), ("solid", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("items", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", _i64), ("max_slots", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", _i64), ("tracks", _i64), ("launches", _i64), ("queued", _i64),
                ("p50_ms", _d), ("p99_ms", _d), ("mean_ms", _d), ("max_ms", _d)]


class Tracks(ctypes.Structure):
    _fields_ = [("x", _p), ("y", _p), ("z", _p), ("dx", _p), ("dy", _p), ("dz", _p), ("n", _i64)]


class Results(ctypes.Structure):
    _fields_ = [("inside", _p), ("dist_in", _p), ("dist_out", _p), ("safety_in", _p),
                ("safety_out", _p)]


# symbol -> (restype, argtypes); the CPU test checks that every declaration of
# include/gv.h appears here and is exported by the library.
class TransportOut(ctypes.Structure):
    _fields_ = [("reason", ctypes.c_void_p), ("steps", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("path", ctypes.c_void_p),
                ("last", ctypes.c_void_p), ("tie", ctypes.c_void_p)]


SIGNATURES = {
    "gv_solid_box": (_i, [_d, _d, _d, _p]),
    "gv_solid_trd": (_i, [_d, _d, _d, _d, _d, _p]),
    "gv_solid_trap": (_i, [_p, _p]),
    "gv_solid_tube": (_i, [_d, _d, _d, _d, _d, _p]),
    "gv_solid_cone": (_i, [_d, _d, _d, _d, _d, _d, _d, _p]),
    "gv_solid_polycone": (_i, [_i, _p, _p, _p, _d, _d, _p]),
    "gv_solid_boolean": (_i, [ctypes.c_int32, _p, _p, _p, _p, _p]),
    "gv_solid_destroy": (None, [_p]),
    "gv_workspace_create": (_i, [_i64, _p]),
    "gv_workspace_destroy": (None, [_p]),
    "gv_workspace_refined": (_i, [_p, _p, _p]),
    "gv_query": (_i, [_p, ctypes.POINTER(Tracks), _i, ctypes.POINTER(Results), _p, _p]),
    "gv_pipeline_create": (_i, [_i64, ctypes.c_int32, _p]),
    "gv_pipeline_destroy": (None, [_p]),
    "gv_pipeline_join": (_i, [_p, _p]),
    "gv_query_host": (_i, [_p, ctypes.POINTER(Tracks), _i, ctypes.POINTER(Results), _p, _p]),
    "gv_batch_create": (_i, [_p, ctypes.c_int32, _p, ctypes.c_int32, _p]),
    "gv_batch_set_config": (_i, [_p, ctypes.POINTER(BatchConfig)]),
    "gv_batch_get_config": (_i, [_p, ctypes.POINTER(BatchConfig)]),
    "gv_batch_run": (_i, [_p, ctypes.POINTER(Tracks), _i, ctypes.POINTER(Results), _p]),
    "gv_batch_autotune": (_i, [_p, ctypes.POINTER(Tracks), _i, ctypes.POINTER(Results), _p,
                               ctypes.POINTER(BatchConfig)]),
    "gv_batch_refined": (_i, [_p, _p, _p]),
    "gv_batch_destroy": (None, [_p]),
    "gv_geom_create": (_i, [ctypes.c_int32, _p, _p, _p, _p, _p]),
    "gv_geom_destroy": (None, [_p]),
    "gv_geom_node_count": (ctypes.c_int32, [_p]),
    "gv_geom_set_voxels": (_i, [_p, ctypes.c_int32]),
    "gv_geom_voxel_count": (ctypes.c_int32, [_p]),
    "gv_nav_locate": (_i, [_p, ctypes.POINTER(Tracks), _p, _p]),
    "gv_nav_step": (_i, [_p, ctypes.POINTER(Tracks), _p, _i, _p, _p, _p, _p, _p]),
    "gv_transport": (_i, [_p, ctypes.POINTER(Tracks), _p, _p, _p, ctypes.c_int32, _p, ctypes.c_int32,
                          ctypes.c_int, ctypes.POINTER(TransportOut), _p]),
    "gv_server_create": (_i, [_p, ctypes.POINTER(ServerConfig), _p]),
    "gv_server_submit": (_i, [_p, _i64, _p, _p, _p]),
    "gv_server_poll": (_i, [_p, _i64, _p]),
    "gv_server_wait": (_i, [_p, _i64, _d, _p]),
    "gv_server_get_stats": (_i, [_p, ctypes.POINTER(ServerStats)]),
    "gv_server_reset_stats": (_i, [_p]),
    "gv_server_destroy": (None, [_p]),
    "gv_query_fp32_static": (_i, [_p, ctypes.POINTER(Tracks), ctypes.POINTER(Results), _p]),
    "gv_debug_status": (_i, [_p, _p, _i]),
    "gv_last_error": (ctypes.c_char_p, []),
    "gv_version": (ctypes.c_char_p, []),
}


class GVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gv status {status}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1512_06637_gb300.build.build() "
                          "(nvcc, sm_103a); there is no fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def check(status: int):
    if status != GV_OK:
        raise GVError(status, lib().gv_last_error().decode())
