"""GB300 track-versus-solid geometry queries (arXiv:1512.06637, VecGeom section).

Python face of the C ABI in ``include/gv.h``: solids, workspaces and the query
call, with PyTorch tensors as device memory and streams.  All work runs in the
CUDA library ``libgvgeo.so`` built for sm_103a; nothing here computes a result.
"""
from __future__ import annotations

import ctypes

from . import _abi
from ._abi import (GV_FP32_REFINE, GV_FP64, GV_INSIDE, GV_OUTSIDE, GV_SURFACE, GVError,  # noqa: F401
                   check, lib)

PRECISIONS = {"fp64": GV_FP64, "fp32_refine": GV_FP32_REFINE}
HAS_FP32_REFINE = True
QUERIES = ("inside", "dist_in", "dist_out", "safety_in", "safety_out")


def _f(v):
    return ctypes.c_double(float(v))


class Solid:
    """A solid handle owned by the library (immutable once created)."""

    def __init__(self, kind: str, *params):
        L = lib()
        h = ctypes.c_void_p()
        if kind == "box":
            st = L.gv_solid_box(*map(_f, params), ctypes.byref(h))
        elif kind == "trd":
            st = L.gv_solid_trd(*map(_f, params), ctypes.byref(h))
        elif kind == "trap":
            p = params[0] if len(params) == 1 else params
            arr = (ctypes.c_double * 11)(*map(float, p))
            st = L.gv_solid_trap(arr, ctypes.byref(h))
        elif kind == "tube":
            st = L.gv_solid_tube(*map(_f, params), ctypes.byref(h))
        elif kind == "cone":
            st = L.gv_solid_cone(*map(_f, params), ctypes.byref(h))
        elif kind == "polycone":
            z, rmin, rmax, sphi, dphi = params
            n = len(z)
            arr = lambda v: (ctypes.c_double * n)(*map(float, v))  # noqa: E731
            st = L.gv_solid_polycone(n, arr(z), arr(rmin), arr(rmax), _f(sphi), _f(dphi), ctypes.byref(h))
        else:
            raise ValueError(f"unknown solid kind {kind!r}")
        check(st)
        self.kind = kind
        self.params = params
        self.handle = h

    @classmethod
    def from_spec(cls, spec: dict) -> "Solid":
        return cls(spec["kind"], *spec["params"])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gv_solid_destroy(h)
            self.handle = None


class Workspace:
    """Device scratch (refinement worklist) for baskets of up to ``max_tracks`` tracks."""

    def __init__(self, max_tracks: int):
        h = ctypes.c_void_p()
        check(lib().gv_workspace_create(int(max_tracks), ctypes.byref(h)))
        self.handle = h
        self.max_tracks = int(max_tracks)

    def refined(self, stream=None) -> int:
        n = ctypes.c_int64()
        check(lib().gv_workspace_refined(self.handle, _stream_ptr(stream), ctypes.byref(n)))
        return n.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gv_workspace_destroy(h)
            self.handle = None


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_tensor(t, dtype, n, name):
    import torch
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor of {n} elements")


def tracks_struct(tr: dict) -> _abi.Tracks:
    import torch
    n = tr["x"].numel()
    for k in ("x", "y", "z", "dx", "dy", "dz"):
        if tr.get(k) is not None:
            _check_tensor(tr[k], torch.float64, n, k)
    return _abi.Tracks(*(_ptr(tr.get(k)) for k in ("x", "y", "z", "dx", "dy", "dz")), n)


def alloc_results(n: int, device, want=QUERIES) -> dict:
    import torch
    out = {}
    for k in want:
        out[k] = torch.empty(n, dtype=torch.int8 if k == "inside" else torch.float64, device=device)
    return out


def results_struct(out: dict, n: int) -> _abi.Results:
    import torch
    for k, v in out.items():
        _check_tensor(v, torch.int8 if k == "inside" else torch.float64, n, k)
    return _abi.Results(*(_ptr(out.get(k)) for k in QUERIES))


def query(solid: Solid, tracks: dict, precision: str = "fp64", out: dict | None = None,
          workspace: Workspace | None = None, stream=None, want=QUERIES) -> dict:
    """Enqueue all requested queries for one basket (dict of CUDA float64 tensors
    x, y, z, dx, dy, dz) against one solid; returns the result tensors."""
    n = tracks["x"].numel()
    if out is None:
        out = alloc_results(n, tracks["x"].device, want)
    t = tracks_struct(tracks)
    r = results_struct(out, n)
    ws = workspace.handle if workspace is not None else None
    check(lib().gv_query(solid.handle, ctypes.byref(t), PRECISIONS[precision], ctypes.byref(r), ws,
                         _stream_ptr(stream)))
    return out


def version() -> str:
    return lib().gv_version().decode()
