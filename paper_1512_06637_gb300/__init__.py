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


BOOL_OPS = {"union": 0, "subtraction": 1, "intersection": 2}


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
        elif kind == "boolean":
            # (op, component a spec, component c spec, R (3x3, c placed in a), t (3))
            op, sa, sc, R, t = params
            a, c = Solid.from_spec(sa), Solid.from_spec(sc)  # the boolean keeps its own copies
            Rv = (ctypes.c_double * 9)(*[float(v) for row in R for v in row])
            tv = (ctypes.c_double * 3)(*map(float, t))
            st = L.gv_solid_boolean(BOOL_OPS[op], a.handle, c.handle, Rv, tv, ctypes.byref(h))
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


class Pipeline:
    """Device staging slots and streams for baskets in host memory (gv_query_host)."""

    def __init__(self, chunk_tracks: int = 1 << 20, slots: int = 3):
        h = ctypes.c_void_p()
        check(lib().gv_pipeline_create(int(chunk_tracks), int(slots), ctypes.byref(h)))
        self.handle = h

    def join(self, stream=None):
        """``stream`` waits for every query_host call made on this pipeline so far."""
        check(lib().gv_pipeline_join(self.handle, _stream_ptr(stream)))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gv_pipeline_destroy(h)
            self.handle = None


def _host_ptr(a, dtype, n, name):
    """Address of a contiguous host array (numpy array or CPU torch tensor)."""
    import numpy as np
    if a is None:
        return None
    if hasattr(a, "is_cuda"):
        import torch
        want = torch.int8 if dtype == np.int8 else torch.float64
        if a.is_cuda or a.dtype != want or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"{name}: expected a contiguous host {want} tensor of {n} elements")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous or a.size != n:
        raise ValueError(f"{name}: expected a contiguous numpy {np.dtype(dtype)} array of {n} elements")
    return ctypes.c_void_p(a.ctypes.data)


def query_host(solid: Solid, tracks: dict, out: dict, pipeline: Pipeline, precision: str = "fp64",
               stream=None) -> dict:
    """gv_query for host arrays (numpy or CPU tensors, pinned for full speed): starts after
    the work on ``stream``; the results are in ``out`` once ``stream`` has passed a later
    ``pipeline.join(stream)``."""
    import numpy as np
    n = int(tracks["x"].size if isinstance(tracks["x"], np.ndarray) else tracks["x"].numel())
    t = _abi.Tracks(*(_host_ptr(tracks.get(k), np.float64, n, k) for k in ("x", "y", "z", "dx", "dy", "dz")), n)
    r = _abi.Results(*(_host_ptr(out.get(k), np.int8 if k == "inside" else np.float64, n, k) for k in QUERIES))
    check(lib().gv_query_host(solid.handle, ctypes.byref(t), PRECISIONS[precision], ctypes.byref(r),
                              pipeline.handle, _stream_ptr(stream)))
    return out


class Batch:
    """Many baskets, each against its own solid, over one shared track set (one
    persistent kernel replayed from a CUDA graph)."""

    def __init__(self, solids: list, offsets, sizes, solid_ids):
        n = len(offsets)
        arr = (_abi.Basket * max(n, 1))()
        for k in range(n):
            arr[k].offset, arr[k].n, arr[k].solid, arr[k].reserved = int(offsets[k]), int(sizes[k]), int(solid_ids[k]), 0
        handles = (ctypes.c_void_p * len(solids))(*[s.handle.value for s in solids])
        h = ctypes.c_void_p()
        check(lib().gv_batch_create(handles, len(solids), arr, n, ctypes.byref(h)))
        self.handle = h
        self.solids = solids  # keep the Python objects alive alongside

    def set_config(self, threads=256, items=2, ctas_per_sm=0):
        c = _abi.BatchConfig(threads, items, ctas_per_sm, 0)
        check(lib().gv_batch_set_config(self.handle, ctypes.byref(c)))

    def config(self) -> dict:
        c = _abi.BatchConfig()
        check(lib().gv_batch_get_config(self.handle, ctypes.byref(c)))
        return {"threads": c.threads, "items": c.items, "ctas_per_sm": c.ctas_per_sm}

    def run(self, tracks: dict, out: dict, precision: str = "fp32_refine", stream=None) -> dict:
        n = tracks["x"].numel()
        t = tracks_struct(tracks)
        r = results_struct(out, n)
        check(lib().gv_batch_run(self.handle, ctypes.byref(t), PRECISIONS[precision], ctypes.byref(r),
                                 _stream_ptr(stream)))
        return out

    def autotune(self, tracks: dict, out: dict, precision: str = "fp32_refine", stream=None) -> dict:
        n = tracks["x"].numel()
        t = tracks_struct(tracks)
        r = results_struct(out, n)
        c = _abi.BatchConfig()
        check(lib().gv_batch_autotune(self.handle, ctypes.byref(t), PRECISIONS[precision], ctypes.byref(r),
                                      _stream_ptr(stream), ctypes.byref(c)))
        return {"threads": c.threads, "items": c.items, "ctas_per_sm": c.ctas_per_sm}

    def refined(self, stream=None) -> int:
        n = ctypes.c_int64()
        check(lib().gv_batch_refined(self.handle, _stream_ptr(stream), ctypes.byref(n)))
        return n.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gv_batch_destroy(h)
            self.handle = None


class Geometry:
    """A tree of placed volumes (node 0 = world; parents precede children)."""

    def __init__(self, solids: list, nodes: list):
        import numpy as np
        self.solids = [s if isinstance(s, Solid) else Solid.from_spec(s) for s in solids]
        n = len(nodes)
        hs = (ctypes.c_void_p * n)(*[self.solids[nd["solid"]].handle.value for nd in nodes])
        par = np.ascontiguousarray([nd["parent"] for nd in nodes], dtype=np.int32)
        R = np.ascontiguousarray(np.array([np.asarray(nd["R"], float).reshape(9) for nd in nodes]))
        t = np.ascontiguousarray(np.array([np.asarray(nd["t"], float).reshape(3) for nd in nodes]))
        h = ctypes.c_void_p()
        check(lib().gv_geom_create(n, hs, par.ctypes.data_as(ctypes.c_void_p), R.ctypes.data_as(ctypes.c_void_p),
                                   t.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        self.handle = h
        self.nnodes = n

    @property
    def voxel_count(self) -> int:
        """Nodes that carry a voxel grid over their daughters."""
        return int(lib().gv_geom_voxel_count(self.handle))

    def set_voxels(self, enable: bool) -> None:
        """Use (True, the default) or bypass the daughters' voxel grids."""
        check(lib().gv_geom_set_voxels(self.handle, 1 if enable else 0))

    def locate(self, tracks: dict, out=None, stream=None):
        import torch
        n = tracks["x"].numel()
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=tracks["x"].device)
        t = tracks_struct(tracks)
        check(lib().gv_nav_locate(self.handle, ctypes.byref(t), _ptr(out), _stream_ptr(stream)))
        return out

    def step(self, tracks: dict, node, precision: str = "fp64", out: dict | None = None,
             workspace: Workspace | None = None, stream=None, safety: bool = True) -> dict:
        """One navigation step; ``safety=False`` leaves the safety out (no "safety" entry)."""
        import torch
        n = tracks["x"].numel()
        dev = tracks["x"].device
        if out is None:
            out = {"step": torch.empty(n, dtype=torch.float64, device=dev),
                   "next": torch.empty(n, dtype=torch.int32, device=dev)}
            if safety:
                out["safety"] = torch.empty(n, dtype=torch.float64, device=dev)
        t = tracks_struct(tracks)
        ws = workspace.handle if workspace is not None else None
        saf = _ptr(out["safety"]) if safety else None
        check(lib().gv_nav_step(self.handle, ctypes.byref(t), _ptr(node), PRECISIONS[precision], _ptr(out["step"]),
                                saf, _ptr(out["next"]), ws, _stream_ptr(stream)))
        return out

    def transport(self, tracks: dict, node0, node_material, sigma_n, xi, kmax: int, out: dict | None = None,
                  stream=None, precision: str = "fp64") -> dict:
        """The transport loop (gv_transport): CUDA tensors; ``node_material`` int32 per node,
        ``sigma_n`` float64 (nmat, 2), ``xi`` float64 (n, kmax, 4) in (0, 1].  ``precision``
        "fp32_refine" ranks candidates and codes in binary32 first (same results)."""
        import torch
        n = tracks["x"].numel()
        dev = tracks["x"].device
        if out is None:
            out = {"reason": torch.empty(n, dtype=torch.int8, device=dev),
                   "steps": torch.empty(n, dtype=torch.int32, device=dev),
                   "x": torch.empty(n, dtype=torch.float64, device=dev),
                   "y": torch.empty(n, dtype=torch.float64, device=dev),
                   "z": torch.empty(n, dtype=torch.float64, device=dev),
                   "path": torch.empty(n, dtype=torch.float64, device=dev),
                   "last": torch.empty(n, dtype=torch.int32, device=dev),
                   "tie": torch.empty(n, dtype=torch.int8, device=dev)}
        if xi.numel() != n * kmax * 4 or node_material.numel() != self.nnodes or sigma_n.numel() % 2:
            raise ValueError("transport: xi must hold n * kmax * 4 numbers, node_material one per node")
        for tns in (node0, node_material, sigma_n, xi):
            if not tns.is_cuda or not tns.is_contiguous():
                raise ValueError("transport: expected contiguous CUDA tensors")
        t = tracks_struct(tracks)
        o = _abi.TransportOut(*(_ptr(out[k]) for k in ("reason", "steps", "x", "y", "z", "path", "last", "tie")))
        check(lib().gv_transport(self.handle, ctypes.byref(t), _ptr(node0), _ptr(node_material), _ptr(sigma_n),
                                 int(sigma_n.numel() // 2), _ptr(xi), int(kmax), PRECISIONS[precision], ctypes.byref(o),
                                 _stream_ptr(stream)))
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gv_geom_destroy(h)
            self.handle = None


class Server:
    """Continuous-batching navigation service (locate + one step per track)."""

    def __init__(self, geometry: "Geometry", arena_bytes: int = 1 << 30, max_slots: int = 1024, streams: int = 4,
                 precision: str = "fp32_refine"):
        c = _abi.ServerConfig(int(arena_bytes), int(max_slots), int(streams), PRECISIONS[precision], 0)
        h = ctypes.c_void_p()
        check(lib().gv_server_create(geometry.handle, ctypes.byref(c), ctypes.byref(h)))
        self.handle = h
        self.geometry = geometry

    @staticmethod
    def buffers(n: int, pin: bool = True):
        """Host buffers for a request of n tracks: input (6, n) float64, output 24 n bytes."""
        import torch
        inp = torch.empty((6, n), dtype=torch.float64)
        out = torch.empty(24 * max(n, 1), dtype=torch.uint8)
        if pin:
            inp, out = inp.pin_memory(), out.pin_memory()
        return inp, out

    @staticmethod
    def unpack(out, n: int) -> dict:
        import numpy as np
        b = out.numpy()[: 24 * n]
        return {"step": b[: 8 * n].view(np.float64), "safety": b[8 * n: 16 * n].view(np.float64),
                "next": b[16 * n: 20 * n].view(np.int32), "node": b[20 * n: 24 * n].view(np.int32)}

    def submit(self, inp, out) -> int:
        n = inp.shape[1]
        t = ctypes.c_int64()
        check(lib().gv_server_submit(self.handle, n, ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int32()
        check(lib().gv_server_poll(self.handle, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_s: float = 30.0) -> float:
        lat = ctypes.c_double()
        check(lib().gv_server_wait(self.handle, ticket, float(timeout_s), ctypes.byref(lat)))
        return lat.value

    def stats(self) -> dict:
        st = _abi.ServerStats()
        check(lib().gv_server_get_stats(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in _abi.ServerStats._fields_}

    def reset_stats(self):
        check(lib().gv_server_reset_stats(self.handle))

    def close(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gv_server_destroy(h)
            self.handle = None

    def __del__(self):
        self.close()


def version() -> str:
    return lib().gv_version().decode()
