"""CPU oracle for the track-versus-solid queries and the navigation step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is a plain scalar
FP64 C implementation (``gv_oracle.c``) of the three geometry questions of the
paper's VecGeom section (inside/outside, minimal distance to the border, maximal
step along a direction) and of the navigation step (Physics and Detector
geometry subsections); it shares no code with the CUDA library.

The C source is compiled with ``-ffp-contract=off`` (no fused multiply-add) so
that its decision quantities round exactly as written.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gv_oracle.c")
_SO = os.path.join(_HERE, "_gv_oracle.so")
# Test hook: the mutation tests point this at a deliberately broken build.
_SO_OVERRIDE = os.environ.get("GV_ORACLE_SO")
_lock = threading.Lock()
_lib = None

INSIDE, SURFACE, OUTSIDE = 0, 1, 2
HALF_TOL = 0.5e-9
MAXZ = 64


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_gv_oracle.so`` (plain gcc, no GPU)."""
    newer = os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gv_oracle.h")))
    if newer and not force:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if _SO_OVERRIDE:
            lib = ctypes.CDLL(_SO_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_SO)
        d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.or_solid_size.restype = i
        lib.or_bool_size.restype = i
        for name, args in [
            ("or_setup_box", [d, d, d, p]),
            ("or_setup_trap", [p, p]),
            ("or_setup_trd", [d, d, d, d, d, p]),
            ("or_setup_tube", [d, d, d, d, d, p]),
            ("or_setup_cone", [d, d, d, d, d, d, d, p]),
            ("or_setup_pcon", [i, p, p, p, d, d, p]),
            ("or_setup_bool", [i, p, p, p, p, p, p]),
        ]:
            getattr(lib, name).argtypes = args
            getattr(lib, name).restype = i
        lib.or_s_code.argtypes = [p, p]
        lib.or_s_code.restype = d
        lib.or_s_code_n.argtypes = [p, i64, p, p, p, p]
        lib.or_s_code_n.restype = None
        lib.or_query.argtypes = [p, i64] + [p] * 6 + [p] * 5 + [i]
        lib.or_query.restype = None
        lib.or_compose.argtypes = [i, p, p, p, p, p]
        lib.or_compose.restype = None
        lib.or_locate.argtypes = [p, i, p, p, p, p, i64, p, p, p, p, i]
        lib.or_locate.restype = None
        lib.or_nav_step.argtypes = [p, i, p, p, p, p, i64] + [p] * 6 + [p, p, p, p, i]
        lib.or_nav_step.restype = None
        lib.or_transport.argtypes = [p, i, p, p, p, p, p, p, i64] + [p] * 7 + [p, i] + [p] * 8 + [i]
        lib.or_transport.restype = None
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


BOOL_OPS = {"union": 0, "subtraction": 1, "intersection": 2}


class Solid:
    """One solid, set up by the oracle's own constructors from user parameters."""

    def __init__(self, kind: str, *params):
        lib = _load()
        self.kind = kind
        self.params = params
        self._buf = ctypes.create_string_buffer(lib.or_solid_size())
        if kind == "box":
            rc = lib.or_setup_box(*map(float, params), self._buf)
        elif kind == "trd":
            rc = lib.or_setup_trd(*map(float, params), self._buf)
        elif kind == "trap":
            p = _f64(params[0] if len(params) == 1 else params)
            assert p.shape == (11,)
            rc = lib.or_setup_trap(_ptr(p), self._buf)
        elif kind == "tube":
            rc = lib.or_setup_tube(*map(float, params), self._buf)
        elif kind == "cone":
            rc = lib.or_setup_cone(*map(float, params), self._buf)
        elif kind == "polycone":
            z, rmin, rmax, sphi, dphi = params
            z, rmin, rmax = _f64(z), _f64(rmin), _f64(rmax)
            rc = lib.or_setup_pcon(len(z), _ptr(z), _ptr(rmin), _ptr(rmax), float(sphi),
                                   float(dphi), self._buf)
        elif kind == "boolean":
            # (op, component a spec, component c spec, R (3x3, c placed in a), t (3))
            op, sa, sc, R, t = params
            self._parts = (Solid.from_spec(sa), Solid.from_spec(sc))
            self._bool = ctypes.create_string_buffer(lib.or_bool_size())
            R, t = _f64(np.asarray(R, np.float64).reshape(9)), _f64(np.asarray(t, np.float64).reshape(3))
            rc = lib.or_setup_bool(BOOL_OPS[op], self._parts[0].handle, self._parts[1].handle, _ptr(R), _ptr(t),
                                   self._bool, self._buf)
        else:
            raise ValueError(f"unknown solid kind {kind!r}")
        if rc != 0:
            raise ValueError(f"invalid {kind} parameters {params!r}")

    @classmethod
    def from_spec(cls, spec: dict) -> "Solid":
        return cls(spec["kind"], *spec["params"])

    @property
    def handle(self):
        return ctypes.cast(self._buf, ctypes.c_void_p)

    def s_code(self, p) -> float:
        p = _f64(p)
        return _load().or_s_code(self.handle, _ptr(p))

    def s_values(self, pts):
        """The decision quantity s (mm, negative inside) for an (n, 3) array of points."""
        pts = np.atleast_2d(_f64(pts))
        x, y, z = (np.ascontiguousarray(pts[:, i]) for i in range(3))
        out = np.empty(len(x))
        _load().or_s_code_n(self.handle, len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(out))
        return out

    def query(self, x, y, z, dx=None, dy=None, dz=None, threads: int | None = None,
              want=("inside", "dist_in", "dist_out", "safety_in", "safety_out")):
        """All five queries for a structure-of-arrays basket; returns a dict."""
        x, y, z = _f64(x), _f64(y), _f64(z)
        n = len(x)
        need_dir = "dist_in" in want or "dist_out" in want
        if need_dir:
            dx, dy, dz = _f64(dx), _f64(dy), _f64(dz)
        out = {}
        for k in want:
            out[k] = np.empty(n, np.int8 if k == "inside" else np.float64)
        _load().or_query(self.handle, n, _ptr(x), _ptr(y), _ptr(z),
                         _ptr(dx) if need_dir else None, _ptr(dy) if need_dir else None,
                         _ptr(dz) if need_dir else None,
                         _ptr(out.get("inside")), _ptr(out.get("dist_in")),
                         _ptr(out.get("dist_out")), _ptr(out.get("safety_in")),
                         _ptr(out.get("safety_out")), int(threads or default_threads()))
        return out

    def inside(self, pts, threads=None):
        pts = np.atleast_2d(_f64(pts))
        return self.query(pts[:, 0], pts[:, 1], pts[:, 2], threads=threads, want=("inside",))["inside"]


def default_threads() -> int:
    return int(os.environ.get("GV_ORACLE_THREADS", os.cpu_count() or 1))


class Geometry:
    """A tree of placed volumes: node 0 is the world, parents precede children.

    ``nodes`` is a list of dicts ``{"solid": index, "parent": int, "R": 3x3, "t": 3}``
    (R, t place the node in its parent: p_parent = R p_local + t).
    """

    def __init__(self, solids: list, nodes: list):
        lib = _load()
        self.solids = [s if isinstance(s, Solid) else Solid.from_spec(s) for s in solids]
        sz = lib.or_solid_size()
        self._arr = ctypes.create_string_buffer(sz * len(self.solids))
        for i, s in enumerate(self.solids):
            ctypes.memmove(ctypes.addressof(self._arr) + i * sz, s._buf, sz)
        nn = len(nodes)
        self.nnodes = nn
        self.node_solid = np.array([nd["solid"] for nd in nodes], np.int32)
        self.parent = np.array([nd["parent"] for nd in nodes], np.int32)
        RL = _f64(np.array([np.asarray(nd["R"], np.float64).reshape(9) for nd in nodes]))
        tl = _f64(np.array([np.asarray(nd["t"], np.float64).reshape(3) for nd in nodes]))
        self.RG = np.empty((nn, 9), np.float64)
        self.tg = np.empty((nn, 3), np.float64)
        lib.or_compose(nn, _ptr(self.parent), _ptr(RL), _ptr(tl), _ptr(self.RG), _ptr(self.tg))

    def _common(self):
        return (ctypes.cast(self._arr, ctypes.c_void_p), self.nnodes, _ptr(self.node_solid),
                _ptr(self.parent), _ptr(self.RG), _ptr(self.tg))

    def locate(self, x, y, z, threads=None):
        x, y, z = _f64(x), _f64(y), _f64(z)
        node = np.empty(len(x), np.int32)
        _load().or_locate(*self._common(), len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(node),
                          int(threads or default_threads()))
        return node

    def transport(self, x, y, z, dx, dy, dz, node0, node_material, sigma_n, xi, kmax, threads=None):
        """Transport loop (Physics subsection; see or_transport): random numbers ``xi`` of
        shape (n, kmax, 4) in (0, 1]; ``sigma_n`` (nmat, 2) = n sigma of the scatter and absorb
        processes per material (1/mm); returns reason, steps, final point, path, last node, tie."""
        x, y, z, dx, dy, dz = map(_f64, (x, y, z, dx, dy, dz))
        n = len(x)
        node0 = np.ascontiguousarray(node0, np.int32)
        mat = np.ascontiguousarray(node_material, np.int32)
        sig = _f64(np.asarray(sigma_n, np.float64).reshape(-1))
        xi = _f64(np.asarray(xi, np.float64).reshape(-1))
        assert xi.size == n * kmax * 4 and mat.size == self.nnodes
        out = {"reason": np.empty(n, np.int8), "steps": np.empty(n, np.int32), "x": np.empty(n), "y": np.empty(n),
               "z": np.empty(n), "path": np.empty(n), "last": np.empty(n, np.int32), "tie": np.empty(n, np.int8)}
        _load().or_transport(*self._common(), _ptr(mat), _ptr(sig), n, _ptr(x), _ptr(y), _ptr(z), _ptr(dx),
                             _ptr(dy), _ptr(dz), _ptr(node0), _ptr(xi), int(kmax), _ptr(out["reason"]),
                             _ptr(out["steps"]), _ptr(out["x"]), _ptr(out["y"]), _ptr(out["z"]),
                             _ptr(out["path"]), _ptr(out["last"]), _ptr(out["tie"]),
                             int(threads or default_threads()))
        return out

    def nav_step(self, x, y, z, dx, dy, dz, node, threads=None):
        x, y, z, dx, dy, dz = map(_f64, (x, y, z, dx, dy, dz))
        node = np.ascontiguousarray(node, np.int32)
        n = len(x)
        step = np.empty(n, np.float64)
        saf = np.empty(n, np.float64)
        nxt = np.empty(n, np.int32)
        _load().or_nav_step(*self._common(), n, _ptr(x), _ptr(y), _ptr(z), _ptr(dx), _ptr(dy),
                            _ptr(dz), _ptr(node), _ptr(step), _ptr(saf), _ptr(nxt),
                            int(threads or default_threads()))
        return {"step": step, "safety": saf, "next": nxt}
