"""The benchmark's CPU baseline: a plain scalar binary64 closed-form loop per solid.

``gv_cpu.cpp`` compiles the library's own binary64 solid code (the closed forms of the
GPU's plain FP64 pass) for the host with -ffp-contract=off and runs it one track per loop
iteration, OpenMP over tracks: the fair CPU counterpart of the GPU path, timed by
``bench.py`` on one core and on all cores, and checked against the oracle by
``tests/test_cpu_baseline.py``.  Measurement infrastructure: the geometry package never
imports it (the library has no CPU path).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "gv_cpu.cpp")
SO = os.path.join(HERE, "_gv_cpu.so")
CSRC = os.path.join(ROOT, "paper_1512_06637_gb300", "csrc")
DEPS = [SRC, os.path.join(HERE, "shim", "cuda_runtime.h"), os.path.join(HERE, "shim", "math_constants.h"),
        os.path.join(CSRC, "solid_fp64.cuh"), os.path.join(CSRC, "desc_build.h"), os.path.join(CSRC, "gv_desc.h"),
        os.path.join(ROOT, "include", "gv.h")]
KINDS = {"box": 0, "trd": 1, "trap": 2, "tube": 3, "cone": 4, "polycone": 5}
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``_gv_cpu.so`` with g++ (no GPU needed)."""
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= max(os.path.getmtime(d) for d in DEPS):
        return SO
    tmp = SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O3", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-I", os.path.join(HERE, "shim"), "-I", os.path.join(ROOT, "include"), "-I", CSRC, SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, SO)
    return SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p, i, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            lib.gvcpu_desc_size.restype = i
            lib.gvcpu_build.argtypes = [i, p, p]
            lib.gvcpu_build.restype = i
            lib.gvcpu_query.argtypes = [p, i64] + [p] * 6 + [p] * 5 + [i]
            lib.gvcpu_query.restype = None
            _lib = lib
        return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Solid:
    """One primitive solid's descriptor, built by the library's host construction code."""

    def __init__(self, spec: dict):
        lib = _load()
        kind, prm = spec["kind"], spec["params"]
        if kind == "trap":
            p = list(prm[0] if len(prm) == 1 else prm)
        elif kind == "polycone":
            z, rmin, rmax, sphi, dphi = prm
            p = [float(len(z))] + list(z) + list(rmin) + list(rmax) + [sphi, dphi]
        elif kind in KINDS:
            p = list(prm)
        else:
            raise ValueError(f"the CPU baseline covers the primitive solids, not {kind!r}")
        arr = np.ascontiguousarray(p, np.float64)
        self._buf = ctypes.create_string_buffer(lib.gvcpu_desc_size())
        st = lib.gvcpu_build(KINDS[kind], _ptr(arr), self._buf)
        if st != 0:
            raise ValueError(f"invalid {kind} parameters (status {st})")

    def query(self, x, y, z, dx, dy, dz, threads: int = 1,
              want=("inside", "dist_in", "dist_out", "safety_in", "safety_out")) -> dict:
        f = lambda a: np.ascontiguousarray(a, np.float64)  # noqa: E731
        x, y, z, dx, dy, dz = map(f, (x, y, z, dx, dy, dz))
        n = len(x)
        out = {k: np.empty(n, np.int8 if k == "inside" else np.float64) for k in want}
        _load().gvcpu_query(self._buf, n, _ptr(x), _ptr(y), _ptr(z), _ptr(dx), _ptr(dy), _ptr(dz),
                            _ptr(out.get("inside")), _ptr(out.get("dist_in")), _ptr(out.get("dist_out")),
                            _ptr(out.get("safety_in")), _ptr(out.get("safety_out")), int(threads))
        return out
