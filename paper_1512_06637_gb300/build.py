"""Build the CUDA library ``libgvgeo.so`` in-tree for sm_103a (with ``GV_DEBUG=1`` in the
environment: ``libgvgeo_debug.so``, the build with device-side checks, objects in ``_build_debug/``).

Each ``csrc/*.cu`` is compiled to an object in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a``; the objects are linked into
``paper_1512_06637_gb300/libgvgeo.so``.  Host code is compiled with
``-ffp-contract=off`` so that the solid constructors round every expression as
written.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
DEBUG = os.environ.get("GV_DEBUG", "0") not in ("", "0")  # the build with device-side checks
OBJ = os.path.join(PKG, "_build_debug" if DEBUG else "_build")
LIB = os.path.join(PKG, "libgvgeo_debug.so" if DEBUG else "libgvgeo.so")
PROBE = os.path.join(PKG, "libgvprobe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgvgeo.so")
    return cand


def flags() -> list[str]:
    # --fmad=false: a multiply-add is fused only where the source writes fmaf/fma, so the
    # single-solid, batched, navigation and service kernels compute the same bits for a
    # track (contraction left to the compiler differs between kernels that inline the
    # same arithmetic).
    return ARCH + ["-O3", "--fmad=false", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xcompiler", "-ffp-contract=off", "-Xptxas", "-warn-spills",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC] + (["-DGV_DEBUG=1"] if DEBUG else [])


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.abspath(__file__), os.path.join(ROOT, "include", "gv.h")]  # flags, ABI
    headers.append(os.path.join(ROOT, "include", "gv.h"))
    srcs = sources()
    objs = [os.path.join(OBJ, os.path.basename(s)[:-3] + ".o") for s in srcs]
    todo = [(s, o) for s, o in zip(srcs, objs) if force or _stale(o, [s] + headers)]
    cc = nvcc()

    def one(so):
        s, o = so
        cmd = [cc, "-c", s, "-o", o + ".tmp"] + flags()
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s}:\n{r.stdout}\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return s, r.stderr

    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for s, err in ex.map(one, todo):
                if verbose and err.strip():
                    print(f"[{os.path.basename(s)}]\n{err}", file=sys.stderr)
    if force or todo or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    build_probe(force)
    return LIB


def build_probe(force: bool = False) -> str:
    """The benchmark's throughput probes (``probe/gvprobe.cu`` -> ``libgvprobe.so``): binary32
    and binary64 multiply-add, integer-pipe and instruction-issue rates.  Not part of the
    geometry library."""
    src = os.path.join(PKG, "probe", "gvprobe.cu")
    if force or _stale(PROBE, [src, os.path.abspath(__file__)]):
        tmp = PROBE + f".tmp{os.getpid()}"
        cmd = [nvcc(), src, "-shared", "-o", tmp, "-lcudart"] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, PROBE)
    return PROBE


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
