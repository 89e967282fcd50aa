"""The C ABI library loads without a GPU and exports every symbol that
include/gv.h declares; the Python binding declares each of them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gv.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gv_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1512_06637_gb300 import build
    return build.build()


def test_header_declares_calls():
    names = declared()
    for must in ("gv_query", "gv_solid_box", "gv_solid_polycone", "gv_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_1512_06637_gb300 import _abi
    assert sorted(_abi.SIGNATURES) == declared()


def test_invalid_solids_rejected_on_host(libpath):
    """Constructors validate on the host; invalid parameters never reach a device."""
    from paper_1512_06637_gb300 import _abi
    lib = _abi.load(libpath)
    h = ctypes.c_void_p()
    d = ctypes.c_double
    assert lib.gv_solid_box(d(-1), d(1), d(1), ctypes.byref(h)) == _abi.GV_ERR_INVALID_ARG
    assert b"box" in lib.gv_last_error()
    assert lib.gv_solid_tube(d(5), d(4), d(1), d(0), d(1), ctypes.byref(h)) == _abi.GV_ERR_INVALID_ARG
    assert lib.gv_solid_tube(d(1), d(4), d(1), d(0), d(0), ctypes.byref(h)) == _abi.GV_ERR_INVALID_ARG
    assert lib.gv_solid_tube(d(1), d(4), d(float("nan")), d(0), d(1), ctypes.byref(h)) == _abi.GV_ERR_INVALID_ARG
    z = (d * 3)(0, 1, 1)
    r0 = (d * 3)(0, 0, 0)
    r1 = (d * 3)(1, 1, 1)
    assert lib.gv_solid_polycone(3, z, r0, r1, d(0), d(7), ctypes.byref(h)) == _abi.GV_ERR_INVALID_ARG
    z40 = (d * 40)(*range(40))
    r40a = (d * 40)(*([0.0] * 40))
    r40b = (d * 40)(*([1.0] * 40))
    assert lib.gv_solid_polycone(40, z40, r40a, r40b, d(0), d(7), ctypes.byref(h)) == _abi.GV_ERR_UNSUPPORTED
    bad_trap = (d * 11)(10, 0, 0, 5, 5, 5, 0, 5, 5, 5, 1.0)  # alpha1 != alpha2 twists a side face
    assert lib.gv_solid_trap(bad_trap, ctypes.byref(h)) == _abi.GV_ERR_INVALID_ARG
    assert b"planar" in lib.gv_last_error()
    assert lib.gv_query(None, None, 0, None, None, None) == _abi.GV_ERR_INVALID_ARG


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_is_plain_c(lang, tmp_path):
    """include/gv.h compiles on its own as strict C99 and as C++17 (no torch or CUDA types)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("t.c" if lang == "c" else "t.cpp")
    src.write_text('#include "gv.h"\nint main(void) { gv_status s = GV_OK; (void)s; return 0; }\n')
    std = "-std=c99" if lang == "c" else "-std=c++17"
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
