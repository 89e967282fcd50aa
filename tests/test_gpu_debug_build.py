"""The GV_DEBUG build: device-side checks of the query passes, read back through gv_debug_status.

A library built with GV_DEBUG=1 (libgvgeo_debug.so) checks on the device that directions are
unit vectors and that the refinement worklists stay within their basket.  Here, in a fresh
process with that build: a clean basket records nothing in either precision, and a basket with
one direction 1% too long records GV_DEBUG_DIRECTION with that track's index.  The release build
answers GV_ERR_UNSUPPORTED.
"""
import ctypes
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import ctypes, json, sys
sys.path.insert(0, ROOT)
import torch
from paper_1512_06637_gb300 import build
build.build()
import paper_1512_06637_gb300 as gv
import workloads as W
L = gv.lib()
codes, first = ctypes.c_uint32(0), ctypes.c_int64(0)
def status(clear=1):
    st = L.gv_debug_status(ctypes.byref(codes), ctypes.byref(first), clear)
    return st, codes.value, first.value
res = {"lib": gv._abi.LIB_PATH, "start": status()}
n = 50000
for name, spec in (("tube", W.TUBE_M2), ("polycone", W.polycone_m3()), ("box", W.BOX_M1)):
    tr = W.tracks_for_solid(spec, n, seed=5)
    dev = {k: torch.from_numpy(v).cuda() for k, v in tr.items()}
    s = gv.Solid.from_spec(spec)
    ws = gv.Workspace(n)
    for prec in ("fp32_refine", "fp64"):
        gv.query(s, dev, precision=prec, workspace=ws)
        res[f"{name}_{prec}_clean"] = status()
        bad = {k: v.clone() for k, v in dev.items()}
        for k in ("dx", "dy", "dz"):
            bad[k][12345] *= 1.01
        gv.query(s, bad, precision=prec, workspace=ws)
        res[f"{name}_{prec}_bad"] = status()
print(json.dumps(res))
""".replace("ROOT", repr(ROOT))


def test_debug_build_records_a_bad_direction():
    env = dict(os.environ, GV_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["lib"].endswith("libgvgeo_debug.so")
    assert res["start"][0] == 0
    for key, val in res.items():
        if key in ("lib", "start"):
            continue
        st, codes, first = val
        assert st == 0, key
        if key.endswith("_clean"):
            assert codes == 0 and first == -1, (key, codes, first)
        else:
            assert codes & 1 and first == 12345, (key, codes, first)


def test_release_build_has_no_device_checks():
    import paper_1512_06637_gb300 as gv
    from paper_1512_06637_gb300 import build
    build.build()
    codes, first = ctypes.c_uint32(7), ctypes.c_int64(7)
    st = gv.lib().gv_debug_status(ctypes.byref(codes), ctypes.byref(first), 0)
    assert st == 2 and codes.value == 0 and first.value == -1
