"""The allocation-free query entry point, checked through the C ABI.

gv_query_fp32_static serves callers that cannot allocate device memory while
they run queries (a framework owning all device memory through its own pool, a
serving loop that cannot take cudaMalloc's implicit synchronisation, a plug-in
without an allocator): its scratch lives in a fixed device array inside the
library.  It runs the same kernels as the workspace-based GV_FP32_REFINE pass, so
two calls in a row must each reproduce that pass bit for bit; the first is also
checked against the CPU oracle at the tests' tolerance (codes exact; 1e-5
relative, 1e-9 mm below 1e-4 mm; sentinels exact).  The baskets are chosen so that
the refinement worklist in the fixed array is used (some tracks are refined).  A
basket above the fixed limit must be refused, an empty one accepted.  This file is
collected last so that a run stopping at the first failure has run every other
test before it.
"""
import ctypes

import pytest

import oracle
import workloads as W
from tests.helpers import QUERIES, compare, to_device

pytestmark = pytest.mark.gpu

LIMIT = 1 << 20


@pytest.fixture(scope="module")
def gv():
    import torch  # noqa: F401
    import paper_1512_06637_gb300 as gv
    from paper_1512_06637_gb300 import build
    build.build()
    return gv


def _static_call(gv, solid, dev, out):
    import torch
    from paper_1512_06637_gb300 import _abi
    t = gv.tracks_struct(dev)
    r = gv.results_struct(out, dev["x"].numel())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _abi.lib().gv_query_fp32_static(solid.handle, ctypes.byref(t), ctypes.byref(r), stream)


@pytest.mark.parametrize("spec,n", [(W.TUBE_M2, 200_003), (W.polycone_m3(), 150_001), (W.BOX_M1, LIMIT)])
def test_static_matches_workspace_pass_twice(gv, spec, n):
    import torch
    tr = W.tracks_for_solid(spec, n, seed=4242)
    dev = to_device(tr, torch)
    s = gv.Solid.from_spec(spec)
    ws = gv.Workspace(n)
    ref = gv.query(s, dev, precision="fp32_refine", workspace=ws)
    torch.cuda.synchronize()
    assert ws.refined() > 0  # the worklist and its counter are exercised
    want = oracle.Solid.from_spec(spec).query(**tr)
    for call in range(2):
        out = gv.alloc_results(n, "cuda")
        for v in out.values():
            v.fill_(7)  # stale values must be overwritten
        st = _static_call(gv, s, dev, out)
        assert st == 0, gv.lib().gv_last_error()
        torch.cuda.synchronize()
        assert set(out) == set(QUERIES)
        for k in QUERIES:
            assert torch.equal(out[k], ref[k]), (call, k)
        if call == 0:
            compare({k: v.cpu().numpy() for k, v in out.items()}, want, "fp32", f"static {spec['kind']}")


def test_static_rejects_oversized_basket(gv):
    import torch
    n = LIMIT + 1
    dev = {k: torch.zeros(n, dtype=torch.float64, device="cuda") for k in ("x", "y", "z", "dx", "dy", "dz")}
    out = gv.alloc_results(n, "cuda")
    s = gv.Solid.from_spec(W.BOX_M1)
    st = _static_call(gv, s, dev, out)
    assert st == 1
    assert b"1048576" in gv.lib().gv_last_error()


def test_static_accepts_empty_basket(gv):
    import torch
    dev = {k: torch.zeros(0, dtype=torch.float64, device="cuda") for k in ("x", "y", "z", "dx", "dy", "dz")}
    out = gv.alloc_results(0, "cuda")
    st = _static_call(gv, gv.Solid.from_spec(W.BOX_M1), dev, out)
    assert st == 0, gv.lib().gv_last_error()
