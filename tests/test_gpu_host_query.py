"""Baskets in host memory (gv_query_host): chunked streaming through device staging
slots gives the same bits as gv_query on device arrays, for both precisions, pinned
and pageable host memory, ragged last chunks, skipped queries, a basket smaller than
one chunk, consecutive calls that overlap on one pipeline, and it agrees with the
oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.helpers import QUERIES, compare, to_device

pytestmark = pytest.mark.gpu

SPECS = {"box": W.BOX_M1, "tube": W.TUBE_M2, "polycone": W.polycone_m3()}


@pytest.fixture(scope="module")
def gv():
    import torch  # noqa: F401
    import paper_1512_06637_gb300 as gv
    from paper_1512_06637_gb300 import build
    build.build()
    return gv


def host_out(n, pinned, want=QUERIES):
    import torch
    out = {}
    for k in want:
        t = torch.empty(n, dtype=torch.int8 if k == "inside" else torch.float64)
        out[k] = t.pin_memory() if pinned else t.numpy()
    return out


def as_np(v):
    return v if isinstance(v, np.ndarray) else v.numpy()


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64"])
@pytest.mark.parametrize("name", list(SPECS))
def test_host_equals_device(gv, name, precision):
    import torch
    spec = SPECS[name]
    chunk = 4096
    n = 3 * chunk + 17
    tr = W.tracks_for_solid(spec, n, seed=41)
    s = gv.Solid.from_spec(spec)
    ws = gv.Workspace(n)
    ref = gv.query(s, to_device(tr, torch), precision=precision, workspace=ws)
    torch.cuda.synchronize()
    for pinned, slots in ((True, 3), (False, 2)):
        p = gv.Pipeline(chunk, slots)
        host_in = {k: torch.from_numpy(v).pin_memory() for k, v in tr.items()} if pinned else tr
        out = host_out(n, pinned)
        gv.query_host(s, host_in, out, p, precision=precision)
        p.join()
        torch.cuda.synchronize()
        for k in QUERIES:
            assert np.array_equal(as_np(out[k]), ref[k].cpu().numpy(), equal_nan=True), (pinned, k)
    want = oracle.Solid.from_spec(spec).query(**tr)
    compare({k: as_np(v) for k, v in out.items()}, want, "fp32" if precision == "fp32_refine" else "fp64",
            f"host-{name}")


def test_host_partial_small_and_overlapping(gv):
    import torch
    p = gv.Pipeline(1000, 2)
    # safeties and codes only, no directions; basket smaller than one chunk
    spec = SPECS["polycone"]
    tr = W.tracks_for_solid(spec, 777, seed=5)
    pts = {k: tr[k] for k in ("x", "y", "z")}
    out = host_out(777, True, ("inside", "safety_in", "safety_out"))
    s = gv.Solid.from_spec(spec)
    gv.query_host(s, pts, out, p, precision="fp64")
    p.join()
    torch.cuda.synchronize()
    want = oracle.Solid.from_spec(spec).query(**tr)
    compare({k: as_np(v) for k, v in out.items()}, want, "fp64", "host-partial")
    # empty basket: nothing enqueued
    empty = {k: np.empty(0) for k in ("x", "y", "z", "dx", "dy", "dz")}
    gv.query_host(s, empty, host_out(0, False), p)
    # two solids back to back on one pipeline: the second call's first chunks overlap
    # the first call's last ones
    specs = [SPECS["box"], SPECS["tube"]]
    outs, trs = [], []
    for i, sp in enumerate(specs):
        t = W.tracks_for_solid(sp, 5 * 1000 + 3, seed=60 + i)
        o = host_out(5003, True)
        gv.query_host(gv.Solid.from_spec(sp), {k: torch.from_numpy(v).pin_memory() for k, v in t.items()}, o, p,
                      precision="fp32_refine")
        outs.append(o)
        trs.append(t)
    p.join()
    torch.cuda.synchronize()
    for sp, t, o in zip(specs, trs, outs):
        compare({k: as_np(v) for k, v in o.items()}, oracle.Solid.from_spec(sp).query(**t), "fp32", "host-seq")


def test_host_rejects_bad_arguments(gv):
    with pytest.raises(gv.GVError) as e:
        gv.Pipeline(1024, 1)
    assert e.value.status == 1
    with pytest.raises(gv.GVError):
        gv.Pipeline(0, 2)
    p = gv.Pipeline(1024, 2)
    s = gv.Solid.from_spec(SPECS["box"])
    tr = W.tracks_for_solid(SPECS["box"], 100, seed=1)
    bad = {k: v for k, v in tr.items()}
    raw = np.zeros(101 * 8 + 4, np.uint8)
    bad["x"] = raw[4:4 + 800].view(np.float64)  # misaligned by 4 bytes
    with pytest.raises(Exception):
        gv.query_host(s, bad, host_out(100, False), p)
