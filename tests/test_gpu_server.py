"""The continuous-batching navigation service (C ABI, worker thread, device arena).

Every request's results are bit-identical to the same tracks computed alone
(locate + step through the direct calls) and agree with the oracle (node and next
exactly, step and safety at the stated tolerances, zeros and sentinels exactly); requests
arrive while others are on the GPU; a request that can never fit is refused; a
wait on a request that cannot be admitted yet times out with a status and the
service stays usable.
"""
import time

import numpy as np
import pytest

import oracle
import workloads as W
from tests.helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    import torch  # noqa: F401
    import paper_1512_06637_gb300 as gv
    from paper_1512_06637_gb300 import build
    build.build()
    return gv


@pytest.fixture(scope="module")
def geo():
    return W.nested_geometry()


def make_request(server_cls, n, seed, geo):
    tr = W.nested_tracks(n, seed=seed, geom=geo)
    inp, out = server_cls.buffers(n)
    for k, key in enumerate(("x", "y", "z", "dx", "dy", "dz")):
        inp[k].copy_(__import__("torch").from_numpy(tr[key]))
    return tr, inp, out


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64"])
def test_server_alone_equals_mix(gv, geo, precision):
    import torch
    G = gv.Geometry(geo["solids"], geo["nodes"])
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    srv = gv.Server(G, arena_bytes=64 << 20, max_slots=64, streams=3, precision=precision)
    sizes = W.request_sizes(48, seed=7, hi=30000)
    reqs = []
    for i, n in enumerate(sizes):
        tr, inp, out = make_request(gv.Server, int(n), 100 + i, geo)
        reqs.append((tr, inp, out, srv.submit(inp, out)))
        if i % 5 == 4:
            time.sleep(0.001)  # some arrive while earlier groups are on the GPU
    lat = [srv.wait(t, timeout_s=60) for (_, _, _, t) in reqs]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["launches"] >= 2
    assert 0 < st["p50_ms"] <= st["p99_ms"] and all(x > 0 for x in lat)
    ws = gv.Workspace(40000)
    for (tr, inp, out, _) in reqs:
        n = tr["x"].size
        got = gv.Server.unpack(out, n)
        dev = to_device(tr, torch)
        node = G.locate(dev)
        alone = G.step(dev, node, precision=precision, workspace=ws)
        torch.cuda.synchronize()
        assert np.array_equal(got["node"], node.cpu().numpy())
        for k in ("step", "safety", "next"):
            assert np.array_equal(got[k], alone[k].cpu().numpy()), k
        onode = O.locate(tr["x"], tr["y"], tr["z"])
        assert np.array_equal(onode, got["node"])
        w = O.nav_step(tr["x"], tr["y"], tr["z"], tr["dx"], tr["dy"], tr["dz"], onode)
        assert np.array_equal(w["next"], got["next"])
        for k in ("step", "safety"):
            want = w[k]
            assert np.array_equal(np.isfinite(want), np.isfinite(got[k])), k
            assert np.array_equal(want <= 0, got[k] <= 0), k
            assert np.array_equal(got[k][want <= 0], want[want <= 0]), k  # zeros and sentinels exactly
            fin = np.isfinite(want) & (want > 0)
            tol = 1e-9 if precision == "fp64" else np.maximum(1e-9, 1e-5 * np.abs(want[fin]))
            assert (np.abs(got[k][fin] - want[fin]) <= tol).all(), k
    srv.close()


def test_server_refuses_and_times_out(gv, geo):
    G = gv.Geometry(geo["solids"], geo["nodes"])
    arena = 4 << 20  # room for one 16k-track group at a time
    srv = gv.Server(G, arena_bytes=arena, max_slots=8, streams=1, precision="fp64")
    big_n = 200_000
    inp, out = gv.Server.buffers(big_n)
    with pytest.raises(gv.GVError) as e:
        srv.submit(inp, out)
    assert e.value.status == 3
    n = 16_000
    r1 = make_request(gv.Server, n, 1, geo)
    r2 = make_request(gv.Server, n, 2, geo)
    t1 = srv.submit(r1[1], r1[2])
    t2 = srv.submit(r2[1], r2[2])
    with pytest.raises(gv.GVError) as e:
        srv.wait(t2, timeout_s=0.0)
    assert e.value.status == 5
    srv.wait(t1, timeout_s=60)
    srv.wait(t2, timeout_s=60)
    assert srv.stats()["completed"] == 2
    srv.close()
