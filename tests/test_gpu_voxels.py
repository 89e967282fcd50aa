"""Voxelised navigation: a node with many daughters carries a uniform grid over their
bounding boxes, and locate, the navigation step and the transport loop give the same
bits with the grids on and off (the grid only skips daughters that cannot matter, and
ties are broken by the same rule), and the same results as the oracle, which always
looks at every daughter.

Geometries: the crowded lattice (1728 daughters of the world, one of them a rotated box
holding 27 more) and the nested detector (a grid in each of the 10 shells)."""
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
def crowded():
    return W.crowded_geometry()


def test_voxel_counts(gv, crowded):
    assert gv.Geometry(crowded["solids"], crowded["nodes"]).voxel_count == 2
    nested = W.nested_geometry()
    assert gv.Geometry(nested["solids"], nested["nodes"]).voxel_count == 10
    # 15 daughters: no grid; 16: a grid
    for k, want in ((15, 0), (16, 1)):
        geo = {"solids": crowded["solids"], "nodes": crowded["nodes"][:1] + crowded["nodes"][2:2 + k]}
        assert gv.Geometry(geo["solids"], geo["nodes"]).voxel_count == want


def both(G, fn):
    G.set_voxels(True)
    on = fn()
    G.set_voxels(False)
    off = fn()
    G.set_voxels(True)
    return on, off


def check_nav(got, want, mode, label):
    assert (got["next"] == want["next"]).all(), (label, np.nonzero(got["next"] != want["next"])[0][:5])
    for k in ("step", "safety"):
        if k not in got:
            continue
        g, w = got[k], want[k]
        special = (w == -1) | (w == 0) | ~np.isfinite(w)
        assert ((g == w) | (np.isinf(g) & np.isinf(w)))[special].all(), (label, k)
        fin = ~special
        tol = 1e-9 if mode == "fp64" else np.where(np.abs(w[fin]) < 1e-4, 1e-9, 1e-5 * np.abs(w[fin]))
        err = np.abs(g[fin] - w[fin])
        assert (err <= tol).all(), (label, k, err.max())


@pytest.mark.parametrize("which", ["crowded", "nested"])
def test_voxel_locate_and_step(gv, crowded, which):
    import torch
    geo = crowded if which == "crowded" else W.nested_geometry()
    G = gv.Geometry(geo["solids"], geo["nodes"])
    n = 400_003
    tr = W.crowded_tracks(geo, n, seed=3) if which == "crowded" else W.nested_tracks(n, seed=3)
    dev = to_device(tr, torch)

    on, off = both(G, lambda: G.locate(dev).cpu().numpy())
    assert np.array_equal(on, off)
    node = torch.from_numpy(on).cuda()
    res = {}
    for precision in ("fp64", "fp32_refine"):
        for saf in (True, False):
            ws = gv.Workspace(n)

            def run():
                o = G.step(dev, node, precision=precision, workspace=ws, safety=saf)
                torch.cuda.synchronize()
                return {k: v.cpu().numpy() for k, v in o.items()}

            s_on, s_off = both(G, run)
            assert ("safety" in s_on) == saf
            label = (which, precision, saf)
            if precision == "fp64":  # binary64: the same bits
                for k in s_on:
                    assert np.array_equal(s_on[k], s_off[k], equal_nan=True), (label, k)
            else:  # the same daughter; values within the binary32 tolerance of each other
                check_nav(s_on, s_off, "fp32", label)
            res[precision, saf] = s_on
    # leaving the safety out changes nothing else
    for k in ("step", "next"):
        assert np.array_equal(res["fp64", True][k], res["fp64", False][k]), k
    check_nav(res["fp32_refine", False], res["fp32_refine", True], "fp32", "fp32 without safety")

    # against the oracle on a sample (the oracle scans every daughter)
    m = 40_000
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    sub = {k: v[:m] for k, v in tr.items()}
    want_node = O.locate(sub["x"], sub["y"], sub["z"])
    assert np.array_equal(on[:m], want_node)
    want = O.nav_step(sub["x"], sub["y"], sub["z"], sub["dx"], sub["dy"], sub["dz"], want_node)
    for precision in ("fp64", "fp32_refine"):
        got = {k: v[:m] for k, v in res[precision, True].items()}
        check_nav(got, want, "fp64" if precision == "fp64" else "fp32", (which, precision))


def test_voxel_transport(gv, crowded):
    import torch
    geo = crowded
    G = gv.Geometry(geo["solids"], geo["nodes"])
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    n, kmax = 50_001, 48
    tr = W.crowded_tracks(geo, n, seed=8, surf_frac=0.0)
    mats = W.crowded_materials(geo)
    xi = W.transport_xi(n, kmax, seed=8)
    node0 = O.locate(tr["x"], tr["y"], tr["z"])
    dev = to_device(tr, torch)
    args = (torch.from_numpy(node0).cuda(), torch.from_numpy(mats["node_material"]).cuda(),
            torch.from_numpy(mats["sigma_n"]).cuda(), torch.from_numpy(xi).cuda())

    def run():
        o = G.transport(dev, *args, kmax)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in o.items()}

    on, off = both(G, run)
    for k in on:
        assert np.array_equal(on[k], off[k]), k
    assert on["steps"].mean() > 3  # tracks cross several daughters
    m = 5_000
    want = O.transport(*(tr[k][:m] for k in ("x", "y", "z", "dx", "dy", "dz")), node0[:m], mats["node_material"],
                       mats["sigma_n"], xi[:m], kmax)
    sure = (on["tie"][:m] == 0) & (want["tie"] == 0)
    assert sure.mean() > 0.98
    for k in ("reason", "steps", "last"):
        assert np.array_equal(on[k][:m][sure], want[k][sure]), k
    worst = 0.0
    for k in ("x", "y", "z", "path"):  # the transport test's bound: 1e-9 mm + 1e-12 relative
        err = np.abs(on[k][:m][sure] - want[k][sure])
        assert (err <= 1e-9 + 1e-12 * np.abs(want[k][sure])).all(), (k, err.max())
        worst = max(worst, float(err.max()))
    print(f"largest end point / path difference: {worst:.3e} mm")
