"""Locate and the navigation step on the GPU (C ABI) against the CPU oracle.

Geometries: the nested detector (world box, 10 tube shells, 32 box cells each)
and a random tree of rotated solids of all six types (overlaps allowed: both
definitions are order-based).  Node ids and `next` are compared exactly; step
and safety within 1e-9 mm (FP64) or 1e-5 relative / 1e-9 mm below 1e-4 mm
(FP32 + refinement).
"""
import math

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


def rot(axis, ang):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def random_tree(seed=5):
    g = np.random.default_rng(seed)
    solids = [{"kind": "box", "params": (300.0, 300.0, 300.0)}] + W.solid_table(12, seed=seed)
    nodes = [{"solid": 0, "parent": -1, "R": np.eye(3), "t": np.zeros(3)}]
    for k in range(8):   # daughters of the world
        nodes.append({"solid": 1 + k % 12, "parent": 0, "R": rot(g.normal(size=3), g.uniform(0, 2 * math.pi)),
                      "t": g.uniform(-150, 150, 3)})
    for k in range(10):  # grand-daughters inside the first daughters
        nodes.append({"solid": 1 + (k + 5) % 12, "parent": 1 + k % 4, "R": rot(g.normal(size=3), g.uniform(0, 6.3)),
                      "t": g.uniform(-20, 20, 3)})
    return {"solids": solids, "nodes": nodes}


def geoms():
    return [("nested", W.nested_geometry()), ("random", random_tree())]


def tracks_for(geo, n, seed):
    hb = np.array(geo["solids"][0]["params"])
    g = np.random.default_rng(seed)
    pts = g.uniform(-1, 1, (n, 3)) * hb
    tr = W.soa(pts, W.isotropic(n, g))
    if geo["solids"][0]["params"][2] == 550.0:  # nested: add points on shell and cell surfaces
        m = n // 10
        k = g.integers(0, 10, m)
        r = np.where(g.random(m) < 0.5, 10.0 + 19 * k, 28.0 + 19 * k) + g.uniform(-1e-9, 1e-9, m)
        ph = g.uniform(0, 2 * math.pi, m)
        tr["x"][:m] = r * np.cos(ph)
        tr["y"][:m] = r * np.sin(ph)
    return tr


@pytest.mark.parametrize("which", [0, 1])
def test_locate_exact(gv, which):
    import torch
    name, geo = geoms()[which]
    G = gv.Geometry(geo["solids"], geo["nodes"])
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    tr = tracks_for(geo, 200_003, seed=11 + which)
    dev = to_device(tr, torch)
    got = G.locate(dev).cpu().numpy()
    want = O.locate(tr["x"], tr["y"], tr["z"])
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, (name, bad[:5], got[bad[:5]], want[bad[:5]])
    assert len(np.unique(want)) > 5


def check_nav(got, want, mode, label):
    assert (got["next"] == want["next"]).all(), (label, np.nonzero(got["next"] != want["next"])[0][:5])
    for k in ("step", "safety"):
        g, w = got[k], want[k]
        special = (w == -1) | (w == 0) | ~np.isfinite(w)
        assert ((g == w) | (np.isinf(g) & np.isinf(w)))[special].all(), (label, k)
        fin = ~special
        err = np.abs(g[fin] - w[fin])
        tol = 1e-9 if mode == "fp64" else np.where(np.abs(w[fin]) < 1e-4, 1e-9, 1e-5 * np.abs(w[fin]))
        assert (err <= tol).all(), (label, k, err.max())


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_nav_step(gv, which, precision):
    import torch
    name, geo = geoms()[which]
    G = gv.Geometry(geo["solids"], geo["nodes"])
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    n = 150_001
    tr = tracks_for(geo, n, seed=21 + which)
    node = O.locate(tr["x"], tr["y"], tr["z"])
    dev = to_device(tr, torch)
    dnode = torch.from_numpy(node).cuda()
    ws = gv.Workspace(n)
    out = G.step(dev, dnode, precision=precision, workspace=ws)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    want = O.nav_step(tr["x"], tr["y"], tr["z"], tr["dx"], tr["dy"], tr["dz"], node)
    check_nav(got, want, "fp64" if precision == "fp64" else "fp32", f"{name}-{precision}")
    if precision == "fp32_refine":
        print(name, "nav refined fraction", ws.refined() / n)


def test_nav_invalid_nodes_and_outside(gv):
    import torch
    geo = W.nested_geometry()
    G = gv.Geometry(geo["solids"], geo["nodes"])
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    tr = tracks_for(geo, 1000, seed=3)
    node = np.full(1000, -1, np.int32)
    node[::3] = 9999
    node[1::3] = 0  # world, even for points inside shells: still a defined step
    dev = to_device(tr, torch)
    for precision in ("fp64", "fp32_refine"):
        out = G.step(dev, torch.from_numpy(node).cuda(), precision=precision, workspace=gv.Workspace(1000))
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        want = O.nav_step(tr["x"], tr["y"], tr["z"], tr["dx"], tr["dy"], tr["dz"], node)
        check_nav(got, want, "fp64" if precision == "fp64" else "fp32", precision)
        assert (got["step"][::3] == -1).all()


def grazing_nested_tracks(geo, n, seed):
    """Nested detector tracks that touch or run along surfaces of placed volumes, six kinds in
    turn: (0) on a shell's outer wall, tangent to it; (1) inside a shell, tangent downstream to
    its inner wall; (2) in the gap outside a shell, tangent downstream to its outer wall;
    (3) in a face plane of a rotated cell, outside the face, running along the plane over it;
    (4) inside a shell, touching an edge of a cell; (5) in the gap between two shells at the
    height of their end planes z = +/-500, running horizontally over a shell's end face."""
    g = np.random.default_rng(seed)
    nodes = geo["nodes"]
    cells = [i for i, nd in enumerate(nodes) if nd["solid"] == 1]
    half = np.array([4.5, 4.5, 112.5])
    P, D = [], []
    for m in range(n):
        kind = m % 6
        k = int(g.integers(1, 9))
        rmin, rmax = 10.0 + 19.0 * k, 28.0 + 19.0 * k
        if kind in (0, 1, 2):
            R = rmin if kind == 1 else rmax
            ph = g.uniform(0, 2 * math.pi)
            z = g.choice([-250.0, 0.0, 250.0]) + g.uniform(-5, 5)
            w = g.uniform(-0.3, 0.3)
            c = math.sqrt(1 - w * w)
            sg = 1.0 if g.random() < 0.5 else -1.0
            d = np.array([-sg * c * math.sin(ph), sg * c * math.cos(ph), w])
            # back off along the ray: kind 1 stays inside the shell, kind 2 in the 1 mm gap
            t0 = {0: 0.0, 1: g.uniform(0.5, 5.0), 2: g.uniform(0.2, 0.9) * math.sqrt(2 * R) / c}[kind]
            P.append(np.array([R * math.cos(ph), R * math.sin(ph), z]) - t0 * d)
            D.append(d)
        elif kind in (3, 4):
            nd = nodes[cells[int(g.integers(0, len(cells)))]]
            Rm, t = np.asarray(nd["R"]), np.asarray(nd["t"])
            i, j = g.choice(3, 2, replace=False)
            kk = 3 - i - j
            si, sj = g.choice([-1.0, 1.0], 2)
            dl = np.zeros(3)
            if kind == 3:
                pl = g.uniform(-1, 1, 3) * (half - 0.5)
                pl[i] = si * half[i]
                pl[j] = sj * (half[j] + g.uniform(0.2, 2.0))
                a = g.uniform(-1.2, 1.2)
                dl[j], dl[kk] = -sj * math.cos(a), math.sin(a)
            else:
                E = np.zeros(3)
                E[i], E[j], E[kk] = si * half[i], sj * half[j], g.uniform(-half[kk] + 1, half[kk] - 1)
                beta = g.uniform(0.2, 1.3)
                dl[i], dl[j] = -si * math.cos(beta), sj * math.sin(beta)
                pl = E - g.uniform(0.2, 2.0) * dl
            P.append(t + Rm @ pl)
            D.append(Rm @ dl)
        else:
            ph = g.uniform(0, 2 * math.pi)
            r = rmax + g.uniform(0.2, 0.8)
            a = ph + math.pi + g.uniform(-0.8, 0.8)
            P.append([r * math.cos(ph), r * math.sin(ph), 500.0 if g.random() < 0.5 else -500.0])
            D.append([math.cos(a), math.sin(a), 0.0])
    D = np.asarray(D)
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    return W.soa(np.asarray(P), D)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_nav_grazing(gv, precision):
    """Locate and the navigation step for rays that touch or run along the surfaces of placed
    volumes (the grazing-ray readings applied in each volume's frame): nodes and `next` exact,
    step and safety within the stated tolerances."""
    import torch
    geo = W.nested_geometry()
    G = gv.Geometry(geo["solids"], geo["nodes"])
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    n = 24_000
    tr = grazing_nested_tracks(geo, n, seed=77)
    dev = to_device(tr, torch)
    node = O.locate(tr["x"], tr["y"], tr["z"])
    assert np.array_equal(G.locate(dev).cpu().numpy(), node)
    out = G.step(dev, torch.from_numpy(node).cuda(), precision=precision, workspace=gv.Workspace(n))
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    want = O.nav_step(tr["x"], tr["y"], tr["z"], tr["dx"], tr["dy"], tr["dz"], node)
    check_nav(got, want, "fp64" if precision == "fp64" else "fp32", f"grazing-{precision}")


def test_nav_fp64_tiles_same_bits(gv):
    """Baskets of at least eight 1024-track tiles per SM take the tiled binary64 step (longer runs
    of one volume kind); the per-track arithmetic is unchanged, so step, safety and next equal
    the 256-track-block pass over small chunks bit for bit, in both geometries."""
    import torch
    for name, geo in geoms():
        G = gv.Geometry(geo["solids"], geo["nodes"])
        O = oracle.Geometry(geo["solids"], geo["nodes"])
        n = (1 << 21) + (1 << 20) + 11
        tr = tracks_for(geo, n, seed=61)
        dev = to_device(tr, torch)
        node = G.locate(dev)
        tiled = {k: v.cpu().numpy() for k, v in G.step(dev, node, precision="fp64").items()}
        chunk = 1 << 16
        parts = []
        for o in range(0, n, chunk):
            sub = {k: v[o:o + chunk].contiguous() for k, v in dev.items()}
            parts.append({k: v.cpu().numpy() for k, v in G.step(sub, node[o:o + chunk].contiguous(), precision="fp64").items()})
        torch.cuda.synchronize()
        for k in tiled:
            plain = np.concatenate([p[k] for p in parts])
            assert np.array_equal(plain.view(np.uint8), tiled[k].view(np.uint8)), (name, k)
        idx = np.arange(0, n, 211)
        sub = {k: v[idx] for k, v in tr.items()}
        want = O.nav_step(sub["x"], sub["y"], sub["z"], sub["dx"], sub["dy"], sub["dz"], node.cpu().numpy()[idx])
        check_nav({k: v[idx] for k, v in tiled.items()}, want, "fp64", f"tiles-{name}")
