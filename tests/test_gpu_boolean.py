"""Boolean solids on the device (binary64 throughout) against the oracle: codes bit-exact,
distances and safeties within 1e-9 mm, on random unions, subtractions and intersections of
every primitive kind; the FP32+refine call gives the same bits (booleans have no binary32
pass); booleans inside a mixed batch and as daughters in navigation; constructor checks."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.helpers import QUERIES, compare, to_device, to_host

pytestmark = pytest.mark.gpu

TABLE = W.boolean_table(24, seed=13)


@pytest.fixture(scope="module")
def gv():
    import torch  # noqa: F401
    import paper_1512_06637_gb300 as gv
    from paper_1512_06637_gb300 import build
    build.build()
    return gv


@pytest.mark.parametrize("i", range(len(TABLE)))
def test_boolean_parity(gv, i):
    import torch
    spec = TABLE[i]
    n = 20011
    tr = W.tracks_for_solid(spec, n, seed=900 + i, near_frac=0.2)
    s = gv.Solid.from_spec(spec)
    dev = to_device(tr, torch)
    got = gv.query(s, dev, precision="fp64")
    ws = gv.Workspace(n)
    got32 = gv.query(s, dev, precision="fp32_refine", workspace=ws)
    torch.cuda.synchronize()
    want = oracle.Solid.from_spec(spec).query(**tr)
    compare(to_host(got), want, "fp64", f"boolean {i} {spec['params'][0]}")
    for k in QUERIES:
        assert torch.equal(got[k], got32[k]), k
    assert ws.refined() == 0


def test_boolean_grazing(gv):
    """A box with a square through-hole (subtraction): points on the hole's wall and on its
    plane above the box, rays into the material, into the hole and along the wall, plus
    rays touching the outer box's edges: parity with the oracle at 1e-9 mm."""
    import torch
    spec = {"kind": "boolean", "params": ("subtraction", {"kind": "box", "params": (20.0, 20.0, 20.0)},
                                          {"kind": "box", "params": (5.0, 5.0, 30.0)}, np.eye(3), np.zeros(3))}
    g = np.random.default_rng(41)
    n = 3000
    y, z = g.uniform(-4, 4, n), g.uniform(-19, 19, n)
    p = np.stack([np.full(n, 5.0), y, z], 1)
    k = g.integers(0, 5, n)
    d = np.zeros((n, 3))
    d[k == 0, 0], d[k == 1, 0], d[k == 2, 2], d[k == 3, 2] = 1.0, -1.0, 1.0, -1.0
    a = g.uniform(0, 2 * np.pi, n)
    d[k == 4, 1], d[k == 4, 2] = np.cos(a[k == 4]), np.sin(a[k == 4])  # in the wall's plane
    top = g.random(n) < 0.3
    p[top, 2] = 25.0
    d[top] = [0.0, 0.0, -1.0]
    tr = W.soa(p, d)
    s = gv.Solid.from_spec(spec)
    got = gv.query(s, to_device(tr, torch), precision="fp64")
    torch.cuda.synchronize()
    compare(to_host(got), oracle.Solid.from_spec(spec).query(**tr), "fp64", "hole-wall")
    # the outer box's edges, touched and crossed: the box family for (10, 20, 30) mapped onto
    # (20, 20, 20) by an axis scaling (lines touching an edge stay lines touching the edge)
    _, tb, _ = W.grazing_tracks("box_edge_touch", 2000, 42)
    sc = np.array([2.0, 1.0, 2.0 / 3.0])
    P = np.stack([tb["x"], tb["y"], tb["z"]], 1) * sc
    D = np.stack([tb["dx"], tb["dy"], tb["dz"]], 1) * sc
    tb = W.soa(P, D / np.linalg.norm(D, axis=1, keepdims=True))
    got = gv.query(s, to_device(tb, torch), precision="fp64")
    torch.cuda.synchronize()
    compare(to_host(got), oracle.Solid.from_spec(spec).query(**tb), "fp64", "outer-edges")


def test_boolean_in_batch_and_navigation(gv):
    import torch
    # a batch mixing booleans and primitives
    solids = [W.BOX_M1, TABLE[0], W.TUBE_M2, TABLE[1], TABLE[2]]
    n_each = 3001
    trs = [W.tracks_for_solid(sp, n_each, seed=950 + j) for j, sp in enumerate(solids)]
    tr = {k: np.concatenate([t[k] for t in trs]) for k in trs[0]}
    offsets = np.arange(len(solids)) * n_each
    b = gv.Batch([gv.Solid.from_spec(sp) for sp in solids], offsets, np.full(len(solids), n_each),
                 np.arange(len(solids)))
    dev = to_device(tr, torch)
    for prec in ("fp64", "fp32_refine"):
        out = gv.alloc_results(len(tr["x"]), "cuda")
        b.run(dev, out, precision=prec)
        torch.cuda.synchronize()
        got = to_host(out)
        for j, sp in enumerate(solids):
            sl = slice(j * n_each, (j + 1) * n_each)
            want = oracle.Solid.from_spec(sp).query(**trs[j])
            compare({k: v[sl] for k, v in got.items()}, want, "fp32" if prec == "fp32_refine" else "fp64",
                    f"batch {prec} {j}")
    # a boolean daughter in the world box
    geo = {"solids": [{"kind": "box", "params": (200.0, 200.0, 200.0)}, TABLE[3], TABLE[4]],
           "nodes": [{"solid": 0, "parent": -1, "R": np.eye(3), "t": np.zeros(3)},
                     {"solid": 1, "parent": 0, "R": np.eye(3), "t": np.array([-80.0, 0, 0])},
                     {"solid": 2, "parent": 0, "R": W.random_rotation(np.random.default_rng(3)),
                      "t": np.array([80.0, 10.0, 0])}]}
    G = gv.Geometry(geo["solids"], geo["nodes"])
    O = oracle.Geometry(geo["solids"], geo["nodes"])
    g = np.random.default_rng(4)
    n = 20000
    P = g.uniform(-1, 1, (n, 3)) * 190.0
    d = W.isotropic(n, g)
    t = W.soa(P, d)
    dt = to_device(t, torch)
    node = G.locate(dt)
    onode = O.locate(t["x"], t["y"], t["z"])
    assert np.array_equal(node.cpu().numpy(), onode)
    want = O.nav_step(t["x"], t["y"], t["z"], t["dx"], t["dy"], t["dz"], onode)
    ws = gv.Workspace(n)
    for prec in ("fp64", "fp32_refine"):
        r = G.step(dt, node, precision=prec, workspace=ws)
        torch.cuda.synchronize()
        assert np.array_equal(r["next"].cpu().numpy(), want["next"]), prec
        st = r["step"].cpu().numpy()
        fin = np.isfinite(want["step"]) & (want["step"] > 0)
        tol = 1e-9 if prec == "fp64" else np.maximum(1e-9, 1e-5 * want["step"][fin])
        assert (np.abs(st[fin] - want["step"][fin]) <= tol).all(), prec


def test_boolean_constructor_checks(gv):
    a, c = W.BOX_M1, W.TUBE_M2
    refl = np.diag([1.0, 1.0, -1.0])
    with pytest.raises(gv.GVError) as e:
        gv.Solid("boolean", "union", a, c, refl, np.zeros(3))
    assert e.value.status == 1
    with pytest.raises(gv.GVError) as e:
        gv.Solid("boolean", "union", a, c, np.eye(3) * 1.01, np.zeros(3))
    assert e.value.status == 1
    nested = {"kind": "boolean", "params": ("union", a, c, np.eye(3), np.zeros(3))}
    with pytest.raises(gv.GVError) as e:
        gv.Solid("boolean", "subtraction", nested, c, np.eye(3), np.zeros(3))
    assert e.value.status == 2
