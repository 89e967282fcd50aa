"""The seeded input generators hold what their recipes state (CPU only): the crowded lattice
(node count, valid tree, proper rotations, daughters whose bounding spheres do not meet,
the second level inside its box), its tracks (surface points on a daughter's surface,
axis-aligned directions) and the bounding boxes that the grids and the samplers use."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def crowded():
    return W.crowded_geometry()


def test_crowded_tree(crowded):
    nodes = crowded["nodes"]
    assert len(nodes) == 1 + 12 ** 3 + 27
    assert nodes[0]["parent"] == -1
    for i, nd in enumerate(nodes[1:], start=1):
        assert 0 <= nd["parent"] < i
        R = np.asarray(nd["R"])
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) > 0
    world_kids = [nd for nd in nodes if nd["parent"] == 0]
    assert len(world_kids) == 12 ** 3
    sub = [i for i, nd in enumerate(nodes) if nd["parent"] == 0 and
           crowded["solids"][nd["solid"]] == {"kind": "box", "params": (28.0, 28.0, 28.0)}]
    assert len(sub) == 1
    assert sum(nd["parent"] == sub[0] for nd in nodes) == 27


def test_crowded_daughters_do_not_meet(crowded):
    solids, nodes = crowded["solids"], crowded["nodes"]
    kids = [nd for nd in nodes if nd["parent"] == 0]
    c = np.array([nd["t"] for nd in kids])
    r = np.array([np.linalg.norm(W.bounding_half(solids[nd["solid"]])) for nd in kids])
    assert (np.abs(c) + r[:, None] <= 600.0).all()  # inside the world box
    # neighbours on the lattice are the only candidates (pitch 100 mm, radii < 70 mm)
    for i in range(len(kids)):
        d = np.linalg.norm(c - c[i], axis=1)
        close = (d > 0) & (d < 150.0)
        assert (d[close] > r[i] + r[close]).all()
    sub = [i for i, nd in enumerate(nodes) if nd["parent"] == 0 and solids[nd["solid"]]["params"] == (28.0, 28.0, 28.0)][0]
    for nd in nodes:
        if nd["parent"] == sub:
            rr = np.linalg.norm(W.bounding_half(solids[nd["solid"]]))
            assert (np.abs(nd["t"]) + rr <= 28.0).all()


@pytest.mark.parametrize("seed", [0, 1])
def test_bounding_half_holds_the_surface(seed):
    g = np.random.default_rng(seed)
    specs = [W.random_solid(k, g, 4.0, 26.0) for k in W.KINDS6] + [W.boolean_random(g, 5.0, 18.0) for _ in range(4)]
    specs += [W._scaled(W.random_solid(k, g, 4.0, 26.0), 0.2) for k in W.KINDS6]
    for spec in specs:
        hb = W.bounding_half(spec)
        pts = W._sample_surface(spec, 2000, g)
        assert (np.abs(pts) <= hb * (1 + 1e-12) + 1e-12).all(), spec["kind"]


def test_scaled_solid_is_similar():
    g = np.random.default_rng(3)
    for k in W.KINDS6:
        spec = W.random_solid(k, g, 4.0, 26.0)
        small = W._scaled(spec, 0.2)
        tr = W.tracks_for_solid(spec, 500, seed=4, near_frac=0.0)
        want = oracle.Solid.from_spec(spec).query(**tr, want=("inside", "dist_out"))
        scaled = {key: v * 0.2 if key in ("x", "y", "z") else v for key, v in tr.items()}
        got = oracle.Solid.from_spec(small).query(**scaled, want=("inside", "dist_out"))
        sure = want["inside"] != 1
        assert (got["inside"][sure] == want["inside"][sure]).all(), k
        fin = sure & (want["dist_out"] > 0)
        assert np.allclose(got["dist_out"][fin], 0.2 * want["dist_out"][fin], rtol=1e-9, atol=1e-9), k


def test_crowded_tracks(crowded):
    n = 20000
    tr = W.crowded_tracks(crowded, n, seed=5)
    d = np.stack([tr["dx"], tr["dy"], tr["dz"]], axis=1)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    axis = (np.abs(d) == 1.0).any(axis=1)
    assert abs(axis.mean() - 0.1) < 0.01
    # 30% of the points were drawn on the surface of a world daughter (a boolean's on either
    # component's surface, not always its own): the oracle classifies them SURFACE there
    O = oracle.Geometry(crowded["solids"], crowded["nodes"])
    node = O.locate(tr["x"], tr["y"], tr["z"])
    solids, nodes = crowded["solids"], crowded["nodes"]
    top = node.copy()
    for i in np.nonzero(top > 0)[0]:
        while nodes[top[i]]["parent"] != 0:
            top[i] = nodes[top[i]]["parent"]
    on_surface = 0
    for v in np.unique(top[top > 0]):
        sel = np.nonzero(top == v)[0]
        R, t = np.asarray(nodes[v]["R"]), np.asarray(nodes[v]["t"])
        p = (np.stack([tr["x"][sel], tr["y"][sel], tr["z"][sel]], axis=1) - t) @ R
        code = oracle.Solid.from_spec(solids[nodes[v]["solid"]]).query(
            x=p[:, 0], y=p[:, 1], z=p[:, 2], want=("inside",))["inside"]
        on_surface += int((code == 1).sum())
    assert 0.2 * n < on_surface <= 0.31 * n
