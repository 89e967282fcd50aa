"""Parity of the binary64 CUDA query pass with the CPU oracle (through the C ABI).

Codes bit-exact, distances and safeties within 1e-9 mm, sentinels exact; seeded
inputs from the workload recipes at sizes that span many blocks plus a ragged
tail, the full 2^20-track tube and cone baskets, sampled 2^24-track baskets, and
edge cases (empty basket, one track, skipped queries, axis-parallel directions,
points on faces, edges and corners, the grazing-ray families, the cone apex).
"""

import numpy as np
import pytest

import oracle
import workloads as W
from tests.helpers import compare, to_device, to_host

pytestmark = pytest.mark.gpu

SPECS = {"box": W.BOX_M1, "trd": W.TRD_M3, "tube": W.TUBE_M2, "cone": W.CONE_M2,
         "polycone": W.polycone_m3()}
TABLE = W.solid_table(24, seed=11)


@pytest.fixture(scope="module")
def gv():
    import torch  # noqa: F401
    import paper_1512_06637_gb300 as gv
    from paper_1512_06637_gb300 import build
    build.build()
    return gv


def run_both(gv, spec, tr, precision="fp64", ws=None):
    import torch
    s = gv.Solid.from_spec(spec)
    dev = to_device(tr, torch)
    out = gv.query(s, dev, precision=precision, workspace=ws)
    torch.cuda.synchronize()
    want = oracle.Solid.from_spec(spec).query(**tr)
    return to_host(out), want


@pytest.mark.parametrize("name", list(SPECS))
def test_fp64_parity_named(gv, name):
    spec = SPECS[name]
    tr = W.tracks_for_solid(spec, (1 << 17) + 37, seed=500 + len(name))
    got, want = run_both(gv, spec, tr)
    compare(got, want, "fp64", name)


@pytest.mark.parametrize("i", range(len(TABLE)))
def test_fp64_parity_random_solids(gv, i):
    spec = TABLE[i]
    tr = W.tracks_for_solid(spec, 20011, seed=600 + i)
    got, want = run_both(gv, spec, tr)
    compare(got, want, "fp64", f"{spec['kind']}#{i}")


def test_fp64_box1024(gv):
    tr = W.box1024()
    got, want = run_both(gv, W.BOX_M1, tr)
    compare(got, want, "fp64", "box1024")


@pytest.mark.parametrize("name", ["tube", "cone"])
def test_fp64_full_1m(gv, name):
    tr = W.tracks_for_solid(SPECS[name], 1 << 20, seed=1)
    got, want = run_both(gv, SPECS[name], tr)
    compare(got, want, "fp64", name + "-1M")


def test_fp64_sampled_16m(gv):
    """2^24 tracks per solid on the GPU; the oracle checks a seeded sample."""
    import torch
    for name in ("box", "trd", "tube", "cone", "polycone"):
        spec = SPECS[name]
        tr = W.tracks_for_solid(spec, 1 << 24, seed=2)
        s = gv.Solid.from_spec(spec)
        out = gv.query(s, to_device(tr, torch), precision="fp64")
        torch.cuda.synchronize()
        g = np.random.default_rng(3)
        idx = np.sort(g.choice(1 << 24, 50000, replace=False))
        sub = {k: v[idx] for k, v in tr.items()}
        want = oracle.Solid.from_spec(spec).query(**sub)
        got = {k: v.cpu().numpy()[idx] for k, v in out.items()}
        compare(got, want, "fp64", name + "-16M-sample")


def test_fp64_empty_and_single(gv):
    import torch
    s = gv.Solid.from_spec(W.TUBE_M2)
    empty = {k: torch.empty(0, dtype=torch.float64, device="cuda") for k in ("x", "y", "z", "dx", "dy", "dz")}
    out = gv.query(s, empty)
    torch.cuda.synchronize()
    assert all(v.numel() == 0 for v in out.values())
    tr = W.tracks_for_solid(W.TUBE_M2, 1, seed=9)
    got, want = run_both(gv, W.TUBE_M2, tr)
    compare(got, want, "fp64", "single")


def test_fp64_skipped_queries(gv):
    import torch
    spec = SPECS["polycone"]
    tr = W.tracks_for_solid(spec, 3000, seed=12)
    s = gv.Solid.from_spec(spec)
    dev = to_device(tr, torch)
    want = oracle.Solid.from_spec(spec).query(**tr)
    for subset in (("inside",), ("dist_out",), ("safety_in", "safety_out"), ("dist_in", "inside")):
        out = gv.query(s, dev, want=subset)
        torch.cuda.synchronize()
        got = to_host(out)
        assert sorted(got) == sorted(subset)
        compare(got, want, "fp64", f"subset{subset}")


def _edge_tracks():
    """Points on faces / edges / corners of the box (10,20,30) with axis-parallel
    and diagonal directions (components exactly zero)."""
    D = np.array([10.0, 20.0, 30.0])
    pts, dirs = [], []
    axes = [np.array(v, float) for v in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]
    diag = [np.array(v, float) / np.linalg.norm(v) for v in ((1, 1, 0), (1, -1, 0), (0, 1, 1), (1, 1, 1), (-1, 1, -1))]
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                for scale in (1.0, 0.5, 1.5):
                    p = np.array([sx, sy, sz], float) * D * scale
                    for d in axes + diag:
                        pts.append(p); dirs.append(d)
    return W.soa(np.array(pts), np.array(dirs))


def test_fp64_box_edges_corners(gv):
    """On faces, edges and corners, with axis-parallel and diagonal directions (exact zero
    components): the readings for rays along a face and through an edge fix every answer,
    so the library matches the oracle exactly."""
    tr = _edge_tracks()
    got, want = run_both(gv, W.BOX_M1, tr)
    compare(got, want, "fp64", "box-edges")


@pytest.mark.parametrize("fam", W.GRAZING_FAMILIES)
def test_fp64_grazing(gv, fam):
    """Rays tangent to a wall, along a cone generator, along a phi plane or a face, through
    or touching an edge, touching a wall: exact parity with the oracle at 1e-9 mm."""
    spec, tr, _ = W.grazing_tracks(fam, 4000, 700 + W.GRAZING_FAMILIES.index(fam))
    got, want = run_both(gv, spec, tr)
    compare(got, want, "fp64", fam)


def test_fp64_cone_axis_apex(gv):
    """Rays along the cone axis, through the apex of its inner surface at z = -40."""
    g = np.random.default_rng(21)
    n = 4000
    z0 = g.uniform(-60, 60, n)
    p = np.stack([np.zeros(n), np.zeros(n), z0], 1)
    d = np.stack([np.zeros(n), np.zeros(n), np.where(g.random(n) < 0.5, 1.0, -1.0)], 1)
    got, want = run_both(gv, W.CONE_M2, W.soa(p, d))
    compare(got, want, "fp64", "cone-axis")

@pytest.mark.parametrize("i", range(len(W.degenerate_table())))
def test_fp64_degenerate_solids(gv, i):
    """Solids at the edges of their parameter ranges (32 planes, phi wedges of 1e-3 rad, exactly
    pi and just below 2 pi, a 1e-6 mm wall, apex cones, 1e-3 mm and 1e4 mm solids, a 60-degree trap)."""
    spec = W.degenerate_table()[i]
    tr = W.tracks_for_solid(spec, 20011, seed=800 + i)
    got, want = run_both(gv, spec, tr)
    compare(got, want, "fp64", f"degenerate {spec['kind']}#{i}")


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["box", "trd", "trap", "tube", "cone", "polycone"])
def test_fp64_class_order_same_bits(gv, kind):
    """A basket large enough to give every SM a tile is evaluated in tiles ordered by work class;
    the per-track arithmetic is unchanged, so every output equals the index-order pass (the same
    tracks queried in small chunks) bit for bit (ragged basket: a partial last tile), and a
    sample is held to the oracle."""
    import torch
    spec = next(sp for sp in TABLE if sp["kind"] == "trap") if kind == "trap" else SPECS[kind]
    n = (1 << 19) + 123
    tr = W.tracks_for_solid(spec, n, seed=31)
    dev = to_device(tr, torch)
    s = gv.Solid.from_spec(spec)
    tiled = to_host(gv.query(s, dev, precision="fp64"))
    chunk = 1 << 15
    parts = []
    for o in range(0, n, chunk):
        sub = {k: v[o:o + chunk].contiguous() for k, v in dev.items()}
        parts.append(to_host(gv.query(s, sub, precision="fp64")))
    torch.cuda.synchronize()
    for k in tiled:
        plain = np.concatenate([p[k] for p in parts])
        assert np.array_equal(plain.view(np.uint8), tiled[k].view(np.uint8)), (kind, k)
    idx = np.arange(0, n, 97)
    sub = {k: v[idx] for k, v in tr.items()}
    want = oracle.Solid.from_spec(spec).query(**sub)
    compare({k: v[idx] for k, v in tiled.items()}, want, "fp64", f"tiled-{kind}")


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["box", "polycone"])
@pytest.mark.parametrize("want", [("inside", "safety_in", "safety_out"), ("dist_in",), ("inside", "dist_out")])
def test_fp64_class_order_subsets(gv, kind, want):
    """Subsets of the queries through the work-class tiles (no directions: the classes come from
    the point alone) give the same bits as the index-order pass over small chunks."""
    import torch
    spec = SPECS[kind]
    n = (1 << 19) + 7
    tr = W.tracks_for_solid(spec, n, seed=41)
    dev = to_device(tr, torch)
    if "dist_in" not in want and "dist_out" not in want:
        for k in ("dx", "dy", "dz"):
            dev[k] = None
    s = gv.Solid.from_spec(spec)
    tiled = to_host(gv.query(s, dev, precision="fp64", want=want))
    chunk = 1 << 15
    parts = []
    for o in range(0, n, chunk):
        sub = {k: (None if v is None else v[o:o + chunk].contiguous()) for k, v in dev.items()}
        parts.append(to_host(gv.query(s, sub, precision="fp64", want=want)))
    torch.cuda.synchronize()
    for k in want:
        plain = np.concatenate([p[k] for p in parts])
        assert np.array_equal(plain.view(np.uint8), tiled[k].view(np.uint8)), (kind, want, k)


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["box", "polycone"])
def test_fp64_class_order_large_tiles(gv, kind):
    """Baskets large enough for the 2048-track tiles (four per resident block) give the same bits
    as the index-order pass over small chunks."""
    import torch
    spec = SPECS[kind]
    n = (1 << 21) + (1 << 19) + 5
    tr = W.tracks_for_solid(spec, n, seed=43)
    dev = to_device(tr, torch)
    s = gv.Solid.from_spec(spec)
    tiled = to_host(gv.query(s, dev, precision="fp64"))
    chunk = 1 << 16
    parts = []
    for o in range(0, n, chunk):
        sub = {k: v[o:o + chunk].contiguous() for k, v in dev.items()}
        parts.append(to_host(gv.query(s, sub, precision="fp64")))
    torch.cuda.synchronize()
    for k in tiled:
        plain = np.concatenate([p[k] for p in parts])
        assert np.array_equal(plain.view(np.uint8), tiled[k].view(np.uint8)), (kind, k)
