"""Parity of the FP32 bulk pass + FP64 refinement with the CPU oracle (C ABI).

Codes bit-exact, distances and safeties within 1e-5 relative (1e-9 mm below
1e-4 mm), sentinels exact; the same inputs as the FP64 parity tests, the full
2^20-track tube and cone baskets, sampled 2^24-track baskets, edge cases, and
the refined fraction reported per solid.
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


def run32(gv, spec, tr):
    import torch
    s = gv.Solid.from_spec(spec)
    dev = to_device(tr, torch)
    ws = gv.Workspace(len(tr["x"]))
    out = gv.query(s, dev, precision="fp32_refine", workspace=ws)
    refined = ws.refined()
    torch.cuda.synchronize()
    return to_host(out), refined


@pytest.mark.parametrize("name", list(SPECS))
def test_fp32_parity_named(gv, name):
    spec = SPECS[name]
    n = (1 << 17) + 37
    tr = W.tracks_for_solid(spec, n, seed=500 + len(name))
    got, refined = run32(gv, spec, tr)
    want = oracle.Solid.from_spec(spec).query(**tr)
    stats = compare(got, want, "fp32", name)
    frac = refined / n
    print(f"{name}: refined fraction {frac:.4f}; {stats}")
    assert frac < 0.2


@pytest.mark.parametrize("i", range(len(TABLE)))
def test_fp32_parity_random_solids(gv, i):
    spec = TABLE[i]
    tr = W.tracks_for_solid(spec, 20011, seed=600 + i)
    got, refined = run32(gv, spec, tr)
    want = oracle.Solid.from_spec(spec).query(**tr)
    compare(got, want, "fp32", f"{spec['kind']}#{i}")


def test_fp32_box1024(gv):
    tr = W.box1024()
    got, _ = run32(gv, W.BOX_M1, tr)
    want = oracle.Solid.from_spec(W.BOX_M1).query(**tr)
    compare(got, want, "fp32", "box1024")


@pytest.mark.parametrize("name", ["tube", "cone"])
def test_fp32_full_1m(gv, name):
    tr = W.tracks_for_solid(SPECS[name], 1 << 20, seed=1)
    got, refined = run32(gv, SPECS[name], tr)
    want = oracle.Solid.from_spec(SPECS[name]).query(**tr)
    compare(got, want, "fp32", name + "-1M")


def test_fp32_sampled_16m(gv):
    """2^24 tracks per solid, in the launch configuration the benchmark times; the
    oracle checks a seeded sample; codes equal the FP64 pass everywhere."""
    import torch
    for name in ("box", "trd", "tube", "cone", "polycone"):
        spec = SPECS[name]
        n = 1 << 24
        tr = W.tracks_for_solid(spec, n, seed=2)
        s = gv.Solid.from_spec(spec)
        dev = to_device(tr, torch)
        ws = gv.Workspace(n)
        out = gv.query(s, dev, precision="fp32_refine", workspace=ws)
        out64 = gv.query(s, dev, precision="fp64", want=("inside",))
        torch.cuda.synchronize()
        assert torch.equal(out["inside"], out64["inside"]), name
        g = np.random.default_rng(3)
        idx = np.sort(g.choice(n, 50000, replace=False))
        sub = {k: v[idx] for k, v in tr.items()}
        want = oracle.Solid.from_spec(spec).query(**sub)
        got = {k: v.cpu().numpy()[idx] for k, v in out.items()}
        compare(got, want, "fp32", name + "-16M-sample")
        print(name, "refined fraction", ws.refined() / n)
        del dev, out, out64


def test_fp32_empty_single_and_subsets(gv):
    import torch
    s = gv.Solid.from_spec(W.TUBE_M2)
    ws = gv.Workspace(4096)
    empty = {k: torch.empty(0, dtype=torch.float64, device="cuda") for k in ("x", "y", "z", "dx", "dy", "dz")}
    out = gv.query(s, empty, precision="fp32_refine", workspace=ws)
    torch.cuda.synchronize()
    assert all(v.numel() == 0 for v in out.values())
    assert ws.refined() == 0
    tr = W.tracks_for_solid(W.TUBE_M2, 1, seed=9)
    got, _ = run32(gv, W.TUBE_M2, tr)
    compare(got, oracle.Solid.from_spec(W.TUBE_M2).query(**tr), "fp32", "single")
    spec = SPECS["polycone"]
    tr = W.tracks_for_solid(spec, 3000, seed=12)
    want = oracle.Solid.from_spec(spec).query(**tr)
    dev = to_device(tr, torch)
    sp = gv.Solid.from_spec(spec)
    full = to_host(gv.query(sp, dev, precision="fp32_refine", workspace=ws))
    for subset in (("inside",), ("dist_out",), ("safety_in", "safety_out"), ("dist_in", "inside")):
        out = gv.query(sp, dev, precision="fp32_refine", workspace=ws, want=subset)
        torch.cuda.synchronize()
        got = to_host(out)
        compare(got, want, "fp32", f"subset{subset}")
        # subsets without distances take the one-track-per-thread pass, the others the
        # lane-refill pass.  The code is decided exactly on both; the other values may come
        # from either precision (a track flagged for its distance gets all its values from
        # binary64), so they are held to the oracle above, not to each other.
        if "inside" in subset:
            assert np.array_equal(got["inside"], full["inside"]), subset


def test_fp32_workspace_too_small(gv):
    import torch
    s = gv.Solid.from_spec(W.BOX_M1)
    ws = gv.Workspace(10)
    tr = to_device(W.box1024(), torch)
    with pytest.raises(gv.GVError) as e:
        gv.query(s, tr, precision="fp32_refine", workspace=ws)
    assert e.value.status == 3
    with pytest.raises(gv.GVError):
        gv.query(s, tr, precision="fp32_refine", workspace=None)


def test_fp32_edges_and_apex(gv):
    """Points on the box's faces, edges and corners with axis-parallel and diagonal
    directions, and rays along the cone axis through its inner apex: parity with the
    oracle (the binary32 pass flags what it cannot certify)."""
    from tests.test_gpu_parity_fp64 import _edge_tracks
    g = np.random.default_rng(21)
    n = 4000
    z0 = g.uniform(-60, 60, n)
    p = np.stack([np.zeros(n), np.zeros(n), z0], 1)
    d = np.stack([np.zeros(n), np.zeros(n), np.where(g.random(n) < 0.5, 1.0, -1.0)], 1)
    for spec, tr, label in ((W.BOX_M1, _edge_tracks(), "box-edges"), (W.CONE_M2, W.soa(p, d), "cone-axis")):
        got, _ = run32(gv, spec, tr)
        compare(got, oracle.Solid.from_spec(spec).query(**tr), "fp32", label)


@pytest.mark.parametrize("fam", W.GRAZING_FAMILIES)
def test_fp32_grazing(gv, fam):
    """The grazing-ray families through the binary32 pass and its refinement: parity with
    the oracle at the stated tolerance (such rays are flagged and refined in binary64)."""
    spec, tr, _ = W.grazing_tracks(fam, 4000, 700 + W.GRAZING_FAMILIES.index(fam))
    got, refined = run32(gv, spec, tr)
    compare(got, oracle.Solid.from_spec(spec).query(**tr), "fp32", fam)

@pytest.mark.parametrize("i", range(len(W.degenerate_table())))
def test_fp32_degenerate_solids(gv, i):
    """The degenerate solids through the binary32 pass and its refinement."""
    spec = W.degenerate_table()[i]
    tr = W.tracks_for_solid(spec, 20011, seed=800 + i)
    got, refined = run32(gv, spec, tr)
    compare(got, oracle.Solid.from_spec(spec).query(**tr), "fp32", f"degenerate {spec['kind']}#{i}")


@pytest.mark.parametrize("kind", ["box", "trd", "trap", "tube", "cone", "polycone"])
def test_fp32_small_basket_one_launch_same_bits(gv, kind):
    """Baskets of at most 65536 tracks take one launch that evaluates uncertain tracks in binary64
    on the spot: the results equal those of the two-pass form (the same tracks inside a larger
    basket) bit for bit, and the workspace reports as many tracks evaluated in binary64 as the
    two-pass form sends to its refinement (the same tracks twice over: exactly twice as many)."""
    import torch
    spec = next(sp for sp in W.solid_table(24, seed=11) if sp["kind"] == "trap") if kind == "trap" else SPECS[kind]
    # 30% of the points within 1e-9 of a surface, across the edge of the 5e-10 surface band:
    # some of them the binary32 pass cannot decide
    big = W.tracks_for_solid(spec, 1 << 17, seed=53, near_frac=0.3, band=1e-9)
    dev = to_device(big, torch)
    s = gv.Solid.from_spec(spec)
    ws = gv.Workspace(1 << 17)
    full = to_host(gv.query(s, dev, precision="fp32_refine", workspace=ws))
    for m in (1, 37, 4096, 40000, 65536):
        sub = {k: v[:m].contiguous() for k, v in dev.items()}
        small = to_host(gv.query(s, sub, precision="fp32_refine", workspace=ws))
        r1 = ws.refined()
        torch.cuda.synchronize()
        for k in small:
            assert np.array_equal(small[k].view(np.uint8), full[k][:m].view(np.uint8)), (kind, m, k)
        twice = {k: torch.cat([v, v]).contiguous() for k, v in sub.items()}
        gv.query(s, twice, precision="fp32_refine", workspace=ws)
        assert ws.refined() == 2 * r1, (kind, m)
        if m == 4096:
            assert r1 > 0, kind
