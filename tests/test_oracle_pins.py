"""Pins of the CPU oracle against what the mathematics fixes.

The paper (VecGeom section) asks three questions of every solid: is the point
inside, how far is the border (safety), how far can it move along its direction
(DistanceToIn / DistanceToOut).  The oracle answers them by enumerating surface
crossings; these tests check it against independent routes: textbook closed
forms (slab method, cylinder quadratic, radial rays), construction (points placed
inside / outside / on a face by design), brute-force ray marching with bisection,
invariants (a returned finite distance lands on the surface; safety never
exceeds any distance), and reductions (a trd with parallel faces is a box; a
polycone with a straight profile does not see its internal planes).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

IN, SURF, OUT = oracle.INSIDE, oracle.SURFACE, oracle.OUTSIDE
H = oracle.HALF_TOL
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

ALL_SPECS = [W.BOX_M1, W.TRD_M3, W.TUBE_M2, W.CONE_M2, W.polycone_m3()] + W.solid_table(18, seed=7)


def sol(spec):
    return oracle.Solid.from_spec(spec)


# ------------------------------------------------------------------ box

def test_box_membership_by_construction():
    D = np.array([10.0, 20.0, 30.0])
    b = oracle.Solid("box", *D)
    g = np.random.default_rng(1)
    inner = g.uniform(-1, 1, (5000, 3)) * (D - 1e-6)
    assert (b.inside(inner) == IN).all()
    outer = g.uniform(-1, 1, (5000, 3)) * D
    ax = g.integers(0, 3, 5000)
    outer[np.arange(5000), ax] = np.sign(g.uniform(-1, 1, 5000)) * (D[ax] + g.uniform(1e-6, 50, 5000))
    assert (b.inside(outer) == OUT).all()
    face = g.uniform(-1, 1, (5000, 3)) * (D - 1e-6)
    sgn = np.where(g.random(5000) < 0.5, -1.0, 1.0)
    face[np.arange(5000), ax] = sgn * D[ax]
    assert (b.inside(face) == SURF).all()
    # the band is h = 0.5e-9 mm on either side
    near_in = face.copy(); near_in[np.arange(5000), ax] -= sgn * 0.4e-9
    near_out = face.copy(); near_out[np.arange(5000), ax] += sgn * 0.4e-9
    assert (b.inside(near_in) == SURF).all() and (b.inside(near_out) == SURF).all()
    deep_in = face.copy(); deep_in[np.arange(5000), ax] -= sgn * 0.7e-9
    far_out = face.copy(); far_out[np.arange(5000), ax] += sgn * 0.7e-9
    assert (b.inside(deep_in) == IN).all() and (b.inside(far_out) == OUT).all()


def _trap_faces(params):
    """The six faces of a trap from its vertices (workloads._trap_vertices, plain numpy):
    per face its centroid and outward unit normal, the normal fitted by a singular value
    decomposition of the face's four vertices (not the library's diagonal cross product)."""
    V = W._trap_vertices(params)
    centre = V.mean(axis=0)
    quads = [(0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5)]
    out = []
    for q in quads:
        P = V[list(q)]
        c = P.mean(axis=0)
        _, sv, vt = np.linalg.svd(P - c)
        assert sv[-1] < 1e-9 * max(1.0, sv[0])  # planar
        n = vt[-1]
        if np.dot(n, c - centre) < 0:
            n = -n
        out.append((c, n))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_trap_membership_by_construction(seed):
    """Random traps (tilted axis, sheared faces, unequal half-lengths): points at each face's
    centroid moved along the face's own normal by -0.7e-9 (INSIDE), +/-0.4e-9 (SURFACE) and
    +0.7e-9 mm (OUTSIDE); the face centroid moved 1 mm inward is INSIDE with SafetyToOut 1 for
    a face nearer than every other."""
    g = np.random.default_rng(70 + seed)
    for j in range(8):
        spec = W.trap_random(g)
        if j % 2:  # the axis at any azimuth, tilted up to 30 deg
            p = list(spec["params"][0])
            p[1], p[2] = g.uniform(0, 30) * W.DEG, g.uniform(0, 360) * W.DEG
            spec = {"kind": "trap", "params": (tuple(p),)}
        params = spec["params"][0]
        s = sol(spec)
        faces = _trap_faces(params)
        for c, n in faces:
            pts = np.array([c - 0.7e-9 * n, c - 0.4e-9 * n, c + 0.4e-9 * n, c + 0.7e-9 * n])
            assert list(s.inside(pts)) == [IN, SURF, SURF, OUT], (params, c, n)
        # unit step inward from the face with the largest inscribed distance at its centroid
        for c, n in faces:
            q = c - 1.0 * n
            others = [np.dot(q - c2, n2) for c2, n2 in faces]
            if max(others) < -1.0 + 1e-9 and sorted(others)[-2] < -1.0 - 1e-6:
                r = s.query([q[0]], [q[1]], [q[2]], [0.0], [0.0], [1.0], want=("inside", "safety_out"))
                assert r["inside"][0] == IN and r["safety_out"][0] == pytest.approx(1.0, abs=1e-9)


def _slab(D, p, d):
    """Textbook slab method for an axis-aligned box (Kay-Kajiya), per track."""
    tn, tf = -np.inf, np.inf
    for i in range(3):
        if d[i] == 0.0:
            if abs(p[i]) > D[i]:
                return np.inf, -np.inf
            continue
        a, b = (-D[i] - p[i]) / d[i], (D[i] - p[i]) / d[i]
        tn, tf = max(tn, min(a, b)), min(tf, max(a, b))
    return tn, tf


def test_box_slab_closed_form():
    D = np.array([10.0, 20.0, 30.0])
    b = oracle.Solid("box", *D)
    g = np.random.default_rng(2)
    n = 20000
    p = g.uniform(-1, 1, (n, 3)) * 2 * D
    d = W.isotropic(n, g)
    # a fifth of the directions axis-parallel or in a coordinate plane (d_i = 0)
    k = n // 5
    d[:k, g.integers(0, 3)] = 0.0
    d[:k] /= np.linalg.norm(d[:k], axis=1, keepdims=True)
    r = b.query(p[:, 0], p[:, 1], p[:, 2], d[:, 0], d[:, 1], d[:, 2])
    for i in range(n):
        tn, tf = _slab(D, p[i], d[i])
        code = r["inside"][i]
        if code == IN:
            assert r["dist_out"][i] == pytest.approx(tf, abs=1e-12)
            assert r["dist_in"][i] == -1
            assert r["safety_out"][i] == pytest.approx(np.min(D - np.abs(p[i])), abs=1e-12)
        elif code == OUT:
            want = tn if (tn < tf and tn > 0) else np.inf
            assert r["dist_in"][i] == pytest.approx(want, abs=1e-12) or (np.isinf(want) and np.isinf(r["dist_in"][i]))
            assert r["dist_out"][i] == -1
            excess = np.maximum(np.abs(p[i]) - D, 0)
            # max of the per-axis excesses: exact for one violated axis, a lower bound otherwise
            assert r["safety_in"][i] == pytest.approx(excess.max(), abs=1e-12)
            assert r["safety_in"][i] <= np.linalg.norm(excess) + 1e-12


# ------------------------------------------------------------- cylinders

def test_full_cylinder_closed_form():
    R, Z = 20.0, 30.0
    c = oracle.Solid("tube", 0.0, R, Z, 0.0, 2 * math.pi)
    g = np.random.default_rng(3)
    n = 20000
    p = g.uniform(-1, 1, (n, 3)) * [2 * R, 2 * R, 2 * Z]
    d = W.isotropic(n, g)
    r = c.query(p[:, 0], p[:, 1], p[:, 2], d[:, 0], d[:, 1], d[:, 2])
    for i in range(n):
        x, y, z = p[i]
        u, v, w = d[i]
        A, B, C = u * u + v * v, x * u + y * v, x * x + y * y - R * R
        rr = math.hypot(x, y)
        code = r["inside"][i]
        if code == IN:
            tr = (-B + math.sqrt(B * B - A * C)) / A if A > 0 else np.inf
            tz = (math.copysign(Z, w) - z) / w if w != 0 else np.inf
            assert r["dist_out"][i] == pytest.approx(min(tr, tz), rel=1e-12, abs=1e-12)
            assert r["safety_out"][i] == pytest.approx(min(R - rr, Z - abs(z)), abs=1e-12)
        elif code == OUT:
            best = np.inf
            disc = B * B - A * C
            if A > 0 and disc > 0 and C > 0:
                t = (-B - math.sqrt(disc)) / A
                if t > 0 and abs(z + t * w) <= Z:
                    best = t
            if w != 0 and abs(z) > Z:
                t = ((-Z if w > 0 else Z) - z) / w
                q = (x + t * u, y + t * v)
                if t > 0 and math.hypot(*q) <= R:
                    best = min(best, t)
            got = r["dist_in"][i]
            if np.isinf(best):
                assert np.isinf(got)
            else:
                assert got == pytest.approx(best, rel=1e-10, abs=1e-10)
            assert r["safety_in"][i] == pytest.approx(max(rr - R, abs(z) - Z), abs=1e-12)


def test_tube_radial_rays_closed_form():
    """Rays from the axis, in the xy-plane, at azimuth a: for a segment (rmin, rmax, 0..270
    deg) DistanceToIn is rmin inside the phi range and +inf outside it."""
    t = oracle.Solid("tube", 5.0, 20.0, 30.0, 0.0, 1.5 * math.pi)
    a = np.linspace(0.01, 2 * math.pi - 0.01, 721)
    d = np.stack([np.cos(a), np.sin(a), np.zeros_like(a)], 1)
    z0 = np.zeros_like(a)
    r = t.query(z0, z0, z0 + 3.0, d[:, 0], d[:, 1], d[:, 2])
    inrange = a < 1.5 * math.pi
    assert np.allclose(r["dist_in"][inrange], 5.0, atol=1e-12)
    assert np.isinf(r["dist_in"][~inrange]).all()
    # from the middle of the wall outwards, DistanceToOut is rmax - 12.5
    p = 12.5 * d
    r = t.query(p[:, 0], p[:, 1], z0, d[:, 0], d[:, 1], d[:, 2])
    assert np.allclose(r["dist_out"][inrange], 7.5, atol=1e-12)
    assert (r["inside"][~inrange] == OUT).all()


def test_cone_axis_parallel_closed_form():
    """Rays parallel to the axis inside a cone frustum: exit through the top plane or,
    where the wall closes in, through the slanted wall at R(z) = r."""
    rmax1, rmax2, dz = 25.0, 10.0, 40.0
    c = oracle.Solid("cone", 0.0, rmax1, 0.0, rmax2, dz, 0.0, 2 * math.pi)
    g = np.random.default_rng(4)
    n = 5000
    z = g.uniform(-dz + 1, dz - 1, n)
    Rz = rmax1 + (z + dz) / (2 * dz) * (rmax2 - rmax1)
    rr = g.uniform(0, 1, n) * (Rz - 1e-6)
    ph = g.uniform(0, 2 * math.pi, n)
    x, y = rr * np.cos(ph), rr * np.sin(ph)
    one, zero = np.ones(n), np.zeros(n)
    r = c.query(x, y, z, zero, zero, one)
    # wall reached where rmax1 + (z' + dz)/(2dz) (rmax2 - rmax1) = rr
    zw = (rr - rmax1) * (2 * dz) / (rmax2 - rmax1) - dz
    want = np.where(zw < dz, zw - z, dz - z)
    assert np.allclose(r["dist_out"], want, rtol=1e-10, atol=1e-10)
    r = c.query(x, y, z, zero, zero, -one)
    assert np.allclose(r["dist_out"], z + dz, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------ reductions

def _away_from_band(s):
    return (np.abs(np.abs(s) - H) > 1e-11)


def test_trd_with_parallel_faces_is_a_box():
    box = oracle.Solid("box", 10, 20, 30)
    trd = oracle.Solid("trd", 10, 10, 20, 20, 30)
    t = W.tracks_for_solid(W.BOX_M1, 20000, seed=5)
    a = box.query(**t)
    b = trd.query(**t)
    s = np.array([box.s_code([t["x"][i], t["y"][i], t["z"][i]]) for i in range(20000)])
    ok = _away_from_band(s)
    assert ok.mean() > 0.99
    assert (a["inside"][ok] == b["inside"][ok]).all()
    for k in ("dist_in", "dist_out", "safety_in", "safety_out"):
        fin = np.isfinite(a[k]) & ok
        assert np.allclose(a[k][fin], b[k][fin], rtol=0, atol=1e-12), k
        assert (np.isinf(a[k][ok]) == np.isinf(b[k][ok])).all()


def test_polycone_internal_planes_are_not_surfaces():
    """A polycone whose extra planes lie on straight segments of the profile is the
    same solid as without them: same codes, same distances; internal planes are
    never reported as surfaces."""
    z2, rn2, rx2 = [-40.0, 40.0], [5.0, 13.0], [10.0, 30.0]
    z4 = [-40.0, -10.0, 15.0, 40.0]
    lerp = lambda r, zz: r[0] + (zz + 40.0) / 80.0 * (r[1] - r[0])  # noqa: E731
    rn4 = [lerp(rn2, zz) for zz in z4]
    rx4 = [lerp(rx2, zz) for zz in z4]
    a = oracle.Solid("polycone", z2, rn2, rx2, 0.3, 4.0)
    b = oracle.Solid("polycone", z4, rn4, rx4, 0.3, 4.0)
    spec = {"kind": "polycone", "params": (tuple(z2), tuple(rn2), tuple(rx2), 0.3, 4.0)}
    t = W.tracks_for_solid(spec, 20000, seed=6)
    # and points exactly on the internal planes, well inside radially
    g = np.random.default_rng(6)
    m = 2000
    zi = np.where(g.random(m) < 0.5, -10.0, 15.0)
    rr = np.array([g.uniform(lerp(rn2, q) + 0.5, lerp(rx2, q) - 0.5) for q in zi])
    ph = 0.3 + g.uniform(0.1, 3.9, m)
    for k, v in zip("x y z".split(), (rr * np.cos(ph), rr * np.sin(ph), zi)):
        t[k] = np.concatenate([t[k], v])
    dd = W.isotropic(m, g)
    for i, k in enumerate(("dx", "dy", "dz")):
        t[k] = np.concatenate([t[k], dd[:, i]])
    ra, rb = a.query(**t), b.query(**t)
    assert (rb["inside"][-m:] == IN).all()
    s = np.array([a.s_code([t["x"][i], t["y"][i], t["z"][i]]) for i in range(len(t["x"]))])
    ok = _away_from_band(s)
    assert (ra["inside"][ok] == rb["inside"][ok]).all()
    for k in ("dist_in", "dist_out"):
        fin = np.isfinite(ra[k]) & ok
        assert np.allclose(ra[k][fin], rb[k][fin], rtol=1e-9, atol=1e-9), k


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("idx", range(len(ALL_SPECS)))
def test_returned_distance_lands_on_surface(idx):
    spec = ALL_SPECS[idx]
    s = sol(spec)
    t = W.tracks_for_solid(spec, 4000, seed=100 + idx)
    r = s.query(**t)
    P = np.stack([t["x"], t["y"], t["z"]], 1)
    D = np.stack([t["dx"], t["dy"], t["dz"]], 1)
    for k in ("dist_in", "dist_out"):
        v = r[k]
        m = np.isfinite(v) & (v > 0)
        q = P[m] + v[m, None] * D[m]
        codes = s.inside(q)
        assert (codes == SURF).all(), (spec["kind"], k, np.bincount(codes, minlength=3))
    # zero distances only from the surface, -1 only from the wrong side
    assert (r["inside"][r["dist_in"] == 0] == SURF).all()
    assert (r["inside"][r["dist_out"] == 0] == SURF).all()
    assert ((r["dist_in"] == -1) == (r["inside"] == IN)).all()
    assert ((r["dist_out"] == -1) == (r["inside"] == OUT)).all()
    assert np.isfinite(r["dist_out"]).all()
    for k in r:
        if k != "inside":
            assert not np.isnan(r[k]).any()


@pytest.mark.parametrize("idx", range(len(ALL_SPECS)))
def test_safety_is_a_lower_bound(idx):
    """0 <= safety <= every distance along any direction (here: the track's own
    direction and 64 Fibonacci directions)."""
    spec = ALL_SPECS[idx]
    s = sol(spec)
    n = 600
    t = W.tracks_for_solid(spec, n, seed=200 + idx)
    r = s.query(**t)
    k = np.arange(64) + 0.5
    th = np.arccos(1 - 2 * k / 64)
    ph = math.pi * (1 + 5 ** 0.5) * k
    fib = np.stack([np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)], 1)
    rep = lambda a: np.repeat(a, 64)  # noqa: E731
    tt = {"x": rep(t["x"]), "y": rep(t["y"]), "z": rep(t["z"]),
          "dx": np.tile(fib[:, 0], n), "dy": np.tile(fib[:, 1], n), "dz": np.tile(fib[:, 2], n)}
    rr = s.query(**tt)
    din = rr["dist_in"].reshape(n, 64)
    dout = rr["dist_out"].reshape(n, 64)
    out = r["inside"] == OUT
    ins = r["inside"] == IN
    assert (r["safety_in"][out] > H).all()
    assert (r["safety_out"][ins] > H).all()
    assert (r["safety_in"][out] <= din[out].min(axis=1) + 1e-9).all()
    assert (r["safety_in"][out] <= np.where(r["dist_in"][out] >= 0, r["dist_in"][out], np.inf) + 1e-9).all()
    assert (r["safety_out"][ins] <= dout[ins].min(axis=1) + 1e-9).all()
    assert (r["safety_out"][ins] <= r["dist_out"][ins] + 1e-9).all()


def test_safety_exact_for_full_tube_interior():
    t = oracle.Solid("tube", 5.0, 20.0, 30.0, 0.0, 2 * math.pi)
    g = np.random.default_rng(9)
    n = 5000
    rr = np.sqrt(g.uniform(26, 399, n))
    ph = g.uniform(0, 2 * math.pi, n)
    z = g.uniform(-29, 29, n)
    r = t.query(rr * np.cos(ph), rr * np.sin(ph), z, want=("safety_out",))
    want = np.minimum(np.minimum(20 - rr, rr - 5), 30 - np.abs(z))
    assert np.allclose(r["safety_out"], want, atol=1e-12)


# -------------------------------------------------------- brute force

def _march(s, P, D, want_inside, tmax, step):
    """First t > 0 at which the (coarsely sampled, then bisected) ray crosses to the
    wanted side of the solid, judged by the sign of s with no tolerance."""
    n = len(P)
    found = np.full(n, np.inf)
    lo = np.zeros(n)
    active = np.ones(n, bool)
    ts = np.arange(step, tmax + step, step)
    for tcur in ts:
        idx = np.nonzero(active)[0]
        if len(idx) == 0:
            break
        q = P[idx] + tcur * D[idx]
        v = s.s_values(q)
        hit = (v <= 0) if want_inside else (v > 0)
        hi_idx = idx[hit]
        found[hi_idx] = tcur
        active[hi_idx] = False
        lo[idx[~hit]] = tcur
    m = np.isfinite(found)
    a, b = lo[m].copy(), found[m].copy()
    Pm, Dm = P[m], D[m]
    for _ in range(50):
        mid = 0.5 * (a + b)
        v = s.s_values(Pm + mid[:, None] * Dm)
        hit = (v <= 0) if want_inside else (v > 0)
        b = np.where(hit, mid, b)
        a = np.where(hit, a, mid)
    found[m] = b
    return found


@pytest.mark.parametrize("idx", [0, 1, 2, 3, 4, 5, 7, 8, 9, 10])
def test_brute_force_ray_march(idx):
    spec = ALL_SPECS[idx]
    s = sol(spec)
    n = 300
    t = W.tracks_for_solid(spec, n, seed=300 + idx, near_frac=0.0)
    P = np.stack([t["x"], t["y"], t["z"]], 1)
    D = np.stack([t["dx"], t["dy"], t["dz"]], 1)
    r = s.query(**t)
    hb = W.bounding_half(spec)
    tmax = 2.0 * np.linalg.norm(hb * 2.0 + 1.0)
    step = float(max(hb.min() / 200.0, 0.01))
    out = r["inside"] == OUT
    ins = r["inside"] == IN
    te = _march(s, P[out], D[out], True, tmax, step)
    tx = _march(s, P[ins], D[ins], False, tmax, step)
    got_e, got_x = r["dist_in"][out], r["dist_out"][ins]
    # the oracle is never later than the march (a thin chord can hide from the march)
    fin = np.isfinite(te)
    assert (got_e[fin] <= te[fin] + 1e-9).all()
    with np.errstate(invalid="ignore"):
        agree_e = np.where(fin, np.abs(got_e - te) <= 1e-9, np.isinf(got_e))
    agree_x = np.abs(got_x - tx) <= 1e-9
    assert agree_e.mean() >= 0.985, agree_e.mean()
    assert agree_x.mean() >= 0.985, agree_x.mean()


DEGEN = W.degenerate_table()


@pytest.mark.parametrize("idx", [0, 1, 3, 7, 8, 11])
def test_degenerate_solids_brute_force(idx):
    """Solids at the edges of their parameter ranges (32 planes with walls pinching to the axis,
    phi wedges of 1e-3 rad, exactly pi and just below 2 pi, apex cones, a 60-degree trap):
    ray marching with bisection on the tolerance-free s agrees with the distances."""
    spec = DEGEN[idx]
    s = sol(spec)
    n = 300
    t = W.tracks_for_solid(spec, n, seed=900 + idx, near_frac=0.0)
    P = np.stack([t["x"], t["y"], t["z"]], 1)
    D = np.stack([t["dx"], t["dy"], t["dz"]], 1)
    r = s.query(**t)
    hb = W.bounding_half(spec)
    tmax = 2.0 * np.linalg.norm(hb * 2.0 + 1.0)
    step = float(max(hb.min() / 400.0, 0.002))
    out, ins = r["inside"] == OUT, r["inside"] == IN
    te = _march(s, P[out], D[out], True, tmax, step)
    tx = _march(s, P[ins], D[ins], False, tmax, step)
    got_e, got_x = r["dist_in"][out], r["dist_out"][ins]
    fin = np.isfinite(te)
    assert (got_e[fin] <= te[fin] + 1e-9).all()
    with np.errstate(invalid="ignore"):
        agree_e = np.where(fin, np.abs(got_e - te) <= 1e-9, np.isinf(got_e))
    agree_x = np.abs(got_x - tx) <= 1e-9
    assert agree_e.mean() >= 0.97, agree_e.mean()
    assert agree_x.mean() >= 0.97, agree_x.mean()


def test_degenerate_thin_wedge_march():
    """A tube segment 1e-3 rad wide: chords across it are about 0.01 mm, so the march steps
    0.002 mm (on fewer rays); it agrees with the distances."""
    spec = DEGEN[2]
    s = sol(spec)
    t = W.tracks_for_solid(spec, 60, seed=902, near_frac=0.0)
    P = np.stack([t["x"], t["y"], t["z"]], 1)
    D = np.stack([t["dx"], t["dy"], t["dz"]], 1)
    r = s.query(**t)
    out, ins = r["inside"] == OUT, r["inside"] == IN
    te = _march(s, P[out], D[out], True, 130.0, 0.002)
    tx = _march(s, P[ins], D[ins], False, 130.0, 0.002)
    fin = np.isfinite(te)
    with np.errstate(invalid="ignore"):
        agree_e = np.where(fin, np.abs(r["dist_in"][out] - te) <= 1e-9, np.isinf(r["dist_in"][out]))
    assert agree_e.all(), agree_e.mean()
    assert (np.abs(r["dist_out"][ins] - tx) <= 1e-9).all()


def test_degenerate_sliver_exit():
    """A tube segment of 2 pi - 1e-9 from phi = 1 rad: the excluded sliver lies between the
    half-planes phi = 1 - 1e-9 and phi = 1, so a ray from inside leaves at the first of: either
    half-plane (crossed at r > 0), r = 20, r = 5 (into the hole), the end planes z = +/-30."""
    spec = DEGEN[4]
    s = sol(spec)
    g = np.random.default_rng(74)
    n = 4000
    rr = g.uniform(5.5, 19.5, n)
    ph = 1.0 + g.uniform(0.01, 2 * math.pi - 0.01, n)
    z = g.uniform(-29, 29, n)
    p = np.stack([rr * np.cos(ph), rr * np.sin(ph), z], 1)
    d = W.isotropic(n, g)
    r = s.query(p[:, 0], p[:, 1], p[:, 2], d[:, 0], d[:, 1], d[:, 2])
    assert (r["inside"] == IN).all()
    edges = [np.array([math.cos(a), math.sin(a)]) for a in (1.0, 1.0 + (2 * math.pi - 1e-9))]
    for i in range(n):
        x, y, zz = p[i]
        u, v, w = d[i]
        cands = []
        A, B = u * u + v * v, x * u + y * v
        for R, hole in ((20.0, False), (5.0, True)):
            C = x * x + y * y - R * R
            disc = B * B - A * C
            if A > 0 and disc > 0:
                t1, t2 = (-B - math.sqrt(disc)) / A, (-B + math.sqrt(disc)) / A
                cands.append(t1 if hole else t2)  # into the hole at its first root, out of r = 20 at the second
        if w != 0:
            cands.append(((30.0 if w > 0 else -30.0) - zz) / w)
        for e in edges:  # crossing of the line through the axis along e, on e's side
            den = e[1] * u - e[0] * v
            if den != 0:
                t = -(e[1] * x - e[0] * y) / den
                qx, qy = x + t * u, y + t * v
                if t > 0 and qx * e[0] + qy * e[1] > 0:
                    cands.append(t)
        want = min(c for c in cands if c > 0)
        assert r["dist_out"][i] == pytest.approx(want, rel=1e-9, abs=1e-9), (i, r["dist_out"][i], want)


@pytest.mark.parametrize("idx", [9, 10])
def test_degenerate_boxes_slab(idx):
    """A box 1e-3 mm wide and one 5000 x 1 x 5000 mm: the slab method."""
    D = np.array(DEGEN[idx]["params"])
    b = sol(DEGEN[idx])
    g = np.random.default_rng(60 + idx)
    n = 5000
    p = g.uniform(-1, 1, (n, 3)) * 2 * D
    d = W.isotropic(n, g)
    r = b.query(p[:, 0], p[:, 1], p[:, 2], d[:, 0], d[:, 1], d[:, 2])
    for i in range(n):
        tn, tf = _slab(D, p[i], d[i])
        if r["inside"][i] == IN:
            assert r["dist_out"][i] == pytest.approx(tf, rel=1e-12, abs=1e-12)
        elif r["inside"][i] == OUT:
            want = tn if (tf - tn > 1e-12 and tn > 0) else np.inf
            got = r["dist_in"][i]
            assert (np.isinf(want) and np.isinf(got)) or got == pytest.approx(want, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("idx", [5, 6])
def test_degenerate_tubes_closed_form(idx):
    """A shell 1e-6 mm thick at r = 10 and a cylinder 3 mm wide and 10 m long (full phi): the
    first crossing of r = rmax (from outside) or r = rmin (from the hole) or of the end planes,
    from the cylinder quadratic."""
    rmin, rmax, dz = DEGEN[idx]["params"][:3]
    c = sol(DEGEN[idx])
    g = np.random.default_rng(70 + idx)
    n = 5000
    zr = min(2 * dz, 100.0)
    p = np.stack([g.uniform(-2, 2, n) * rmax, g.uniform(-2, 2, n) * rmax, g.uniform(-1, 1, n) * zr], 1)
    d = W.isotropic(n, g)
    r = c.query(p[:, 0], p[:, 1], p[:, 2], d[:, 0], d[:, 1], d[:, 2])

    def roots(R, x, y, u, v):
        A, B, C = u * u + v * v, x * u + y * v, x * x + y * y - R * R
        disc = B * B - A * C
        if A == 0 or disc <= 0:
            return None
        sq = math.sqrt(disc)
        return (-B - sq) / A, (-B + sq) / A

    checked = 0
    for i in range(n):
        if r["inside"][i] != OUT:
            continue
        x, y, z = p[i]
        u, v, w = d[i]
        rr = math.hypot(x, y)
        if abs(z) >= dz or abs(rr - rmax) < 1e-3 or abs(rr - rmin) < 1e-3:
            continue  # entries through the end planes and near-surface starts: other pins
        if rr > rmax:
            q = roots(rmax, x, y, u, v)
            want = q[0] if q is not None and q[0] > 0 else np.inf
        else:  # in the hole
            q = roots(rmin, x, y, u, v)
            want = q[1]
        if np.isfinite(want) and abs(z + want * w) >= dz:
            continue
        got = r["dist_in"][i]
        assert (np.isinf(want) and np.isinf(got)) or got == pytest.approx(want, rel=1e-9, abs=1e-9), (i, got, want)
        checked += 1
    assert checked > 500


# ------------------------------------------------------------ grazing rays
#
# Rays that touch a surface, run along it, or pass exactly through an edge (the VecGeom
# section's third question for the rays where it is hardest).  Each family is placed by
# construction (workloads.grazing_tracks) and the answers are closed forms:
#   * a ray tangent to a convex wall leaves it, to a concave wall enters the solid;
#   * a ray running along a surface (a plane, a phi plane, a cone generator) stays on
#     the boundary, which is not the interior: DistanceToOut 0 from the surface, and no
#     entry through that surface;
#   * a ray that touches an edge or a wall (a double root) does not enter.

def _gq(fam, n, seed):
    spec, tr, m = W.grazing_tracks(fam, n, seed)
    return oracle.Solid.from_spec(spec).query(**tr), m


def test_tangent_to_convex_wall_leaves():
    """Tube (5, 20, 30, phi 0-270 deg), points on r = 20 (and within the band), directions
    tangent to the wall: the ray is outside r = 20 for every t > 0."""
    r, m = _gq("tube_outer_tangent", 3000, 31)
    assert (r["inside"] == SURF).all()
    assert (r["dist_out"] == 0).all()
    assert (np.isinf(r["dist_in"]) & (r["dist_in"] > 0)).all()
    assert (r["safety_in"] == 0).all() and (r["safety_out"] == 0).all()


def test_tangent_to_concave_wall_enters():
    """Full tube (5, 20, 30), points on r = 5, tangent directions d = (c t, w): the ray goes
    into the wall at once and leaves through r = 20 after sqrt(20^2 - 5^2) / c."""
    r, m = _gq("tube_inner_tangent", 3000, 32)
    assert (r["inside"] == SURF).all()
    assert (r["dist_in"] == 0).all()
    want = math.sqrt(20.0 ** 2 - 5.0 ** 2) / m["c"]
    assert np.abs(r["dist_out"] - want).max() <= 1e-9


@pytest.mark.parametrize("fam", ["cone_outer_generator", "cone_inner_generator"])
def test_ray_along_cone_generator(fam):
    """Cone (0, 10, 5, 25, 40): points on the outer (inner) wall, directions along the
    wall's straight generator up or down: the ray stays on the boundary to the end plane
    and leaves there, so it never gets into the interior."""
    r, m = _gq(fam, 3000, 33)
    assert (r["inside"] == SURF).all()
    assert (r["dist_out"] == 0).all()
    assert (np.isinf(r["dist_in"]) & (r["dist_in"] > 0)).all()


def test_ray_along_phi_plane():
    """Tube (5, 20, 30, phi 0-270 deg), rays in the plane of the phi = 0 or phi = 270 deg face,
    directions radial (+/-) with a small z part (xy length c):
      on the face:          DistanceToOut 0; toward the axis the ray crosses the hole and
                            enters at r = 5 on the opposite half-plane, (r0 + 5) / c away
                            (phi + 180 deg is inside the segment), else no entry;
      beyond rmax on it:    the same entry toward the axis, none away from it;
      on the opposite half-plane (inside the solid): leaves at r = 5 or r = 20."""
    r, m = _gq("phi_face_slide", 3000, 34)
    k, r0, c, sg = m["kind"], m["r0"], m["c"], m["sign"]
    toward = sg < 0
    assert (r["inside"] == np.where(k == 0, SURF, np.where(k == 1, OUT, IN))).all()
    on = k < 2
    want_in = np.where(toward, (r0 + 5.0) / c, np.inf)
    got = r["dist_in"][on]
    fin = np.isfinite(want_in[on])
    assert (np.isinf(got[~fin]) & (got[~fin] > 0)).all()
    assert np.abs(got[fin] - want_in[on][fin]).max() <= 1e-9
    assert (r["dist_out"][k == 0] == 0).all()
    want_out = np.where(toward, (r0 - 5.0) / c, (20.0 - r0) / c)[k == 2]
    assert np.abs(r["dist_out"][k == 2] - want_out).max() <= 1e-9


def test_box_edge_touch_and_crossing():
    """Box (10, 20, 30): rays through an edge point E at t0; a ray that arrives from
    beyond one face and leaves beyond the adjacent one only touches (no entry), a ray
    that arrives from beyond both faces enters at E."""
    r, m = _gq("box_edge_touch", 3000, 35)
    assert (r["inside"] == OUT).all()
    touch = m["kind"] == 0
    assert (np.isinf(r["dist_in"][touch]) & (r["dist_in"][touch] > 0)).all()
    assert np.abs(r["dist_in"][~touch] - m["t0"][~touch]).max() <= 1e-9


def test_box_face_slide():
    """Box (10, 20, 30): rays in the plane of a face (the normal component exactly zero),
    from the face (SURFACE: DistanceToOut 0, no entry) or from beyond its edge toward it
    (the ray only runs along the face: no entry)."""
    r, m = _gq("box_face_slide", 2000, 36)
    on = m["kind"] == 0
    assert (r["inside"][on] == SURF).all() and (r["inside"][~on] == OUT).all()
    assert (r["dist_out"][on] == 0).all()
    assert (np.isinf(r["dist_in"]) & (r["dist_in"] > 0)).all()


def test_wall_touch_is_not_a_crossing():
    """Full tube (5, 20, 30): a ray from inside the wall touching the hole r = 5 at t0 stays
    in the solid and leaves through r = 20 at t0 + sqrt(20^2 - 5^2); a ray from outside
    touching r = 20 never enters."""
    r, m = _gq("hole_touch", 3000, 37)
    assert (r["inside"] == IN).all()
    want = m["t0"] + math.sqrt(20.0 ** 2 - 5.0 ** 2)
    assert np.abs(r["dist_out"] - want).max() <= 1e-9
    r, m = _gq("outer_touch", 3000, 38)
    assert (r["inside"] == OUT).all()
    assert (np.isinf(r["dist_in"]) & (r["dist_in"] > 0)).all()


def test_end_plane_slide():
    """Full tube (5, 20, 30): rays in the plane z = +/-30, from the end face (SURFACE:
    DistanceToOut 0) or from beyond rmax toward the axis: they only run over the face."""
    r, m = _gq("z_face_slide", 2000, 39)
    out = m["out"]
    assert (r["inside"][~out] == SURF).all() and (r["inside"][out] == OUT).all()
    assert (r["dist_out"][~out] == 0).all()
    assert (np.isinf(r["dist_in"]) & (r["dist_in"] > 0)).all()


# ------------------------------------------------------------- golden

def test_golden_analytic_cases():
    with open(os.path.join(GOLDEN, "analytic_cases.json")) as f:
        cases = json.load(f)["cases"]
    assert len(cases) >= 20
    for c in cases:
        s = oracle.Solid(c["kind"], *c["params"])
        p, d = c["p"], c["d"]
        r = s.query([p[0]], [p[1]], [p[2]], [d[0]], [d[1]], [d[2]])
        for k, v in c["expect"].items():
            got = r[k][0]
            want = eval(str(v), {"__builtins__": {}}, {"sqrt": math.sqrt, "inf": math.inf, "atan": math.atan})
            if math.isinf(want):
                assert np.isinf(got) and got > 0, (c["name"], k, got)
            else:
                assert got == pytest.approx(want, abs=1e-12), (c["name"], k, got, want)


# ------------------------------------------------------------ navigation

def _nested():
    g = W.nested_geometry()
    return g, oracle.Geometry(g["solids"], g["nodes"])


def test_locate_by_construction():
    g, geo = _nested()
    nodes = g["nodes"]
    # cell centres are in their cell; shell mid-radius points between cells are in the shell
    cell_ids = [i for i, nd in enumerate(nodes) if nd["solid"] == 1]
    c = np.array([nodes[i]["t"] for i in cell_ids])
    assert (geo.locate(c[:, 0], c[:, 1], c[:, 2]) == np.array(cell_ids)).all()
    shells = [i for i, nd in enumerate(nodes) if nd["parent"] == 0]
    rmid = np.array([g["solids"][nodes[i]["solid"]]["params"][0] + 9.0 for i in shells])
    z = np.zeros_like(rmid)
    assert (geo.locate(rmid, z, z) == np.array(shells)).all()       # phi = 0: between cells
    assert (geo.locate(rmid * 0 + 9.5, z, z) == 0).all()           # gap inside the first shell
    assert (geo.locate(np.array([300.0, 0.0]), np.array([0.0, 0.0]), np.array([0.0, 600.0])) == -1).all()


def test_nav_step_radial_closed_form():
    """A track in a shell at azimuth 0 (between cells) moving radially outwards leaves
    through the shell's outer wall: step = rmax - r, next = -1; safety = min(distance
    to the walls, distance to the nearest cell)."""
    g, geo = _nested()
    nodes = g["nodes"]
    shells = [i for i, nd in enumerate(nodes) if nd["parent"] == 0]
    n = len(shells)
    rmin = np.array([g["solids"][nodes[i]["solid"]]["params"][0] for i in shells])
    r0 = rmin + 2.0
    z = np.full(n, 7.0)
    one, zero = np.ones(n), np.zeros(n)
    res = geo.nav_step(r0, zero, z, one, zero, zero, np.array(shells, np.int32))
    assert np.allclose(res["step"], rmin + 18.0 - r0, atol=1e-12)
    assert (res["next"] == -1).all()
    assert (res["safety"] >= 0).all() and (res["safety"] <= 2.0 + 1e-12).all()


def test_nav_step_brute_force_tree():
    """The navigation step equals the minimum over the mother's exit and every daughter's
    entry, computed here with explicit frame changes and the per-solid queries."""
    g, geo = _nested()
    nodes = g["nodes"]
    t = W.nested_tracks(3000, seed=1, geom=g)
    node = geo.locate(t["x"], t["y"], t["z"])
    keep = node >= 0
    for k in t:
        t[k] = t[k][keep]
    node = node[keep]
    res = geo.nav_step(t["x"], t["y"], t["z"], t["dx"], t["dy"], t["dz"], node)
    solids = [oracle.Solid.from_spec(s) for s in g["solids"]]
    # global placement by explicit composition along the parent chain
    Rg, tg = [], []
    for i, nd in enumerate(nodes):
        R, tt = np.asarray(nd["R"], float), np.asarray(nd["t"], float)
        if nd["parent"] >= 0:
            R, tt = Rg[nd["parent"]] @ R, Rg[nd["parent"]] @ tt + tg[nd["parent"]]
        Rg.append(R); tg.append(tt)
    P = np.stack([t["x"], t["y"], t["z"]], 1)
    D = np.stack([t["dx"], t["dy"], t["dz"]], 1)
    for i in range(0, len(node), 7):
        v = node[i]
        pl, dl = Rg[v].T @ (P[i] - tg[v]), Rg[v].T @ D[i]
        rm = solids[nodes[v]["solid"]].query([pl[0]], [pl[1]], [pl[2]], [dl[0]], [dl[1]], [dl[2]])
        cands = [(rm["dist_out"][0], -1)]
        saf = [rm["safety_out"][0]]
        for c in range(len(nodes)):
            if nodes[c]["parent"] != v:
                continue
            pc, dc = Rg[c].T @ (P[i] - tg[c]), Rg[c].T @ D[i]
            rc = solids[nodes[c]["solid"]].query([pc[0]], [pc[1]], [pc[2]], [dc[0]], [dc[1]], [dc[2]])
            if rc["dist_in"][0] >= 0:
                cands.append((rc["dist_in"][0], c))
            if rc["safety_in"][0] >= 0:
                saf.append(rc["safety_in"][0])
        best = min(cands, key=lambda tc: (tc[0], 0 if tc[1] >= 0 else 1, tc[1]))
        assert res["step"][i] == pytest.approx(best[0], abs=1e-9)
        assert res["next"][i] == best[1]
        assert res["safety"][i] == pytest.approx(min(saf), abs=1e-9)


def test_nav_tie_rules():
    """Equal distances: a daughter wins over the mother, and the lowest daughter index
    wins among daughters (world box of half 10; daughters touching its +x face)."""
    solids = [{"kind": "box", "params": (10.0, 10.0, 10.0)}, {"kind": "box", "params": (10.0, 10.0, 10.0)},
              {"kind": "box", "params": (2.0, 2.0, 2.0)}]
    eye = np.eye(3)
    nodes = [{"solid": 0, "parent": -1, "R": eye, "t": np.zeros(3)},
             {"solid": 1, "parent": 0, "R": eye, "t": np.array([20.0, 0, 0])},   # entered at x = 10
             {"solid": 2, "parent": 0, "R": eye, "t": np.array([0.0, 6.0, 0])},  # entered at y = 4
             {"solid": 2, "parent": 0, "R": eye, "t": np.array([0.0, 6.0, 0])}]  # same as node 2
    geo = oracle.Geometry(solids, nodes)
    one, zero = np.ones(1), np.zeros(1)
    r = geo.nav_step(zero, zero, zero, one, zero, zero, np.zeros(1, np.int32))
    assert r["step"][0] == 10.0 and r["next"][0] == 1          # daughter beats the mother at 10
    r = geo.nav_step(zero, zero, zero, zero, one, zero, np.zeros(1, np.int32))
    assert r["step"][0] == 4.0 and r["next"][0] == 2           # lower index among equal daughters
    r = geo.nav_step(zero, zero, zero, zero, -one, zero, np.zeros(1, np.int32))
    assert r["step"][0] == 10.0 and r["next"][0] == -1         # leaves through the mother


# ------------------------------------------------------------ transport loop

def _box_world(D):
    return oracle.Geometry([{"kind": "box", "params": tuple(D)}],
                           [{"solid": 0, "parent": -1, "R": np.eye(3), "t": np.zeros(3)}])


def test_transport_absorber_closed_form():
    """One box of absorber (no scatter): a track is absorbed after s = -ln(xi_1) / (n sigma)
    if that is shorter than its straight exit distance (slab method), else it escapes there."""
    D = np.array([30.0, 20.0, 10.0])
    geo = _box_world(D)
    n, kmax, sig = 600, 4, 0.05
    g = np.random.default_rng(71)
    P = g.uniform(-1, 1, (n, 3)) * D * 0.999
    d = W.isotropic(n, g)
    xi = 1.0 - g.random((n, kmax, 4))
    r = geo.transport(P[:, 0], P[:, 1], P[:, 2], d[:, 0], d[:, 1], d[:, 2], np.zeros(n, np.int32),
                      np.zeros(1, np.int32), [[0.0, sig]], xi, kmax)
    for i in range(n):
        t_exit = _slab(D, P[i], d[i])[1]
        s = -math.log(xi[i, 0, 1]) / sig
        absorbed = s < t_exit
        assert r["reason"][i] == (1 if absorbed else 0)
        assert r["steps"][i] == 1
        L = min(s, t_exit)
        assert r["path"][i] == pytest.approx(L, rel=1e-12, abs=1e-9)
        end = P[i] + L * d[i]
        assert np.allclose([r["x"][i], r["y"][i], r["z"][i]], end, rtol=0, atol=1e-9)
        assert r["last"][i] == (0 if absorbed else -1)


def test_transport_scatter_two_steps_closed_form():
    """A scatterer box with the random numbers chosen so that the first step scatters after
    exactly a mm (xi_0 = exp(-a n sigma)) and the second leaves the box: the end point is
    p + a d0 + t_exit(d1) d1 with d1 = (sin u cos v, sin u sin v, cos u), cos u = 2 xi_2 - 1,
    v = 2 pi xi_3."""
    D = np.array([40.0, 40.0, 40.0])
    geo = _box_world(D)
    n, kmax, sig, a = 300, 2, 0.2, 1.5
    g = np.random.default_rng(72)
    P = g.uniform(-1, 1, (n, 3)) * 20.0
    d0 = W.isotropic(n, g)
    xi = np.empty((n, kmax, 4))
    xi[:, 0, 0] = math.exp(-a * sig)
    xi[:, 0, 1] = 0.5
    xi[:, 0, 2:] = g.uniform(0.01, 0.99, (n, 2))
    xi[:, 1, :] = 1e-300      # second physics step: -ln(1e-300) / sig = 3454 mm, beyond the box
    r = geo.transport(P[:, 0], P[:, 1], P[:, 2], d0[:, 0], d0[:, 1], d0[:, 2], np.zeros(n, np.int32),
                      np.zeros(1, np.int32), [[sig, 0.0]], xi, kmax)
    for i in range(n):
        q = P[i] + a * d0[i]
        cu = 2.0 * xi[i, 0, 2] - 1.0
        v = 2.0 * math.pi * xi[i, 0, 3]
        su = math.sqrt(1.0 - cu * cu)
        d1 = np.array([su * math.cos(v), su * math.sin(v), cu])
        t_exit = _slab(D, q, d1)[1]
        assert r["reason"][i] == 0 and r["steps"][i] == 2
        assert r["path"][i] == pytest.approx(a + t_exit, rel=1e-12, abs=1e-9)
        assert np.allclose([r["x"][i], r["y"][i], r["z"][i]], q + t_exit * d1, rtol=0, atol=1e-9)


def test_transport_vacuum_crosses_every_boundary():
    """No material anywhere: every track flies straight out of the nested detector; its path
    is the straight exit distance from the world box (slab method) and it ends on the world's
    surface; with one step allowed, a track whose first boundary is inside the world stops on
    that boundary (truncated, its point on the surface of the volume it started in)."""
    geo_spec = W.nested_geometry()
    geo = oracle.Geometry(geo_spec["solids"], geo_spec["nodes"])
    D = np.array(geo_spec["solids"][0]["params"])
    n = 400
    t = W.nested_tracks(n, seed=9, geom=geo_spec)
    node = geo.locate(t["x"], t["y"], t["z"])
    nn = len(geo_spec["nodes"])
    xi = np.full((n, 64, 4), 0.5)
    r = geo.transport(t["x"], t["y"], t["z"], t["dx"], t["dy"], t["dz"], node, np.zeros(nn, np.int32),
                      [[0.0, 0.0]], xi, 64)
    P = np.stack([t["x"], t["y"], t["z"]], 1)
    Dd = np.stack([t["dx"], t["dy"], t["dz"]], 1)
    for i in range(n):
        t_exit = _slab(D, P[i], Dd[i])[1]
        assert r["reason"][i] == 0
        assert r["path"][i] == pytest.approx(t_exit, rel=1e-12, abs=1e-8)
        end = np.array([r["x"][i], r["y"][i], r["z"][i]])
        assert abs(np.max(np.abs(end) / D) - 1.0) < 1e-12
    r1 = geo.transport(t["x"], t["y"], t["z"], t["dx"], t["dy"], t["dz"], node, np.zeros(nn, np.int32),
                       [[0.0, 0.0]], xi[:, :1].copy(), 1)
    solids = [oracle.Solid.from_spec(s) for s in geo_spec["solids"]]
    trunc = r1["reason"] == 2
    assert trunc.sum() > n // 4 and (r1["steps"] == 1).all()
    for i in np.nonzero(trunc)[0][:80]:
        v = node[i]
        Rg, tg = geo.RG[v].reshape(3, 3), geo.tg[v]
        pl = Rg.T @ (np.array([r1["x"][i], r1["y"][i], r1["z"][i]]) - tg)
        code = solids[geo_spec["nodes"][v]["solid"]].inside(pl[None, :])[0]
        on_daughter = False
        for c in range(nn):
            if geo_spec["nodes"][c]["parent"] == v:
                Rc, tc = geo.RG[c].reshape(3, 3), geo.tg[c]
                pc = Rc.T @ (np.array([r1["x"][i], r1["y"][i], r1["z"][i]]) - tc)
                on_daughter |= solids[geo_spec["nodes"][c]["solid"]].inside(pc[None, :])[0] == 1
        assert code == 1 or on_daughter


# ------------------------------------------------------------ boolean solids

BOOL_SPECS = W.boolean_table(12, seed=2)


def _bool(op, a, c, R=np.eye(3), t=(0.0, 0.0, 0.0)):
    return {"kind": "boolean", "params": (op, a, c, np.asarray(R, float), np.asarray(t, float))}


@pytest.mark.parametrize("kind", ["box", "tube", "polycone"])
def test_boolean_identities(kind):
    """A u A = A n A = A \\ (c far away) = A n (c holding A) = A, query for query."""
    g = np.random.default_rng(81)
    a = W.random_solid(kind, g, 5.0, 40.0)
    far = {"kind": "box", "params": (1.0, 1.0, 1.0)}
    big = {"kind": "box", "params": (500.0, 500.0, 500.0)}
    t = W.tracks_for_solid(a, 800, seed=82)
    want = sol(a).query(**t)
    for spec in (_bool("union", a, a), _bool("intersection", a, a), _bool("subtraction", a, far, t=(1e3, 0, 0)),
                 _bool("intersection", a, big)):
        got = sol(spec).query(**t)
        for k in want:
            assert np.array_equal(got[k], want[k]) or np.allclose(got[k], want[k], rtol=0, atol=1e-12), (spec, k)


def test_boolean_disjoint_boxes_closed_form():
    """Two boxes far apart: the union is entered at the earlier of the two slab entries,
    and a point inside one box leaves the union where it leaves that box."""
    D1, D2, t2 = np.array([10.0, 8.0, 6.0]), np.array([5.0, 5.0, 5.0]), np.array([40.0, 3.0, -2.0])
    spec = _bool("union", {"kind": "box", "params": tuple(D1)}, {"kind": "box", "params": tuple(D2)}, t=t2)
    g = np.random.default_rng(83)
    n = 500
    P = g.uniform(-1, 1, (n, 3)) * np.array([60.0, 20.0, 20.0]) + np.array([20.0, 0, 0])
    d = W.isotropic(n, g)
    r = sol(spec).query(P[:, 0], P[:, 1], P[:, 2], d[:, 0], d[:, 1], d[:, 2])
    for i in range(n):
        a1, b1 = _slab(D1, P[i], d[i])
        a2, b2 = _slab(D2, P[i] - t2, d[i])
        in1, in2 = a1 < 0 < b1, a2 < 0 < b2
        if r["inside"][i] == OUT:
            cands = [a for a, b in ((a1, b1), (a2, b2)) if a < b and a > 0]
            want = min(cands) if cands else np.inf
            assert r["dist_in"][i] == pytest.approx(want, abs=1e-9) or (np.isinf(want) and np.isinf(r["dist_in"][i]))
        elif r["inside"][i] == IN:
            want = b1 if in1 else b2
            assert in1 or in2
            assert r["dist_out"][i] == pytest.approx(want, abs=1e-9)


def test_boolean_box_with_hole_closed_form():
    """A slab (box) minus a box-shaped hole through it along x: a point in the wall moving
    along +x leaves the solid at the hole's face or the slab's far face."""
    A = {"kind": "box", "params": (20.0, 20.0, 5.0)}
    C = {"kind": "box", "params": (4.0, 4.0, 10.0)}
    s = sol(_bool("subtraction", A, C))
    g = np.random.default_rng(84)
    n = 300
    P = np.stack([g.uniform(-19, -5, n), g.uniform(-3, 3, n), g.uniform(-4, 4, n)], 1)
    one, zero = np.ones(n), np.zeros(n)
    r = s.query(P[:, 0], P[:, 1], P[:, 2], one, zero, zero)
    assert (r["inside"] == IN).all()
    assert np.allclose(r["dist_out"], -4.0 - P[:, 0], atol=1e-9)          # the hole's -x face
    assert np.allclose(r["safety_out"], np.minimum.reduce([-4.0 - P[:, 0], 20.0 + P[:, 0], 5.0 - np.abs(P[:, 2])]),
                       atol=1e-9)
    q = np.stack([np.full(n, -4.0 + 1e-3), P[:, 1], P[:, 2]], 1)          # inside the hole
    r2 = s.query(q[:, 0], q[:, 1], q[:, 2], one, zero, zero)
    assert (r2["inside"] == OUT).all()
    assert np.allclose(r2["dist_in"], 8.0 - 1e-3, atol=1e-9)                # re-enters at x = +4


def test_boolean_slide_along_subtracted_face():
    """Box (20, 20, 20) minus a box (5, 5, 30) through it along z.  On the hole's wall x = 5:
    into the material (+x) the ray enters at once and leaves at x = 20 (15 mm); into the hole
    (-x) it leaves at once and enters again at x = -5 (10 mm); along the wall (+/-z) it stays
    on the boundary (no entry, DistanceToOut 0).  From above the box on the plane of that
    wall the ray runs down the wall (no entry); beside the hole (|y| > 5) it enters at
    z = 20."""
    s = sol(_bool("subtraction", {"kind": "box", "params": (20.0, 20.0, 20.0)},
                  {"kind": "box", "params": (5.0, 5.0, 30.0)}))
    g = np.random.default_rng(40)
    n = 400
    y, z = g.uniform(-4, 4, n), g.uniform(-19, 19, n)
    x = np.full(n, 5.0)
    one, zero = np.ones(n), np.zeros(n)
    r = s.query(x, y, z, one, zero, zero)
    assert (r["inside"] == SURF).all() and (r["dist_in"] == 0).all()
    assert np.abs(r["dist_out"] - 15.0).max() <= 1e-12
    r = s.query(x, y, z, -one, zero, zero)
    assert (r["dist_out"] == 0).all() and np.abs(r["dist_in"] - 10.0).max() <= 1e-12
    for sz in (1.0, -1.0):
        r = s.query(x, y, z, zero, zero, sz * one)
        assert (r["dist_out"] == 0).all() and np.isinf(r["dist_in"]).all()
    ztop = np.full(n, 25.0)
    r = s.query(x, y, ztop, zero, zero, -one)
    assert (r["inside"] == OUT).all() and np.isinf(r["dist_in"]).all()
    yb = np.where(g.random(n) < 0.5, -1.0, 1.0) * g.uniform(6, 19, n)
    r = s.query(x, yb, ztop, zero, zero, -one)
    assert np.abs(r["dist_in"] - 5.0).max() <= 1e-12


@pytest.mark.parametrize("idx", range(len(BOOL_SPECS)))
def test_boolean_brute_force_ray_march(idx):
    spec = BOOL_SPECS[idx]
    s = sol(spec)
    n = 200
    t = W.tracks_for_solid(spec, n, seed=400 + idx, near_frac=0.0)
    P = np.stack([t["x"], t["y"], t["z"]], 1)
    D = np.stack([t["dx"], t["dy"], t["dz"]], 1)
    r = s.query(**t)
    hb = W.bounding_half(spec)
    tmax = 2.0 * np.linalg.norm(hb * 2.0 + 1.0)
    step = float(max(hb.min() / 200.0, 0.01))
    out = r["inside"] == OUT
    ins = r["inside"] == IN
    te = _march(s, P[out], D[out], True, tmax, step)
    tx = _march(s, P[ins], D[ins], False, tmax, step)
    fin = np.isfinite(te)
    assert (r["dist_in"][out][fin] <= te[fin] + 1e-9).all()
    with np.errstate(invalid="ignore"):
        agree_e = np.where(fin, np.abs(r["dist_in"][out] - te) <= 1e-9, np.isinf(r["dist_in"][out]))
    agree_x = np.abs(r["dist_out"][ins] - tx) <= 1e-9
    assert agree_e.mean() >= 0.98, agree_e.mean()
    assert agree_x.mean() >= 0.98, agree_x.mean()


@pytest.mark.parametrize("idx", range(0, len(BOOL_SPECS), 2))
def test_boolean_safety_is_a_lower_bound(idx):
    """As for the primitives: 0 <= safety <= every distance along 64 Fibonacci directions."""
    spec = BOOL_SPECS[idx]
    s = sol(spec)
    n = 300
    t = W.tracks_for_solid(spec, n, seed=500 + idx)
    r = s.query(**t)
    k = np.arange(64) + 0.5
    th = np.arccos(1 - 2 * k / 64)
    ph = math.pi * (1 + 5 ** 0.5) * k
    fib = np.stack([np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)], 1)
    rep = lambda a: np.repeat(a, 64)  # noqa: E731
    tt = {"x": rep(t["x"]), "y": rep(t["y"]), "z": rep(t["z"]),
          "dx": np.tile(fib[:, 0], n), "dy": np.tile(fib[:, 1], n), "dz": np.tile(fib[:, 2], n)}
    rr = s.query(**tt)
    din, dout = rr["dist_in"].reshape(n, 64), rr["dist_out"].reshape(n, 64)
    out, ins = r["inside"] == OUT, r["inside"] == IN
    assert (r["safety_in"][out] > 0).all() and (r["safety_out"][ins] > 0).all()
    assert (r["safety_in"][out] <= din[out].min(axis=1) + 1e-9).all()
    assert (r["safety_out"][ins] <= dout[ins].min(axis=1) + 1e-9).all()
