"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws random numbers: solid descriptions, point/direction
baskets, basket tables and the nested detector layout.  It holds none of the
query arithmetic (no inside test, no distance, no safety); points are placed by
sampling each solid's parametric description (its faces, its radial and
azimuthal ranges), and a point "near a surface" is a sampled surface point moved
by an isotropic offset no longer than the stated band.

Workloads (random points and isotropic directions, as in the paper's speed test
of the VecGeom section, where random particles are tested against a Box and a
Tube):

* ``box1024``     -- box (10,20,30) mm, 1024 tracks uniform in a (20,40,60) mm world
                     box, 5% of them within 1e-10 mm of a face.
* ``tube_cone_1m``-- tube segment (5,20,30, phi 0-270 deg) and cone segment
                     (0,10,5,25,40, full phi), 2^20 tracks each, half sampled
                     inside the solid and half uniform in a world box twice the
                     bounding box, 10% within 1e-8 mm of a surface.
* ``precision_16m``-- 2^24 tracks per solid over box, trd (10,20,15,5,30), tube,
                     cone and an 8-plane polycone, same recipe.
* ``batched``     -- 4096 baskets, sizes log-uniform in [16, 4096], each against one
                     of 64 solids of the six types with parameters in 1-100 mm.
* ``nested``      -- world box holding 10 concentric tube shells holding 32 box
                     cells each; requests with sizes log-uniform in [1, 65536].
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1512_06637
TWO_PI = 2.0 * math.pi
DEG = math.pi / 180.0

# ----------------------------------------------------------------- solids

BOX_M1 = {"kind": "box", "params": (10.0, 20.0, 30.0)}
TUBE_M2 = {"kind": "tube", "params": (5.0, 20.0, 30.0, 0.0, 270.0 * DEG)}
CONE_M2 = {"kind": "cone", "params": (0.0, 10.0, 5.0, 25.0, 40.0, 0.0, TWO_PI)}
TRD_M3 = {"kind": "trd", "params": (10.0, 20.0, 15.0, 5.0, 30.0)}


def rng(tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(tag)))


def polycone_m3(seed: int = 2, nz: int = 8) -> dict:
    """8 z-planes sorted in [-50, 50] at least 2 mm apart, 1 <= rmin < rmax <= 50, full phi."""
    g = rng(1000 + seed)
    u = np.sort(g.uniform(0.0, 100.0 - 2.0 * (nz - 1), nz))
    z = -50.0 + u + 2.0 * np.arange(nz)
    rmin = g.uniform(1.0, 40.0, nz)
    rmax = np.minimum(50.0, rmin + g.uniform(2.0, 30.0, nz))
    return {"kind": "polycone", "params": (tuple(z), tuple(rmin), tuple(rmax), 0.0, TWO_PI)}


def trap_random(g: np.random.Generator, lo=1.0, hi=100.0) -> dict:
    """A planar trapezoid: the +dz face is k times the -dz face (k in [0.5, 1.5]) so
    that paired edges stay parallel; theta, phi in [0, 15] deg, alpha1 = alpha2."""
    dz = g.uniform(lo, hi)
    dy1 = g.uniform(lo, hi / 1.5)
    dx1 = g.uniform(lo, hi / 1.5)
    dx2 = g.uniform(lo, hi / 1.5)
    k = g.uniform(0.5, 1.5)
    th = g.uniform(0, 15) * DEG
    ph = g.uniform(0, 15) * DEG
    al = g.uniform(-15, 15) * DEG
    return {"kind": "trap", "params": ((dz, th, ph, dy1, dx1, dx2, al, k * dy1, k * dx1, k * dx2, al),)}


def random_solid(kind: str, g: np.random.Generator, lo=1.0, hi=100.0) -> dict:
    """One solid of the given kind with seeded parameters in [lo, hi] mm."""
    u = lambda a=lo, b=hi: float(g.uniform(a, b))  # noqa: E731
    if kind == "box":
        return {"kind": "box", "params": (u(), u(), u())}
    if kind == "trd":
        return {"kind": "trd", "params": (u(), u(), u(), u(), u())}
    if kind == "trap":
        return trap_random(g, lo, hi)
    phi_choice = g.integers(0, 3)
    if phi_choice == 0:
        sphi, dphi = 0.0, TWO_PI
    else:
        sphi = float(g.uniform(0, 360)) * DEG
        dphi = float(g.uniform(30, 330)) * DEG
    if kind == "tube":
        rmax = u(lo + 1.0, hi)
        rmin = float(g.uniform(0, rmax - 0.5)) if g.integers(0, 4) else 0.0
        return {"kind": "tube", "params": (rmin, rmax, u(), sphi, dphi)}
    if kind == "cone":
        rmax1, rmax2 = u(lo + 1.0, hi), u(lo + 1.0, hi)
        rmin1 = float(g.uniform(0, rmax1 - 0.5)) if g.integers(0, 3) else 0.0
        rmin2 = float(g.uniform(0, rmax2 - 0.5)) if g.integers(0, 3) else 0.0
        return {"kind": "cone", "params": (rmin1, rmax1, rmin2, rmax2, u(), sphi, dphi)}
    if kind == "polycone":
        nz = int(g.integers(2, 9))
        span = u(10.0, hi)
        z = np.sort(g.uniform(-span, span, nz))
        z = z + 0.5 * np.arange(nz)  # strictly increasing
        rmin = g.uniform(0.0, 0.5 * hi, nz) * (g.random(nz) < 0.7)
        rmax = rmin + g.uniform(lo, 0.5 * hi, nz)
        return {"kind": "polycone", "params": (tuple(z), tuple(rmin), tuple(rmax), sphi, dphi)}
    raise ValueError(kind)


KINDS6 = ("box", "trd", "trap", "tube", "cone", "polycone")


def solid_table(n: int = 64, seed: int = 3) -> list[dict]:
    """n solids of the six types in turn (type i % 6), seeded parameters in 1-100 mm."""
    g = rng(2000 + seed)
    return [random_solid(KINDS6[i % 6], g) for i in range(n)]


# ------------------------------------------------- parametric descriptions

def _trap_vertices(p):
    dz, th, ph, dy1, dx1, dx2, a1, dy2, dx3, dx4, a2 = p
    out = []
    for zf, dy, dxa, dxb, al in ((-dz, dy1, dx1, dx2, a1), (dz, dy2, dx3, dx4, a2)):
        cx = zf * math.tan(th) * math.cos(ph)
        cy = zf * math.tan(th) * math.sin(ph)
        sh = dy * math.tan(al)
        out += [(cx - sh - dxa, cy - dy, zf), (cx - sh + dxa, cy - dy, zf),
                (cx + sh - dxb, cy + dy, zf), (cx + sh + dxb, cy + dy, zf)]
    return np.array(out)


def _as_trap(spec):
    k, p = spec["kind"], spec["params"]
    if k == "box":
        dx, dy, dz = p
        return (dz, 0, 0, dy, dx, dx, 0, dy, dx, dx, 0)
    if k == "trd":
        dx1, dx2, dy1, dy2, dz = p
        return (dz, 0, 0, dy1, dx1, dx1, 0, dy2, dx2, dx2, 0)
    return tuple(p[0])


def _as_pcon(spec):
    k, p = spec["kind"], spec["params"]
    if k == "tube":
        rmin, rmax, dz, sphi, dphi = p
        return [-dz, dz], [rmin, rmin], [rmax, rmax], sphi, dphi
    if k == "cone":
        rmin1, rmax1, rmin2, rmax2, dz, sphi, dphi = p
        return [-dz, dz], [rmin1, rmin2], [rmax1, rmax2], sphi, dphi
    z, rmin, rmax, sphi, dphi = p
    return list(z), list(rmin), list(rmax), sphi, dphi


def random_rotation(g: np.random.Generator) -> np.ndarray:
    """A uniformly random proper rotation (QR of a Gaussian matrix, signs fixed)."""
    q, r = np.linalg.qr(g.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def boolean_random(g: np.random.Generator, lo=5.0, hi=60.0, op: str | None = None) -> dict:
    """op(a, c): two random primitives, c smaller, rotated at random and shifted by up to
    0.3 of a's extent so that the two overlap."""
    kinds = ("box", "trd", "trap", "tube", "cone", "polycone")
    op = op or str(g.choice(["union", "subtraction", "intersection"]))
    a = random_solid(str(g.choice(kinds)), g, lo, hi)
    c = random_solid(str(g.choice(kinds)), g, lo, hi * 0.7)
    R = random_rotation(g)
    t = g.uniform(-0.3, 0.3, 3) * bounding_half(a)
    return {"kind": "boolean", "params": (op, a, c, R, t)}


def boolean_table(n: int = 24, seed: int = 9) -> list[dict]:
    g = rng(8000 + seed)
    ops = ("union", "subtraction", "intersection")
    return [boolean_random(g, op=ops[i % 3]) for i in range(n)]


def _bool_parts(spec):
    op, a, c, R, t = spec["params"]
    return op, a, c, np.asarray(R, np.float64).reshape(3, 3), np.asarray(t, np.float64).reshape(3)


def bounding_half(spec) -> np.ndarray:
    """Half-lengths of an axis-aligned box around the origin that holds the solid."""
    if spec["kind"] == "boolean":
        _, a, c, R, t = _bool_parts(spec)
        hc = bounding_half(c)
        corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]) * hc
        return np.maximum(bounding_half(a), np.abs(corners @ R.T + t).max(axis=0))
    if spec["kind"] in ("box", "trd", "trap"):
        v = _trap_vertices(_as_trap(spec))
        return np.abs(v).max(axis=0)
    z, rmin, rmax, _, _ = _as_pcon(spec)
    r = max(rmax)
    return np.array([r, r, max(abs(z[0]), abs(z[-1]))])


def _sample_inside(spec, n, g):
    """Points drawn from the solid's parametric interior (not uniform in volume).  For a
    boolean: from either component's interior (placed), whatever the operation keeps."""
    if spec["kind"] == "boolean":
        _, a, c, R, t = _bool_parts(spec)
        na = n // 2
        return np.concatenate([_sample_inside(a, na, g), _sample_inside(c, n - na, g) @ R.T + t])
    if spec["kind"] in ("box", "trd", "trap"):
        v = _trap_vertices(_as_trap(spec))
        a, b, c = g.random(n), g.random(n), g.random(n)
        # trilinear blend of the 8 vertices: v[4j + 2i + k] at (k = x-side, i = y-side, j = z-side)
        w = np.empty((n, 8))
        for j in range(2):
            for i in range(2):
                for k in range(2):
                    w[:, 4 * j + 2 * i + k] = (c if j else 1 - c) * (b if i else 1 - b) * (a if k else 1 - a)
        return w @ v
    z, rmin, rmax, sphi, dphi = _as_pcon(spec)
    z, rmin, rmax = map(np.asarray, (z, rmin, rmax))
    zz = g.uniform(z[0], z[-1], n)
    k = np.clip(np.searchsorted(z, zz, side="right") - 1, 0, len(z) - 2)
    f = (zz - z[k]) / (z[k + 1] - z[k])
    r0 = rmin[k] + f * (rmin[k + 1] - rmin[k])
    r1 = rmax[k] + f * (rmax[k + 1] - rmax[k])
    rr = np.sqrt(g.uniform(r0 * r0, r1 * r1))
    ph = sphi + g.random(n) * min(dphi, TWO_PI)
    return np.stack([rr * np.cos(ph), rr * np.sin(ph), zz], axis=1)


def _sample_surface(spec, n, g):
    """Points drawn on the solid's faces, face chosen with probability ~ its area."""
    if spec["kind"] == "boolean":  # on either component's surface (placed)
        _, a, c, R, t = _bool_parts(spec)
        na = n // 2
        return np.concatenate([_sample_surface(a, na, g), _sample_surface(c, n - na, g) @ R.T + t])
    if spec["kind"] in ("box", "trd", "trap"):
        v = _trap_vertices(_as_trap(spec))
        quads = [(0, 1, 3, 2), (4, 5, 7, 6), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5)]
        areas = []
        for q in quads:
            A, B, C, D = v[list(q)]
            areas.append(0.5 * np.linalg.norm(np.cross(C - A, D - B)))
        areas = np.array(areas)
        f = g.choice(6, size=n, p=areas / areas.sum())
        a, b = g.random(n), g.random(n)
        out = np.empty((n, 3))
        for fi, q in enumerate(quads):
            m = f == fi
            A, B, C, D = v[list(q)]
            aa, bb = a[m, None], b[m, None]
            out[m] = (1 - aa) * (1 - bb) * A + aa * (1 - bb) * B + aa * bb * C + (1 - aa) * bb * D
        return out
    z, rmin, rmax, sphi, dphi = _as_pcon(spec)
    z, rmin, rmax = map(np.asarray, (z, rmin, rmax))
    dp = min(dphi, TWO_PI)
    has_phi = dphi < TWO_PI
    # faces: lateral outer/inner per section, two end caps, two phi planes
    faces, areas = [], []
    for k in range(len(z) - 1):
        h = z[k + 1] - z[k]
        for side, rr in (("out", rmax), ("in", rmin)):
            slant = math.hypot(h, rr[k + 1] - rr[k])
            a = 0.5 * (rr[k] + rr[k + 1]) * dp * slant
            if a > 0:
                faces.append((side, k)); areas.append(a)
    for j in (0, len(z) - 1):
        faces.append(("cap", j)); areas.append(0.5 * dp * (rmax[j] ** 2 - rmin[j] ** 2))
    if has_phi:
        prof = sum((z[k + 1] - z[k]) * 0.5 * ((rmax[k] - rmin[k]) + (rmax[k + 1] - rmin[k + 1]))
                   for k in range(len(z) - 1))
        faces += [("phi", 0), ("phi", 1)]; areas += [prof, prof]
    areas = np.array(areas)
    f = g.choice(len(faces), size=n, p=areas / areas.sum())
    out = np.empty((n, 3))
    u, w = g.random(n), g.random(n)
    for fi, (kind, k) in enumerate(faces):
        m = f == fi
        cnt = int(m.sum())
        if cnt == 0:
            continue
        ph = sphi + u[m] * dp
        if kind in ("out", "in"):
            rr = rmax if kind == "out" else rmin
            zz = z[k] + w[m] * (z[k + 1] - z[k])
            r = rr[k] + (zz - z[k]) / (z[k + 1] - z[k]) * (rr[k + 1] - rr[k])
        elif kind == "cap":
            zz = np.full(cnt, z[k])
            r = np.sqrt(rmin[k] ** 2 + w[m] * (rmax[k] ** 2 - rmin[k] ** 2))
        else:
            ph = np.full(cnt, sphi + (dp if k else 0.0))
            sec = np.clip(np.searchsorted(z, z[0] + w[m] * (z[-1] - z[0]), side="right") - 1, 0, len(z) - 2)
            zz = z[0] + w[m] * (z[-1] - z[0])
            fr = (zz - z[sec]) / (z[sec + 1] - z[sec])
            r0 = rmin[sec] + fr * (rmin[sec + 1] - rmin[sec])
            r1 = rmax[sec] + fr * (rmax[sec + 1] - rmax[sec])
            r = r0 + g.random(cnt) * (r1 - r0)
        out[m] = np.stack([r * np.cos(ph), r * np.sin(ph), zz], axis=1)
    return out


def isotropic(n: int, g: np.random.Generator) -> np.ndarray:
    v = g.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _offset(n, band, g):
    return isotropic(n, g) * g.uniform(0.0, band, (n, 1))


def tracks_for_solid(spec: dict, n: int, seed: int, near_frac=0.10, band=1e-8,
                     inside_frac=0.5, world_scale=2.0) -> dict:
    """Half (inside_frac) parametric interior points, the rest uniform in a world box
    world_scale times the bounding box; near_frac of all points moved onto a surface
    point plus an isotropic offset of length <= band.  Directions are isotropic."""
    g = rng(seed)
    hb = bounding_half(spec) * world_scale + 1.0
    n_in = int(round(n * inside_frac))
    pts = np.empty((n, 3))
    pts[:n_in] = _sample_inside(spec, n_in, g)
    pts[n_in:] = g.uniform(-1, 1, (n - n_in, 3)) * hb
    n_near = int(round(n * near_frac))
    if n_near:
        idx = g.choice(n, n_near, replace=False)
        pts[idx] = _sample_surface(spec, n_near, g) + _offset(n_near, band, g)
    perm = g.permutation(n)
    pts = pts[perm]
    d = isotropic(n, g)
    return soa(pts, d)


def soa(pts, d) -> dict:
    pts = np.asarray(pts, np.float64)
    d = np.asarray(d, np.float64)
    return {"x": np.ascontiguousarray(pts[:, 0]), "y": np.ascontiguousarray(pts[:, 1]),
            "z": np.ascontiguousarray(pts[:, 2]), "dx": np.ascontiguousarray(d[:, 0]),
            "dy": np.ascontiguousarray(d[:, 1]), "dz": np.ascontiguousarray(d[:, 2])}


def box1024(n: int = 1024, seed: int = 0) -> dict:
    """Box (10,20,30): points uniform in a (20,40,60) world box, 5% within 1e-10 mm of a face."""
    g = rng(seed)
    D = np.array(BOX_M1["params"])
    pts = g.uniform(-1, 1, (n, 3)) * (2 * D)
    n_face = int(round(0.05 * n))
    idx = g.choice(n, n_face, replace=False)
    axis = g.integers(0, 3, n_face)
    sign = np.where(g.random(n_face) < 0.5, -1.0, 1.0)
    face_pts = g.uniform(-1, 1, (n_face, 3)) * D
    face_pts[np.arange(n_face), axis] = sign * D[axis] + g.uniform(-1e-10, 1e-10, n_face)
    pts[idx] = face_pts
    return soa(pts, isotropic(n, g))


# --------------------------------------------------------- batched form

def batched(n_baskets: int = 4096, seed: int = 4, lo: int = 16, hi: int = 4096,
            n_solids: int = 64) -> dict:
    """Basket table {offset, n, solid} with log-uniform sizes and the tracks of every
    basket drawn for its own solid; returns solids, baskets and one SoA of all tracks."""
    g = rng(3000 + seed)
    solids = solid_table(n_solids, seed)
    sizes = np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), n_baskets))).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    sid = g.integers(0, n_solids, n_baskets).astype(np.int32)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    total = int(sizes.sum())
    cols = {k: np.empty(total) for k in ("x", "y", "z", "dx", "dy", "dz")}
    for b in range(n_baskets):
        t = tracks_for_solid(solids[sid[b]], int(sizes[b]), seed=10_000 + 7919 * seed + b)
        o = offs[b]
        for k in cols:
            cols[k][o:o + sizes[b]] = t[k]
    return {"solids": solids, "offset": offs, "n": sizes, "solid": sid, "tracks": cols}


# ------------------------------------------------------ nested geometry

def nested_geometry(n_shells: int = 10, cells_phi: int = 8, cells_z: int = 4) -> dict:
    """World box (250,250,550) mm holding 10 tube shells (rmin = 10 + 19k, rmax = rmin + 18,
    dz = 500, full phi), each holding 32 box cells (4.5, 4.5, 112.5) centred at the shell's
    mid radius, 8 in phi (22.5 + 45 j deg, rotated about z) by 4 in z (-375, -125, 125, 375)."""
    solids = [{"kind": "box", "params": (250.0, 250.0, 550.0)},
              {"kind": "box", "params": (4.5, 4.5, 112.5)}]
    ident = np.eye(3)
    nodes = [{"solid": 0, "parent": -1, "R": ident, "t": np.zeros(3)}]
    shell_nodes = []
    for k in range(n_shells):
        rmin = 10.0 + 19.0 * k
        solids.append({"kind": "tube", "params": (rmin, rmin + 18.0, 500.0, 0.0, TWO_PI)})
        nodes.append({"solid": len(solids) - 1, "parent": 0, "R": ident, "t": np.zeros(3)})
        shell_nodes.append(len(nodes) - 1)
    for k, sn in enumerate(shell_nodes):
        rmid = 10.0 + 19.0 * k + 9.0
        for iz, zc in enumerate((-375.0, -125.0, 125.0, 375.0)[:cells_z]):
            for j in range(cells_phi):
                ph = (22.5 + 45.0 * j) * DEG
                c, s = math.cos(ph), math.sin(ph)
                R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
                nodes.append({"solid": 1, "parent": sn, "R": R, "t": np.array([rmid * c, rmid * s, zc])})
    return {"solids": solids, "nodes": nodes}


def nested_tracks(n: int, seed: int, geom: dict | None = None) -> dict:
    """Points uniform in the world box, isotropic directions."""
    g = rng(4000 + seed)
    hb = np.array((geom or nested_geometry())["solids"][0]["params"])
    pts = g.uniform(-1, 1, (n, 3)) * hb
    return soa(pts, isotropic(n, g))


def _scaled(spec: dict, f: float) -> dict:
    """A primitive solid with every length multiplied by f (angles kept)."""
    kind, p = spec["kind"], spec["params"]
    if kind in ("box", "trd"):
        return {"kind": kind, "params": tuple(f * v for v in p)}
    if kind == "trap":
        q = list(p[0])
        for i in (0, 3, 4, 5, 7, 8, 9):
            q[i] *= f
        return {"kind": kind, "params": (tuple(q),)}
    if kind == "tube":
        return {"kind": kind, "params": (f * p[0], f * p[1], f * p[2], p[3], p[4])}
    if kind == "cone":
        return {"kind": kind, "params": tuple(f * v for v in p[:5]) + (p[5], p[6])}
    z, rmin, rmax, sphi, dphi = p
    return {"kind": kind, "params": (tuple(f * v for v in z), tuple(f * v for v in rmin),
                                     tuple(f * v for v in rmax), sphi, dphi)}


def crowded_geometry(lattice: int = 12, seed: int = 0) -> dict:
    """A volume with many daughters: world box (600, 600, 600) mm holding a lattice^3 array of
    daughters at a 100 mm pitch (1728 by default), each a random solid of the six kinds or
    a boolean (every eighth), randomly rotated about its lattice point and shifted by up to
    5 mm, its bounding sphere under 45 mm so that neighbours do not overlap.  The daughter
    at lattice point (0, 0, 0) is instead a box (28, 28, 28), rotated, that holds a 3 x 3 x 3
    array of small solids at an 18 mm pitch, bounding spheres under 9 mm (27 daughters, a
    second level with its own grid)."""
    g = rng(8000 + seed)
    solids = [{"kind": "box", "params": (600.0, 600.0, 600.0)}]
    table = []
    while len(table) < 40:
        k = len(table)
        spec = boolean_random(g, lo=5.0, hi=18.0) if k % 8 == 7 else random_solid(KINDS6[k % 6], g, lo=4.0, hi=26.0)
        if np.linalg.norm(bounding_half(spec)) < 45.0:
            table.append(spec)
    small = []
    while len(small) < 12:
        spec = _scaled(random_solid(KINDS6[len(small) % 6], g, lo=4.0, hi=26.0), 0.2)
        if np.linalg.norm(bounding_half(spec)) < 9.0:
            small.append(spec)
    solids += table + small + [{"kind": "box", "params": (28.0, 28.0, 28.0)}]
    first_small, sub_box = 1 + len(table), len(solids) - 1
    nodes = [{"solid": 0, "parent": -1, "R": np.eye(3), "t": np.zeros(3)}]
    c0 = -0.5 * (lattice - 1) * 100.0
    sub = -1
    for i in range(lattice):
        for j in range(lattice):
            for k in range(lattice):
                t = np.array([c0 + 100.0 * i, c0 + 100.0 * j, c0 + 100.0 * k])
                if i == j == k == 0:
                    sub = len(nodes)
                    nodes.append({"solid": sub_box, "parent": 0, "R": random_rotation(g), "t": t})
                else:
                    nodes.append({"solid": 1 + int(g.integers(len(table))), "parent": 0, "R": random_rotation(g),
                                  "t": t + g.uniform(-5, 5, 3)})
    for i in range(3):
        for j in range(3):
            for k in range(3):
                nodes.append({"solid": first_small + int(g.integers(len(small))), "parent": sub,
                              "R": random_rotation(g), "t": np.array([18.0 * (i - 1), 18.0 * (j - 1), 18.0 * (k - 1)])})
    return {"solids": solids, "nodes": nodes}


def crowded_tracks(geom: dict, n: int, seed: int, surf_frac: float = 0.3, axis_frac: float = 0.1) -> dict:
    """Points for a crowded geometry: uniform in the world box, except a fraction drawn on the
    surfaces of random daughters of the world (placed in world coordinates); isotropic
    directions, except a fraction along +-x, +-y or +-z (rays parallel to grid planes)."""
    g = rng(9000 + seed)
    hb = np.array(geom["solids"][0]["params"])
    pts = g.uniform(-1, 1, (n, 3)) * hb
    d = isotropic(n, g)
    m = int(n * surf_frac)
    kids = [i for i, nd in enumerate(geom["nodes"]) if nd["parent"] == 0]
    pick = g.choice(kids, m)
    for v in np.unique(pick):
        sel = np.nonzero(pick == v)[0]
        nd = geom["nodes"][v]
        loc = _sample_surface(geom["solids"][nd["solid"]], len(sel), g)
        pts[sel] = loc @ np.asarray(nd["R"]).T + nd["t"]
    a = int(n * axis_frac)
    idx = g.choice(n, a, replace=False)
    ax = g.integers(0, 3, a)
    d[idx] = 0.0
    d[idx, ax] = np.where(g.random(a) < 0.5, -1.0, 1.0)
    perm = g.permutation(n)
    return soa(pts[perm], d)


def crowded_materials(geom: dict) -> dict:
    """Materials for the transport loop in a crowded geometry: the world a light material
    (mean free paths 400 / 2000 mm), the daughters a dense one (20 / 80 mm)."""
    mat = np.array([0 if nd["parent"] < 0 else 1 for nd in geom["nodes"]], np.int32)
    return {"node_material": mat, "sigma_n": np.array([[0.0025, 0.0005], [0.05, 0.0125]])}


def transport_materials(geom: dict) -> dict:
    """Materials of the nested detector for the transport loop: the world is vacuum, the tube
    shells a light material, the box cells a dense one; n sigma of (scatter, absorb) in 1/mm
    (mean free paths 100 / 500 mm in the shells, 20 / 50 mm in the cells)."""
    nodes = geom["nodes"]
    mat = np.zeros(len(nodes), np.int32)
    for i, nd in enumerate(nodes):
        if nd["parent"] == 0:
            mat[i] = 1
        elif nd["parent"] > 0:
            mat[i] = 2
    sigma_n = np.array([[0.0, 0.0], [0.01, 0.002], [0.05, 0.02]])
    return {"node_material": mat, "sigma_n": sigma_n}


def transport_xi(n: int, kmax: int, seed: int) -> np.ndarray:
    """Uniform random numbers in (0, 1] for the transport loop, shape (n, kmax, 4)."""
    return 1.0 - rng(7000 + seed).random((n, kmax, 4))


def request_sizes(n_req: int, seed: int, lo: int = 1, hi: int = 65536) -> np.ndarray:
    g = rng(5000 + seed)
    return np.clip(np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), n_req))), lo, hi).astype(np.int64)


def poisson_arrivals(n_req: int, rate_per_s: float, seed: int) -> np.ndarray:
    g = rng(6000 + seed)
    return np.cumsum(g.exponential(1.0 / rate_per_s, n_req))


# ------------------------------------------------------------ grazing rays
#
# Rays that touch a surface, run along it, or cross exactly through an edge: each
# family places points on a surface (or on the plane or line of one) by construction
# and gives directions that lie in it or touch it.  ``meta`` holds the construction
# values (radii, touch distances, direction scale) that closed forms are written in.

TUBE_FULL = {"kind": "tube", "params": (5.0, 20.0, 30.0, 0.0, TWO_PI)}

GRAZING_FAMILIES = ("tube_outer_tangent", "tube_inner_tangent", "cone_outer_generator",
                    "cone_inner_generator", "phi_face_slide", "box_edge_touch", "box_face_slide",
                    "hole_touch", "outer_touch", "z_face_slide")


def grazing_tracks(family: str, n: int, seed: int):
    """(solid spec, tracks, meta) for one family of grazing rays."""
    g = rng(seed)
    one, zero = np.ones(n), np.zeros(n)
    if family in ("tube_outer_tangent", "tube_inner_tangent"):
        outer = family == "tube_outer_tangent"
        spec = TUBE_M2 if outer else TUBE_FULL
        R = 20.0 if outer else 5.0
        ph = g.uniform(0.02, 1.5 * math.pi - 0.02 if outer else TWO_PI, n)
        # a third exactly on the wall, the rest moved radially within the band
        dr = np.where(np.arange(n) % 3 == 0, 0.0, g.uniform(-0.4e-9, 0.4e-9, n))
        z = g.uniform(-20, 20, n)
        w = np.where(g.random(n) < 0.5, 0.0, g.uniform(-0.3, 0.3, n))
        c = np.sqrt(1 - w * w)
        sg = np.where(g.random(n) < 0.5, -1.0, 1.0)
        p = np.stack([(R + dr) * np.cos(ph), (R + dr) * np.sin(ph), z], 1)
        d = np.stack([-sg * c * np.sin(ph), sg * c * np.cos(ph), w], 1)
        return spec, soa(p, d), {"z": z, "w": w, "c": c}
    if family in ("cone_outer_generator", "cone_inner_generator"):
        spec = CONE_M2
        a, r1 = (15.0 / 80.0, 10.0) if family == "cone_outer_generator" else (5.0 / 80.0, 0.0)
        z = g.uniform(-39, 39, n)
        R = a * (z + 40.0) + r1
        ph = g.uniform(0, TWO_PI, n)
        sg = np.where(g.random(n) < 0.5, -1.0, 1.0)
        k = 1.0 / math.sqrt(1 + a * a)
        p = np.stack([R * np.cos(ph), R * np.sin(ph), z], 1)
        d = sg[:, None] * np.stack([a * k * np.cos(ph), a * k * np.sin(ph), k * one], 1)
        return spec, soa(p, d), {"z": z, "sign": sg}
    if family == "phi_face_slide":
        spec = TUBE_M2
        face = np.where(g.random(n) < 0.5, 0.0, 1.5 * math.pi)
        kind = g.integers(0, 3, n)  # 0: on the face, 1: beyond rmax on its plane, 2: the interior half-plane
        r0 = np.where(kind == 0, g.uniform(6, 19, n), np.where(kind == 1, g.uniform(21, 30, n), g.uniform(6, 19, n)))
        phr = np.where(kind == 2, face + math.pi, face)
        z = g.uniform(-10, 10, n)
        w = np.where(g.random(n) < 0.5, 0.0, g.uniform(-0.3, 0.3, n))
        c = np.sqrt(1 - w * w)
        sg = np.where(g.random(n) < 0.5, -1.0, 1.0)  # +1 away from the axis
        p = np.stack([r0 * np.cos(phr), r0 * np.sin(phr), z], 1)
        d = np.stack([sg * c * np.cos(phr), sg * c * np.sin(phr), w], 1)
        return spec, soa(p, d), {"kind": kind, "r0": r0, "c": c, "sign": sg}
    if family in ("box_edge_touch", "box_face_slide"):
        spec = BOX_M1
        D = np.array(spec["params"])
        p = np.empty((n, 3))
        d = np.zeros((n, 3))
        meta = {"t0": np.zeros(n), "kind": np.zeros(n, int)}
        for m in range(n):
            i, j = g.choice(3, 2, replace=False)
            k = 3 - i - j
            si, sj = g.choice([-1.0, 1.0], 2)
            if family == "box_edge_touch":
                E = np.zeros(3)
                E[i], E[j], E[k] = si * D[i], sj * D[j], g.uniform(-D[k] + 1, D[k] - 1)
                beta = g.uniform(0.1, 1.4)
                through = g.random() < 0.25  # a quarter cross the edge into the box
                e = np.zeros(3)
                e[i] = -si * math.cos(beta)
                e[j] = (-sj if through else sj) * math.sin(beta)
                e[k] = g.uniform(-0.3, 0.3) if g.random() < 0.5 else 0.0
                e /= np.linalg.norm(e)
                t0 = g.uniform(1, 10)
                p[m] = E - t0 * e
                d[m] = e
                meta["t0"][m], meta["kind"][m] = t0, int(through)
            else:
                q = g.uniform(-1, 1, 3) * (D - 1)
                q[i] = si * D[i]
                out = g.random() < 0.5  # beyond the face's edge, on its plane
                if out:
                    q[j] = sj * (D[j] + g.uniform(1, 10))
                e = np.zeros(3)
                ang = g.uniform(0, TWO_PI)
                e[j], e[k] = math.cos(ang), math.sin(ang)
                if out:
                    e[j] = -sj * abs(e[j])  # toward the face
                p[m], d[m] = q, e
                meta["kind"][m] = int(out)
        return spec, soa(p, d), meta
    if family in ("hole_touch", "outer_touch"):
        spec = TUBE_FULL
        R = 5.0 if family == "hole_touch" else 20.0
        ph = g.uniform(0, TWO_PI, n)
        z = g.uniform(-20, 20, n)
        t0 = g.uniform(1, 15, n)
        T = np.stack([R * np.cos(ph), R * np.sin(ph), z], 1)
        e = np.stack([-np.sin(ph), np.cos(ph), zero], 1)
        return spec, soa(T - t0[:, None] * e, e), {"t0": t0}
    if family == "z_face_slide":
        spec = TUBE_FULL
        top = np.where(g.random(n) < 0.5, 30.0, -30.0)
        out = g.random(n) < 0.4
        rr = np.where(out, g.uniform(21, 40, n), g.uniform(6, 19, n))
        ph = g.uniform(0, TWO_PI, n)
        ang = g.uniform(0, TWO_PI, n)
        dxy = np.stack([np.cos(ang), np.sin(ang)], 1)
        # points beyond rmax move toward the axis
        toward = -np.stack([np.cos(ph), np.sin(ph)], 1)
        dxy = np.where(out[:, None], toward, dxy)
        p = np.stack([rr * np.cos(ph), rr * np.sin(ph), top], 1)
        d = np.stack([dxy[:, 0], dxy[:, 1], zero], 1)
        return spec, soa(p, d), {"out": out}
    raise ValueError(family)


# ------------------------------------------------------------ degenerate solids

def degenerate_table() -> list[dict]:
    """Solids at the edges of their parameter ranges: the largest polycone (32 planes, walls
    pinching to the axis), phi wedges of 1e-3 rad, exactly pi and just below 2 pi, a wall 1e-6 mm
    thick, cones whose outer radius shrinks to 1e-3 mm at one end, a tube 1e4 mm long, a box 1e-3 mm
    wide, and a trap tilted 60 degrees."""
    g = rng(4242)
    z = np.sort(g.uniform(-80.0, 80.0, 32))
    z = z + np.arange(32) * 1e-3  # strictly increasing
    rmax = g.uniform(5.0, 40.0, 32)
    rmin = np.where(g.random(32) < 0.3, 0.0, rmax * g.uniform(0.1, 0.9, 32))
    return [
        {"kind": "polycone", "params": (tuple(z), tuple(rmin), tuple(rmax), 0.0, TWO_PI)},
        {"kind": "polycone", "params": (tuple(z), tuple(rmin), tuple(rmax), 0.4, 4.0)},
        {"kind": "tube", "params": (5.0, 20.0, 30.0, 0.3, 1e-3)},
        {"kind": "tube", "params": (5.0, 20.0, 30.0, 0.3, math.pi)},
        {"kind": "tube", "params": (5.0, 20.0, 30.0, 1.0, TWO_PI - 1e-9)},
        {"kind": "tube", "params": (10.0, 10.0 + 1e-6, 30.0, 0.0, TWO_PI)},
        {"kind": "tube", "params": (0.0, 3.0, 5000.0, 0.0, TWO_PI)},
        {"kind": "cone", "params": (0.0, 1e-3, 0.0, 20.0, 30.0, 0.0, TWO_PI)},
        {"kind": "cone", "params": (2.0, 20.0, 0.0, 1e-3, 30.0, 0.5, 2.0)},
        {"kind": "box", "params": (1e-3, 1e-3, 1e-3)},
        {"kind": "box", "params": (5000.0, 1.0, 5000.0)},
        {"kind": "trap", "params": ((20.0, 60.0 * DEG, 30.0 * DEG, 10.0, 5.0, 8.0, 20.0 * DEG, 10.0, 5.0, 8.0, 20.0 * DEG),)},
    ]

