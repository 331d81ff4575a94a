"""Seeded synthetic inputs for walk on stars: boundaries, boundary data and
evaluation points.

This module holds only input generation: geometry, exact test solutions and
point sets.  It contains none of the estimator's arithmetic, so both the CUDA
path and the CPU oracle may be fed from it.

The paper's own scenes (a CT-scanned toaster, a lizard mesh, a lung model,
Sec. 6.5) are not available; these generators produce inputs with their
shapes: slice-plane grids of evaluation points, boundaries of 1e3-1e6
elements with large Neumann regions, mixed boundary conditions.

A scene is a plain dict:
  dim       2 (line segments) or 3 (triangles)
  vertices  float32 [V, dim]
  prims     int32   [P, dim]   (2D: segment a->b, outward normal (t.y, -t.x);
                                3D: triangle a,b,c, outward normal (b-a)x(c-a))
  flags     uint8   [P]        0 = Dirichlet, 1 = Neumann
  g, h, f   field dicts:
            {"kind": "none"}
            {"kind": "analytic", "fn": name, "params": [..]}
            {"kind": "per_vertex", "values": float32 [V]}
            {"kind": "per_corner", "values": float32 [P, dim]}
            {"kind": "grid", "origin": [..], "spacing": [..], "dims": [..],
             "values": float32 (x fastest)}   (f only)
  exact     (fn, params) of the exact solution, when one is known

Analytic solution names: zero, exp_cos (e^x cos y), sin2x_cos3y,
quad3 (x^2 - y^2 + z/2), bump ((1-|x|^2)/(2 dim), source 1), linear
(p0 + p1 x + p2 y + p3 z), log_radial (2D p0 + p1 log|x-c|, 3D p0 + p1/|x-c|),
exp_plane (p0 exp(p1 x + p2 y + p3 z), which solves -Lap u + sigma u = 0 for
sigma = p1^2 + p2^2 + p3^2).
"""
from __future__ import annotations

import math

import numpy as np

FN_NAMES = ("zero", "exp_cos", "sin2x_cos3y", "quad3", "bump", "linear", "log_radial", "exp_plane")


# ---------------------------------------------------------------------------
# exact solutions (problem data for tests; the PDE is -Lap u = f)
# ---------------------------------------------------------------------------
def exact_u(fn: str, params, pts: np.ndarray) -> np.ndarray:
    """Exact solution u at points [N, dim] (float64)."""
    p = np.zeros(8)
    if params is not None:
        p[: len(params)] = params
    x = np.asarray(pts, dtype=np.float64)
    dim = x.shape[1]
    X, Y = x[:, 0], x[:, 1]
    Z = x[:, 2] if dim == 3 else np.zeros_like(X)
    if fn == "zero":
        return np.zeros_like(X)
    if fn == "exp_cos":
        return np.exp(X) * np.cos(Y)
    if fn == "sin2x_cos3y":
        return np.sin(2 * X) * np.cos(3 * Y)
    if fn == "quad3":
        return X * X - Y * Y + 0.5 * Z
    if fn == "bump":
        return (1.0 - (X * X + Y * Y + Z * Z)) / (2.0 * dim)
    if fn == "linear":
        return p[0] + p[1] * X + p[2] * Y + p[3] * Z
    if fn == "log_radial":
        c = np.array([p[2], p[3], p[4] if dim == 3 else 0.0])
        rho = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        return p[0] + p[1] * np.log(rho) if dim == 2 else p[0] + p[1] / rho
    if fn == "exp_plane":
        return p[0] * np.exp(p[1] * X + p[2] * Y + p[3] * Z)
    if fn == "polar_angle":
        return np.mod(np.arctan2(Y, X), 2 * np.pi)
    if fn == "crack_mode":
        return np.sqrt(np.hypot(X, Y)) * np.cos(np.mod(np.arctan2(Y, X), 2 * np.pi) / 2)
    raise ValueError(fn)


def exact_grad(fn: str, params, pts: np.ndarray) -> np.ndarray:
    p = np.zeros(8)
    if params is not None:
        p[: len(params)] = params
    x = np.asarray(pts, dtype=np.float64)
    dim = x.shape[1]
    X, Y = x[:, 0], x[:, 1]
    Z = x[:, 2] if dim == 3 else np.zeros_like(X)
    zero = np.zeros_like(X)
    if fn == "zero":
        g = (zero, zero, zero)
    elif fn == "exp_cos":
        g = (np.exp(X) * np.cos(Y), -np.exp(X) * np.sin(Y), zero)
    elif fn == "sin2x_cos3y":
        g = (2 * np.cos(2 * X) * np.cos(3 * Y), -3 * np.sin(2 * X) * np.sin(3 * Y), zero)
    elif fn == "quad3":
        g = (2 * X, -2 * Y, 0.5 + zero)
    elif fn == "bump":
        g = (-X / dim, -Y / dim, -Z / dim)
    elif fn == "linear":
        g = (p[1] + zero, p[2] + zero, p[3] + zero)
    elif fn == "log_radial":
        c = np.array([p[2], p[3], p[4] if dim == 3 else 0.0])
        d = np.stack([X - c[0], Y - c[1], Z - c[2]], 1)
        rho = np.linalg.norm(d, axis=1)
        s = p[1] / rho**2 if dim == 2 else -p[1] / rho**3
        g = (d[:, 0] * s, d[:, 1] * s, d[:, 2] * s)
    elif fn == "exp_plane":
        u = p[0] * np.exp(p[1] * X + p[2] * Y + p[3] * Z)
        g = (u * p[1], u * p[2], u * p[3])
    else:
        raise ValueError(fn)
    return np.stack(g[:dim], 1)


def prim_normals(scene: dict) -> np.ndarray:
    """Unit outward normals per primitive, float64 [P, dim]."""
    V = scene["vertices"].astype(np.float64)
    P = scene["prims"]
    if scene["dim"] == 2:
        t = V[P[:, 1]] - V[P[:, 0]]
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        return np.stack([t[:, 1], -t[:, 0]], 1)
    c = np.cross(V[P[:, 1]] - V[P[:, 0]], V[P[:, 2]] - V[P[:, 0]])
    return c / np.linalg.norm(c, axis=1, keepdims=True)


def per_vertex_fields(scene: dict, fn: str, params=None) -> dict:
    """g = u and h = du/dn as per-vertex values (h averaged over the Neumann
    primitives that share a vertex)."""
    V = scene["vertices"].astype(np.float64)
    g = exact_u(fn, params, V).astype(np.float32)
    n = prim_normals(scene)
    grad = exact_grad(fn, params, V)
    P = scene["prims"]
    acc = np.zeros(len(V))
    cnt = np.zeros(len(V))
    nmask = scene["flags"] == 1
    for k in range(scene["dim"]):
        idx = P[nmask, k]
        np.add.at(acc, idx, np.sum(grad[idx] * n[nmask], 1))
        np.add.at(cnt, idx, 1)
    h = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0.0).astype(np.float32)
    return {"g": {"kind": "per_vertex", "values": g}, "h": {"kind": "per_vertex", "values": h}}


def per_corner_fields(scene: dict, fn: str, params=None) -> dict:
    """g = u and h = grad u . n_face at every primitive corner (exact for a
    linear gradient on flat faces)."""
    V = scene["vertices"].astype(np.float64)
    P = scene["prims"]
    n = prim_normals(scene)
    g = np.stack([exact_u(fn, params, V[P[:, k]]) for k in range(scene["dim"])], 1)
    h = np.stack([np.sum(exact_grad(fn, params, V[P[:, k]]) * n, 1) for k in range(scene["dim"])], 1)
    return {"g": {"kind": "per_corner", "values": g.astype(np.float32)},
            "h": {"kind": "per_corner", "values": h.astype(np.float32)}}


def analytic(fn: str, params=None) -> dict:
    return {"kind": "analytic", "fn": fn, "params": list(params or [])}


def _make(dim, V, P, flags, fn, params=(), source=False, data="analytic"):
    sc = {"dim": dim, "vertices": np.ascontiguousarray(V, np.float32),
          "prims": np.ascontiguousarray(P, np.int32),
          "flags": np.ascontiguousarray(flags, np.uint8),
          "exact": (fn, list(params))}
    if data == "analytic":
        sc["g"] = analytic(fn, params)
        sc["h"] = analytic(fn, params)
    elif data == "per_vertex":
        sc.update(per_vertex_fields(sc, fn, params))
    elif data == "per_corner":
        sc.update(per_corner_fields(sc, fn, params))
    else:
        raise ValueError(data)
    sc["f"] = analytic(fn, params) if source else {"kind": "none"}
    return sc


# ---------------------------------------------------------------------------
# 2D building blocks
# ---------------------------------------------------------------------------
def closed_polyline(V: np.ndarray) -> np.ndarray:
    n = len(V)
    i = np.arange(n)
    return np.stack([i, (i + 1) % n], 1)


def point_in_polygon(pts: np.ndarray, poly: np.ndarray) -> np.ndarray:
    """Even-odd crossing test of points [N,2] against a closed polygon [M,2]."""
    x, y = pts[:, 0:1], pts[:, 1:2]
    a = poly[None, :, :]
    b = np.roll(poly, -1, axis=0)[None, :, :]
    cond = (a[..., 1] > y) != (b[..., 1] > y)
    with np.errstate(divide="ignore", invalid="ignore"):
        xc = a[..., 0] + (y - a[..., 1]) * (b[..., 0] - a[..., 0]) / (b[..., 1] - a[..., 1])
    cross = cond & (x < xc)
    return (np.count_nonzero(cross, axis=1) % 2) == 1


def _star_angles(poly: np.ndarray):
    """Vertex angles about the origin sorted ascending with the matching
    vertex order, if the polygon is star-shaped about the origin with its
    vertices in angular order (either orientation); else None."""
    th = np.arctan2(poly[:, 1], poly[:, 0])
    if np.any(np.hypot(poly[:, 0], poly[:, 1]) == 0):
        return None
    order = np.argsort(th, kind="stable")
    n = len(poly)
    # in angular order the polygon's successor relation must be a rotation
    pos = np.empty(n, int)
    pos[order] = np.arange(n)
    step = (pos[(np.arange(n) + 1) % n] - pos) % n
    if not (np.all(step == 1) or np.all(step == n - 1)):
        return None
    return th[order], poly[order]


def _inside_star(pts, th, V):
    """Inside test for a polygon star-shaped about the origin: the ray from
    the origin through p meets the boundary once, at the edge between the
    two vertices whose angles bracket p's; p is inside iff it is nearer."""
    n = len(V)
    tp = np.arctan2(pts[:, 1], pts[:, 0])
    k = (np.searchsorted(th, tp, side="right") - 1) % n
    a, b = V[k], V[(k + 1) % n]
    e = b - a
    rho = np.hypot(pts[:, 0], pts[:, 1])
    d = pts / np.maximum(rho, 1e-300)[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (a[:, 0] * e[:, 1] - a[:, 1] * e[:, 0]) / (d[:, 0] * e[:, 1] - d[:, 1] * e[:, 0])
    return rho < t


def _inside_chunked(pts, poly, chunk=4096):
    star = _star_angles(poly) if len(poly) > 256 else None
    if star is not None:
        return _inside_star(pts, *star)
    out = np.zeros(len(pts), bool)
    for s in range(0, len(pts), chunk):
        out[s:s + chunk] = point_in_polygon(pts[s:s + chunk], poly)
    return out


def polygon_distance(pts: np.ndarray, poly: np.ndarray, chunk=2048) -> np.ndarray:
    """Distance from points to a closed polygon's edges (input filtering)."""
    a = poly
    b = np.roll(poly, -1, axis=0)
    e = b - a
    ee = np.maximum(np.sum(e * e, 1), 1e-300)
    out = np.empty(len(pts))
    for s in range(0, len(pts), chunk):
        q = pts[s:s + chunk, None, :]
        t = np.clip(np.sum((q - a) * e, -1) / ee, 0, 1)
        c = a + t[..., None] * e
        out[s:s + chunk] = np.sqrt(np.min(np.sum((q - c) ** 2, -1), 1))
    return out


def regular_polygon(n: int, radius=1.0, center=(0.0, 0.0), cw=False) -> np.ndarray:
    th = 2 * np.pi * np.arange(n) / n
    V = np.stack([center[0] + radius * np.cos(th), center[1] + radius * np.sin(th)], 1)
    return V[::-1].copy() if cw else V


def disk_scene(n=256, fn="exp_cos", params=(), neumann=None, source=False, data="analytic"):
    """Regular n-gon approximating the unit circle.  `neumann` is a boolean
    mask over segments (default: all Dirichlet)."""
    V = regular_polygon(n)
    P = closed_polyline(V)
    flags = np.zeros(n, np.uint8) if neumann is None else np.asarray(neumann, np.uint8)
    return _make(2, V, P, flags, fn, params, source, data)


def square_scene(m=8, fn="linear", params=(0.0, 0.0, 1.0, 0.0), neumann_sides=("bottom", "top"),
                 data="analytic"):
    """Unit square [0,1]^2, CCW, each side split into m segments; the sides
    named in neumann_sides are Neumann."""
    pts, side = [], []
    s = np.arange(m) / m
    for name, (p0, p1) in (("bottom", ((0, 0), (1, 0))), ("right", ((1, 0), (1, 1))),
                           ("top", ((1, 1), (0, 1))), ("left", ((0, 1), (0, 0)))):
        p0, p1 = np.array(p0, float), np.array(p1, float)
        pts.append(p0[None] + s[:, None] * (p1 - p0)[None])
        side += [name] * m
    V = np.concatenate(pts)
    P = closed_polyline(V)
    flags = np.array([1 if sd in neumann_sides else 0 for sd in side], np.uint8)
    return _make(2, V, P, flags, fn, params, False, data)


def annulus_scene(n_out=256, n_in=128, r_in=0.3, a=1.0, b=0.5, data="analytic"):
    """Annulus r_in < |x| < 1: outer circle Dirichlet, inner circle Neumann
    (clockwise, so its normal points into the hole); u = a + b log|x|."""
    Vo = regular_polygon(n_out)
    Vi = regular_polygon(n_in, r_in, cw=True)
    V = np.concatenate([Vo, Vi])
    P = np.concatenate([closed_polyline(Vo), closed_polyline(Vi) + n_out])
    flags = np.concatenate([np.zeros(n_out), np.ones(n_in)]).astype(np.uint8)
    return _make(2, V, P, flags, "log_radial", (a, b, 0.0, 0.0, 0.0), False, data)


def flower_polygon(n=64) -> np.ndarray:
    th = 2 * np.pi * np.arange(n) / n
    r = 1 + 0.3 * np.sin(5 * th)
    return np.stack([r * np.cos(th), r * np.sin(th)], 1)


def sample_inside_2d(rng, n, outer, holes=(), box=None, margin=0.0):
    """Seeded rejection sampling of n points inside `outer` and outside
    every hole, at least `margin` away from all boundaries."""
    lo = outer.min(0) if box is None else np.array(box[0])
    hi = outer.max(0) if box is None else np.array(box[1])
    out = []
    while sum(len(o) for o in out) < n:
        c = lo + (hi - lo) * rng.random((4 * n, 2))
        ok = _inside_chunked(c, outer)
        for hpoly in holes:
            ok &= ~_inside_chunked(c, hpoly)
        c = c[ok]
        if margin > 0 and len(c):
            d = polygon_distance(c, outer)
            for hpoly in holes:
                d = np.minimum(d, polygon_distance(c, hpoly))
            c = c[d > margin]
        out.append(c)
    return np.concatenate(out)[:n].astype(np.float32)


# ---------------------------------------------------------------------------
# Workload 1: 64-segment flower, alternating D/N, u = e^x cos y
# ---------------------------------------------------------------------------
def config1(n_points=256, data="analytic", seed=1001):
    """64-vertex polygon r = 1 + 0.3 sin(5 theta), CCW; even segments
    Dirichlet (g = u), odd segments Neumann (h = du/dn), u = e^x cos y.
    256 points uniform inside; 512 walks; eps = r_min = 1e-3; cap 1024."""
    V = flower_polygon(64)
    P = closed_polyline(V)
    flags = (np.arange(64) % 2).astype(np.uint8)
    sc = _make(2, V, P, flags, "exp_cos", (), False, data)
    rng = np.random.default_rng(seed)
    sc["points"] = sample_inside_2d(rng, n_points, V, box=((-1.3, -1.3), (1.3, 1.3)))
    sc["walks"] = 512
    sc["epsilon"] = 1e-3
    sc["r_min"] = 1e-3
    sc["max_steps"] = 1024
    sc["name"] = "flower64_laplace_2d"
    return sc


# ---------------------------------------------------------------------------
# Workload 2: Koch snowflake with a random-walk hole, u = sin2x cos3y, f = 13u
# ---------------------------------------------------------------------------
def koch_snowflake(level=5, radius=1.0) -> np.ndarray:
    th = np.pi / 2 + 2 * np.pi * np.arange(3) / 3
    V = np.stack([radius * np.cos(th), radius * np.sin(th)], 1)  # CCW triangle
    rot = np.array([[math.cos(-math.pi / 3), -math.sin(-math.pi / 3)],
                    [math.sin(-math.pi / 3), math.cos(-math.pi / 3)]])
    for _ in range(level):
        a = V
        b = np.roll(V, -1, axis=0)
        d = (b - a) / 3.0
        p1 = a + d
        p3 = a + 2 * d
        p2 = p1 + d @ rot.T  # bump to the right of travel = outward for CCW
        V = np.stack([a, p1, p2, p3], 1).reshape(-1, 2)
    return V


def random_walk_hole(rng, n=1024, base=0.25, lo=0.15, hi=0.35, sigma=0.01) -> np.ndarray:
    steps = rng.normal(0.0, sigma, n)
    cs = np.cumsum(steps)
    cs -= np.arange(1, n + 1) / n * cs[-1]  # remove the linear drift: closes up
    rho = np.clip(base * np.exp(cs), lo, hi)
    th = 2 * np.pi * np.arange(n) / n
    V = np.stack([rho * np.cos(th), rho * np.sin(th)], 1)
    return V[::-1].copy()  # clockwise: normals point into the hole


def config2(grid=512, data="analytic", seed=2001, level=5, max_steps=65536):
    """Level-5 Koch snowflake (3072 segments, CCW) with a 1024-segment
    random-walk hole (CW, all Neumann).  The outer boundary is split in two
    contiguous halves by arc length from a seeded start vertex: Dirichlet,
    then Neumann.  u = sin 2x cos 3y, f = -Lap u = 13 u (analytic).  Points:
    interior cell centres of a grid x grid raster over the snowflake's
    bounding box.  256 walks; eps = r_min = 1e-4.  Walks here are long
    (thousands of steps: most of the boundary reflects), so the step cap is
    65536 rather than 1024, which would stop about half of them."""
    rng = np.random.default_rng(seed)
    outer = koch_snowflake(level)
    hole = random_walk_hole(rng)
    no, nh = len(outer), len(hole)
    start = int(rng.integers(no))
    outer = np.roll(outer, -start, axis=0)
    seg_len = np.linalg.norm(np.roll(outer, -1, axis=0) - outer, axis=1)
    arc = np.cumsum(seg_len) - 0.5 * seg_len
    oflags = (arc > 0.5 * seg_len.sum()).astype(np.uint8)
    V = np.concatenate([outer, hole])
    P = np.concatenate([closed_polyline(outer), closed_polyline(hole) + no])
    flags = np.concatenate([oflags, np.ones(nh, np.uint8)])
    sc = _make(2, V, P, flags, "sin2x_cos3y", (), True, data)
    lo, hi = outer.min(0), outer.max(0)
    cs = (np.arange(grid) + 0.5) / grid
    gx, gy = np.meshgrid(lo[0] + cs * (hi[0] - lo[0]), lo[1] + cs * (hi[1] - lo[1]), indexing="xy")
    pts = np.stack([gx.ravel(), gy.ravel()], 1)
    ok = _inside_chunked(pts, outer) & ~_inside_chunked(pts, hole)
    sc["points"] = pts[ok].astype(np.float32)
    sc["walks"] = 256
    sc["epsilon"] = 1e-4
    sc["r_min"] = 1e-4
    sc["max_steps"] = max_steps
    sc["name"] = f"koch{level}_hole_poisson_2d_grid{grid}"
    return sc


# ---------------------------------------------------------------------------
# 3D building blocks
# ---------------------------------------------------------------------------
def cube_mesh(m=32, half=1.0):
    """Axis-aligned cube [-half, half]^3, each face an m x m grid of quads
    split into 2 triangles, outward normals.  Returns V, P."""
    Vs, Ps = [], []
    off = 0
    g = np.linspace(-half, half, m + 1)
    A, B = np.meshgrid(g, g, indexing="ij")
    for axis in range(3):
        for sign in (-1.0, 1.0):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            V = np.zeros(((m + 1) ** 2, 3))
            V[:, axis] = sign * half
            V[:, u_ax] = A.ravel()
            V[:, v_ax] = B.ravel()
            idx = np.arange((m + 1) ** 2).reshape(m + 1, m + 1)
            a = idx[:-1, :-1].ravel(); b = idx[1:, :-1].ravel()
            c = idx[1:, 1:].ravel(); d = idx[:-1, 1:].ravel()
            T = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)])
            # orient outward: (b-a)x(c-a) along +sign*axis
            e = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
            flip = e[:, axis] * sign < 0
            T[flip] = T[flip][:, [0, 2, 1]]
            Vs.append(V); Ps.append(T + off); off += len(V)
    return weld(np.concatenate(Vs), np.concatenate(Ps))


def weld(V: np.ndarray, P: np.ndarray, decimals=9):
    """Merge coincident vertices so that shared edges are shared indices."""
    key = np.round(V, decimals)
    U, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.ravel()
    first = np.full(len(U), -1)
    first[inv[::-1]] = np.arange(len(V))[::-1]
    return V[first], inv[P]


def _hash3(ix, iy, iz, seed):
    h = (ix.astype(np.uint64) * np.uint64(0x8DA6B343) ^ iy.astype(np.uint64) * np.uint64(0xD8163841)
         ^ iz.astype(np.uint64) * np.uint64(0xCB1AB31F) ^ np.uint64(seed) * np.uint64(0x9E3779B1))
    h &= np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(15)
    h = (h * np.uint64(0x2C1B3C6D)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(12)
    h = (h * np.uint64(0x297A2D39)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(15)
    return h.astype(np.float64) / 4294967295.0 * 2.0 - 1.0


def value_noise(p: np.ndarray, seed: int, octaves=3, freq=4.0, gain=0.5) -> np.ndarray:
    """Fractal value noise in about [-1, 1]: hashed lattice values,
    quintic-smoothed trilinear interpolation, summed over octaves."""
    total = np.zeros(len(p))
    amp, norm = 1.0, 0.0
    for o in range(octaves):
        q = p * freq * (2 ** o)
        i0 = np.floor(q).astype(np.int64)
        f = q - i0
        w = f * f * f * (f * (f * 6 - 15) + 10)
        acc = np.zeros(len(p))
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    val = _hash3(i0[:, 0] + dx + 1000, i0[:, 1] + dy + 1000, i0[:, 2] + dz + 1000, seed + o)
                    wt = ((w[:, 0] if dx else 1 - w[:, 0]) * (w[:, 1] if dy else 1 - w[:, 1])
                          * (w[:, 2] if dz else 1 - w[:, 2]))
                    acc += wt * val
        total += amp * acc
        norm += amp
        amp *= gain
    return total / norm


def torus_mesh(nu=500, nv=200, R=0.5, r=0.2, amp=0.03, seed=3001, inward=True):
    """Torus about z with nu x nv quads (2 nu nv triangles), displaced along
    the analytic normal by amp * value_noise.  inward=True orients the
    triangle normals into the solid torus (outward for the domain around
    it).  Returns V, P and a function giving the surface tube radius."""
    th = 2 * np.pi * np.arange(nu) / nu
    ph = 2 * np.pi * np.arange(nv) / nv
    T, PH = np.meshgrid(th, ph, indexing="ij")
    n = np.stack([np.cos(PH) * np.cos(T), np.cos(PH) * np.sin(T), np.sin(PH)], -1).reshape(-1, 3)
    c = np.stack([R * np.cos(T), R * np.sin(T), np.zeros_like(T)], -1).reshape(-1, 3)
    base = c + r * n
    disp = amp * value_noise(base, seed)
    V = base + disp[:, None] * n
    idx = np.arange(nu * nv).reshape(nu, nv)
    a = idx.ravel()
    b = np.roll(idx, -1, axis=0).ravel()
    cc = np.roll(np.roll(idx, -1, axis=0), -1, axis=1).ravel()
    d = np.roll(idx, -1, axis=1).ravel()
    Tri = np.concatenate([np.stack([a, b, cc], 1), np.stack([a, cc, d], 1)])
    e = np.cross(V[Tri[:, 1]] - V[Tri[:, 0]], V[Tri[:, 2]] - V[Tri[:, 0]])
    centroid = V[Tri].mean(1)
    ring = centroid.copy()
    ring[:, 2] = 0
    ring = R * ring / np.linalg.norm(ring, axis=1, keepdims=True)
    out_of_tube = np.sum(e * (centroid - ring), 1) > 0
    flip = out_of_tube if inward else ~out_of_tube
    Tri[flip] = Tri[flip][:, [0, 2, 1]]

    def tube_radius(q):
        tq = np.arctan2(q[:, 1], q[:, 0])
        ringq = np.stack([R * np.cos(tq), R * np.sin(tq), np.zeros(len(q))], 1)
        dq = q - ringq
        rho = np.linalg.norm(dq, axis=1)
        nq = dq / np.maximum(rho, 1e-12)[:, None]
        bq = ringq + r * nq
        return rho, r + amp * value_noise(bq, seed)

    return V, Tri, tube_radius


def config3(grid=578, data="per_corner", seed=3001, nu=500, nv=200, cube_m=32, margin=2e-3):
    """Cube [-1,1]^3 (6 x 32 x 32 x 2 = 12,288 Dirichlet triangles) around a
    noisy torus (R = 0.5, r = 0.2, 500 x 200 x 2 = 200,000 Neumann
    triangles, displaced by 0.03 value noise), u = x^2 - y^2 + z/2.
    Points: the planes x=0, y=0, z=0, each a grid x grid raster of [-1,1]^2,
    minus duplicates and points inside the torus (with a margin).
    128 walks; eps = r_min = 1e-3; cap 1024."""
    Vc, Pc = cube_mesh(cube_m)
    Vt, Pt, tube_radius = torus_mesh(nu, nv, seed=seed)
    V = np.concatenate([Vc, Vt])
    P = np.concatenate([Pc, Pt + len(Vc)])
    flags = np.concatenate([np.zeros(len(Pc)), np.ones(len(Pt))]).astype(np.uint8)
    sc = _make(3, V, P, flags, "quad3", (), False, data)
    s = (np.arange(grid) + 0.5) / grid * 2 - 1
    A, B = np.meshgrid(s, s, indexing="ij")
    A, B = A.ravel(), B.ravel()
    Z0 = np.zeros_like(A)
    pts = np.concatenate([np.stack([Z0, A, B], 1), np.stack([A, Z0, B], 1), np.stack([A, B, Z0], 1)])
    pts = np.unique(pts.astype(np.float32), axis=0).astype(np.float64)
    rho, rs = tube_radius(pts)
    pts = pts[rho > rs + margin]
    sc["points"] = pts.astype(np.float32)
    sc["walks"] = 128
    sc["epsilon"] = 1e-3
    sc["r_min"] = 1e-3
    sc["max_steps"] = 1024
    sc["name"] = f"cube{cube_m}_torus{nu}x{nv}_laplace_3d_grid{grid}"
    return sc


def sphere_mesh(n_lat=16, n_lon=32, radius=1.0, center=(0, 0, 0), inward=False):
    """UV sphere (closed), outward normals unless inward=True."""
    V = [[0, 0, radius], [0, 0, -radius]]
    for i in range(1, n_lat):
        t = np.pi * i / n_lat
        for j in range(n_lon):
            p = 2 * np.pi * j / n_lon
            V.append([radius * np.sin(t) * np.cos(p), radius * np.sin(t) * np.sin(p), radius * np.cos(t)])
    V = np.array(V) + np.array(center)
    ring = lambda i, j: 2 + (i - 1) * n_lon + (j % n_lon)
    T = []
    for j in range(n_lon):
        T.append([0, ring(1, j), ring(1, j + 1)])
        T.append([1, ring(n_lat - 1, j + 1), ring(n_lat - 1, j)])
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            a, b, c, d = ring(i, j), ring(i + 1, j), ring(i + 1, j + 1), ring(i, j + 1)
            T.append([a, b, c]); T.append([a, c, d])
    T = np.array(T)
    e = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    outward = np.sum(e * (V[T].mean(1) - np.array(center)), 1) > 0
    flip = outward if inward else ~outward
    T[flip] = T[flip][:, [0, 2, 1]]
    return V, T


def box_sphere_scene(m=4, n_lat=12, n_lon=24, r_in=0.4, fn="quad3", params=(), data="per_corner"):
    """Cube [-1,1]^3 (Dirichlet) around a Neumann sphere of radius r_in
    whose normals point into the sphere (out of the domain)."""
    Vc, Pc = cube_mesh(m)
    Vs, Ps = sphere_mesh(n_lat, n_lon, r_in, inward=True)
    V = np.concatenate([Vc, Vs])
    P = np.concatenate([Pc, Ps + len(Vc)])
    flags = np.concatenate([np.zeros(len(Pc)), np.ones(len(Ps))]).astype(np.uint8)
    return _make(3, V, P, flags, fn, params, False, data)


def cube_scene(m=4, fn="quad3", params=(), source=False, data="analytic", neumann_faces=()):
    """Cube [-1,1]^3; faces listed in neumann_faces (0..5 = -x,+x,-y,+y,-z,+z)
    are Neumann."""
    V, P = cube_mesh(m)
    per_face = 2 * m * m
    face = np.arange(len(P)) // per_face
    flags = np.isin(face, list(neumann_faces)).astype(np.uint8)
    return _make(3, V, P, flags, fn, params, source, data)


def ball_points(rng, n, dim, radius):
    x = rng.normal(size=(n, dim))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / dim)
    return (x * r[:, None]).astype(np.float32)


# ---------------------------------------------------------------------------
# Double-sided boundaries (App. B): a slit and thin Neumann sheets
# ---------------------------------------------------------------------------
def _square_loop(m):
    """Vertices of the square [-1,1]^2, CCW, m segments per side, starting at
    (1, 0) (so that (1, 0) is a vertex)."""
    t = np.arange(4 * m) / (4 * m)
    pts = []
    for k in range(4 * m):
        # perimeter parameter from (1, 0) going up the right side
        s = 8.0 * t[k]
        if s < 1:
            pts.append((1.0, s))
        elif s < 3:
            pts.append((1.0 - (s - 1), 1.0))
        elif s < 5:
            pts.append((-1.0, 1.0 - (s - 3)))
        elif s < 7:
            pts.append((-1.0 + (s - 5), -1.0))
        else:
            pts.append((1.0, -1.0 + (s - 7)))
    return np.array(pts)


def polar_angle(pts):
    """Angle in [0, 2 pi) measured from the positive x axis: harmonic off
    the cut along the positive x axis."""
    return np.mod(np.arctan2(pts[:, 1], pts[:, 0]), 2 * np.pi)


def slit_square_scene(m=16, n_slit=16):
    """The square [-1,1]^2 with a slit from (0, 0) to (1, 0): a double-sided
    Dirichlet segment chain (flag 2).  u = the polar angle in [0, 2 pi),
    harmonic in the slit square; it is 0 on the slit's upper side and 2 pi
    on its lower side.  The slit runs along +x, so its normal n+ = (0, -1):
    its + side (the one n+ points away from) is the upper one, g+ = 0,
    g- = 2 pi.  Box data per corner, each segment on its own branch of the
    angle (the right side's segments above and below (1, 0) differ)."""
    Vb = _square_loop(m)
    nb = len(Vb)
    xs = np.linspace(0.0, 1.0, n_slit + 1)
    Vs = np.c_[xs, np.zeros_like(xs)]
    V = np.concatenate([Vb, Vs])
    Pb = closed_polyline(Vb)
    Ps = np.c_[np.arange(n_slit), np.arange(1, n_slit + 1)] + nb
    P = np.concatenate([Pb, Ps])
    flags = np.concatenate([np.zeros(len(Pb)), np.full(n_slit, 2)]).astype(np.uint8)
    mid = 0.5 * (V[P[:, 0]] + V[P[:, 1]])
    th_mid = polar_angle(mid)
    g = np.zeros((len(P), 2))
    for k in range(2):
        c = V[P[:, k]]
        d = np.arctan2(c[:, 1], c[:, 0]) - th_mid
        g[:, k] = th_mid + (d + np.pi) % (2 * np.pi) - np.pi  # the corner on its segment's branch
    ns = len(Pb)
    g[ns:] = 0.0
    gm = np.zeros_like(g)
    gm[ns:] = 2 * np.pi
    return {"dim": 2, "vertices": V.astype(np.float32), "prims": P.astype(np.int32), "flags": flags,
            "g": {"kind": "per_corner", "values": g.astype(np.float32)},
            "g_minus": {"kind": "per_corner", "values": gm.astype(np.float32)},
            "h": {"kind": "none"}, "f": {"kind": "none"}, "exact": ("polar_angle", [])}


def crack_square_scene(m=16, n_slit=16):
    """The square [-1,1]^2 with a crack from (0, 0) to (1, 0): a
    double-sided Neumann segment chain (flag 3) with zero flux on both
    sides.  u = sqrt(rho) cos(theta / 2), theta in [0, 2 pi), is harmonic off
    the crack with zero normal derivative on both of its sides, and jumps
    from sqrt(rho) above to -sqrt(rho) below: a walk that crossed the crack
    would pick up the other side's values.  Dirichlet data on the box per
    corner, each segment on its own branch of theta."""
    sc = slit_square_scene(m, n_slit)
    V, P = sc["vertices"].astype(np.float64), sc["prims"]
    ns = len(P) - n_slit
    theta = sc["g"]["values"].astype(np.float64)  # per-corner angle on each box segment's branch
    rho = np.stack([np.hypot(V[P[:, k], 0], V[P[:, k], 1]) for k in range(2)], 1)
    g = np.sqrt(rho) * np.cos(theta / 2)
    g[ns:] = 0.0
    flags = sc["flags"].copy()
    flags[ns:] = 3
    return {"dim": 2, "vertices": sc["vertices"], "prims": P, "flags": flags,
            "g": {"kind": "per_corner", "values": g.astype(np.float32)},
            "h": {"kind": "per_corner", "values": np.zeros((len(P), 2), np.float32)},
            "f": {"kind": "none"}, "exact": ("crack_mode", [])}


def sheet_square_scene(m=8, n_sheet=16, y0=0.1, half=0.5, params=(0.5, 0.3, 1.5, 0.0), data="analytic"):
    """The Dirichlet square [-1,1]^2 with a double-sided Neumann sheet (flag
    3) from (-half, y0) to (half, y0) inside, u linear (harmonic).  The sheet
    runs along +x: n+ = (0, -1), h+ = du/dn+ = -p2, h- = +p2.  data:
    "analytic", or "per_corner" with h- given ("per_corner_minus") or left
    NONE (then h- = -h+)."""
    Vb = _square_loop(m)
    xs = np.linspace(-half, half, n_sheet + 1)
    Vs = np.c_[xs, np.full_like(xs, y0)]
    V = np.concatenate([Vb, Vs])
    Pb = closed_polyline(Vb)
    Ps = np.c_[np.arange(n_sheet), np.arange(1, n_sheet + 1)] + len(Vb)
    P = np.concatenate([Pb, Ps])
    flags = np.concatenate([np.zeros(len(Pb)), np.full(n_sheet, 3)]).astype(np.uint8)
    sc = _make(2, V, P, flags, "linear", params, False, "analytic" if data == "analytic" else "per_corner")
    if data == "per_corner_minus":
        h = sc["h"]["values"].copy()
        sc["h_minus"] = {"kind": "per_corner", "values": (-h).astype(np.float32)}
        sc["h_minus"]["values"][: len(Pb)] = 0.0
    return sc


def plate_cube_scene(m=3, k=4, z0=0.1, half=0.5, params=(0.5, 0.3, -0.4, 1.5)):
    """The Dirichlet cube [-1,1]^3 with a double-sided Neumann square plate
    (flag 3) at z = z0 over [-half, half]^2, k x k quads, u linear
    (analytic data)."""
    Vc, Pc = cube_mesh(m)
    g = np.linspace(-half, half, k + 1)
    A, B = np.meshgrid(g, g, indexing="ij")
    Vp = np.c_[A.ravel(), B.ravel(), np.full(A.size, z0)]
    idx = np.arange((k + 1) ** 2).reshape(k + 1, k + 1)
    a = idx[:-1, :-1].ravel(); b = idx[1:, :-1].ravel(); c = idx[1:, 1:].ravel(); d = idx[:-1, 1:].ravel()
    Pp = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)]) + len(Vc)
    V = np.concatenate([Vc, Vp])
    P = np.concatenate([Pc, Pp])
    flags = np.concatenate([np.zeros(len(Pc)), np.full(len(Pp), 3)]).astype(np.uint8)
    return _make(3, V, P, flags, "linear", params, False, "analytic")


# ---------------------------------------------------------------------------
# Neumann-dominated stress scene: the "keyhole" of the paper's limitations
# ---------------------------------------------------------------------------
def keyhole_scene(seg=0.05, gap=0.1, window=0.4, n_points=64, seed=81):
    """Two 2 x 2 rooms joined by a corridor 0.4 long and `gap` wide; every
    wall is Neumann except a window of height `window` in the far wall of
    the right room (Dirichlet).  u = x (harmonic; h = n_x on every wall).
    Points uniform in the left room: a walk must find the corridor and then
    the window, reflecting off Neumann walls all the way (the paper's
    keyhole regime, Sec. 7, with mean walks of hundreds of steps)."""
    g, w = gap / 2, window / 2
    corners = [(-2, -1), (0, -1), (0, -g), (0.4, -g), (0.4, -1), (2.4, -1), (2.4, -w), (2.4, w), (2.4, 1),
               (0.4, 1), (0.4, g), (0, g), (0, 1), (-2, 1)]
    V, dirichlet = [], []
    for k in range(len(corners)):
        a = np.array(corners[k], float)
        b = np.array(corners[(k + 1) % len(corners)], float)
        n = max(1, int(np.ceil(np.linalg.norm(b - a) / seg)))
        for i in range(n):
            V.append(a + (b - a) * i / n)
            dirichlet.append(k == 6)  # the window (2.4, -w) -> (2.4, w)
    V = np.array(V)
    P = closed_polyline(V)
    flags = (~np.array(dirichlet)).astype(np.uint8)
    sc = _make(2, V, P, flags, "linear", (0.0, 1.0, 0.0, 0.0), False, "analytic")
    rng = np.random.default_rng(seed)
    sc["points"] = np.c_[rng.uniform(-1.9, -0.1, n_points), rng.uniform(-0.9, 0.9, n_points)].astype(np.float32)
    sc["walks"], sc["epsilon"], sc["r_min"], sc["max_steps"] = 256, 1e-3, 1e-3, 1 << 20
    sc["name"] = "keyhole_neumann_2d"
    return sc


# ---------------------------------------------------------------------------
# Workload 4: many scenes of uneven size, point count and walk count
# ---------------------------------------------------------------------------
def radial_polygon(n, rng, base=1.0, amp=0.25, lobes=5, rough=0.03):
    th = 2 * np.pi * np.arange(n) / n
    k = np.arange(1, 9)
    ph = rng.uniform(0, 2 * np.pi, len(k))
    noise = np.sum(np.sin(np.outer(th, k) + ph) / k, 1)
    r = base * (1 + amp * np.sin(lobes * th) + rough * noise / 2.7)
    return np.stack([r * np.cos(th), r * np.sin(th)], 1)


def batched_scene(i, n_prims, dim, d_frac, n_points, walks, seed):
    """One scene of the batched workload: about n_prims primitives, a
    contiguous Dirichlet fraction d_frac, n_points evaluation points."""
    rng = np.random.default_rng(seed)
    if dim == 2:
        n_hole = max(16, n_prims // 4)
        n_out = max(32, n_prims - n_hole)
        outer = radial_polygon(n_out, rng)
        hole = random_walk_hole(rng, n_hole, base=0.3, lo=0.2, hi=0.4, sigma=0.5 / np.sqrt(n_hole))
        seg = np.linalg.norm(np.roll(outer, -1, axis=0) - outer, axis=1)
        arc = np.cumsum(seg) - 0.5 * seg
        total = seg.sum() + np.linalg.norm(np.roll(hole, -1, axis=0) - hole, axis=1).sum()
        oflags = (arc > d_frac * total).astype(np.uint8)  # Dirichlet first along the outer arc
        V = np.concatenate([outer, hole])
        P = np.concatenate([closed_polyline(outer), closed_polyline(hole) + n_out])
        flags = np.concatenate([oflags, np.ones(n_hole, np.uint8)])
        sc = _make(2, V, P, flags, "sin2x_cos3y", (), True, "analytic")
        sc["points"] = sample_inside_2d(rng, n_points, outer, holes=(hole,))
    else:
        m = 8
        n_t = max(200, n_prims - 6 * 2 * m * m)
        nv = max(8, int(np.sqrt(n_t / 2 / 2.5)))
        nu = max(8, int(n_t / 2 / nv))
        Vc, Pc = cube_mesh(m)
        Vt, Pt, tube_radius = torus_mesh(nu, nv, seed=seed)
        cz = Vt[Pt].mean(1)[:, 2]
        # Dirichlet: the cube plus the torus below a z threshold
        want_d = d_frac * (len(Pc) + len(Pt)) - len(Pc)
        zt = np.quantile(cz, np.clip(want_d / len(Pt), 0, 1)) if want_d > 0 else -np.inf
        tflags = (cz >= zt).astype(np.uint8)
        V = np.concatenate([Vc, Vt])
        P = np.concatenate([Pc, Pt + len(Vc)])
        flags = np.concatenate([np.zeros(len(Pc), np.uint8), tflags])
        sc = _make(3, V, P, flags, "quad3", (), False, "per_corner")
        pts = []
        while sum(len(p) for p in pts) < n_points:
            q = rng.uniform(-0.95, 0.95, (4 * n_points + 16, 3))
            rho, rs = tube_radius(q)
            pts.append(q[rho > rs + 2e-3])
        sc["points"] = np.concatenate(pts)[:n_points].astype(np.float32)
    sc["walks"] = int(walks)
    sc["epsilon"] = 1e-3
    sc["r_min"] = 1e-3
    sc["max_steps"] = 16384
    sc["seed"] = int(seed)
    sc["name"] = f"batch{i}_{dim}d_{len(sc['prims'])}p"
    return sc


def config4(n_scenes=64, seed=4001, prims=(1e3, 5e5), points=(1, 1e6), walks=(16, 4096), max_scene=None):
    """The batched workload: n_scenes scenes, dimension by coin flip,
    primitive counts, point counts and walks per point log-uniform over the
    given ranges, Dirichlet fraction U(0.2, 0.8).  Returns scene dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        dim = 2 if rng.random() < 0.5 else 3
        n_p = int(np.exp(rng.uniform(np.log(prims[0]), np.log(prims[1]))))
        n_x = int(np.exp(rng.uniform(np.log(points[0]), np.log(points[1]))))
        w = int(np.exp(rng.uniform(np.log(walks[0]), np.log(walks[1]))))
        f = rng.uniform(0.2, 0.8)
        if max_scene:
            n_p = min(n_p, int(max_scene))
        out.append(batched_scene(i, n_p, dim, f, max(1, n_x), max(1, w), seed * 100 + i))
    return out


# ---------------------------------------------------------------------------
# Workload 5: resident 3D scenes and a Poisson stream of requests
# ---------------------------------------------------------------------------
def config5_scenes(n_scenes=8, total=5_000_000, lo=2e4, hi=2e6, seed=5001):
    """Resident 3D scenes (cube + noisy torus like workload 3) whose torus
    triangle counts are log-uniform in [lo, hi], rescaled to sum to about
    `total`."""
    rng = np.random.default_rng(seed)
    t = np.exp(rng.uniform(np.log(lo), np.log(hi), n_scenes))
    t = t * total / t.sum()
    out = []
    for i, n_t in enumerate(t):
        nv = max(8, int(np.sqrt(n_t / 2 / 2.5)))
        nu = max(8, int(n_t / 2 / nv))
        sc = config3(grid=4, nu=nu, nv=nv, seed=seed * 10 + i)
        sc["tube"] = (0.5, 0.2, 0.03, seed * 10 + i)
        sc["name"] = f"serve{i}_torus{nu}x{nv}"
        out.append(sc)
    return out


def plane_points(rng, n, tube):
    """n points uniform on a random plane slice of [-1,1]^3 (unit normal,
    offset U(-0.8, 0.8)), outside the torus of `tube` = (R, r, amp, seed)."""
    R, r, amp, tseed = tube
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    off = rng.uniform(-0.8, 0.8)
    a = np.cross(nrm, [1.0, 0, 0] if abs(nrm[0]) < 0.9 else [0, 1.0, 0])
    a /= np.linalg.norm(a)
    b = np.cross(nrm, a)
    out = []
    got = 0
    while got < n:
        uv = rng.uniform(-1.8, 1.8, (4 * n + 64, 2))
        q = off * nrm + uv[:, :1] * a + uv[:, 1:] * b
        q = q[np.all(np.abs(q) < 0.97, axis=1)]
        tq = np.arctan2(q[:, 1], q[:, 0])
        ring = np.stack([R * np.cos(tq), R * np.sin(tq), np.zeros(len(q))], 1)
        dq = q - ring
        rho = np.linalg.norm(dq, axis=1)
        bq = ring + r * dq / np.maximum(rho, 1e-12)[:, None]
        rs = r + amp * value_noise(bq, tseed)
        q = q[rho > rs + 2e-3]
        out.append(q)
        got += len(q)
    return np.concatenate(out)[:n].astype(np.float32)


def config5_requests(duration_s=600.0, rate=200.0, n_scenes=8, seed=5002, points=(1e3, 2.56e5)):
    """Poisson arrivals: (time, scene id, n_points, target SE, seed)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        n = int(np.exp(rng.uniform(np.log(points[0]), np.log(points[1]))))
        out.append({"t": t, "scene": int(rng.integers(n_scenes)), "n_points": n,
                    "target_se": 1e-2 if rng.random() < 0.5 else 1e-3, "seed": int(rng.integers(1 << 62))})
    return out
