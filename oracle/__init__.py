"""FP64 brute-force CPU oracle for walk on stars -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports, links or runs it, and it shares no code with them.

The arithmetic lives in ``wost_oracle.c`` (plain C, double precision,
brute-force queries, the walk of Alg. 1 in the paper's order); this module only
compiles that file with gcc and marshals numpy arrays through ctypes.

Parity status of the functions (what pins them, see tests/test_oracle_*.py):
  philox            published known-answer vectors (Salmon et al., SC'11)
  green_ball(_norm) App. A closed forms, quadrature of the ball integral
  source_radius     KS test against the radial CDF of the normalised G_B
  closest_dirichlet hand-derived distances on tiny shapes
  silhouette_distance  convex-from-inside (none), reflex vertex (closed form),
                    subdivision independence of a straight wall, 3D edge
  intersect_neumann hand-derived hits on segments / triangles
  neumann_sample    E[1/pdf] = measure of the Neumann boundary in the ball
  silhouette_distance_tol, intersect_neumann_tol
                    (test-only threshold brackets) reduce to the two
                    functions above at 0 and are monotone in the threshold
  solve / walk      exact harmonic and Poisson solutions (pure Dirichlet =
                    walk on spheres, mixed Dirichlet/Neumann, sources,
                    3D), arc harmonic measure (Poisson kernel of the disk),
                    1/sqrt(N) convergence

Boundary data and analytic solutions, and the pins that exercise each:
  data none         f absent in every source-free walk pin
  data analytic     every exact-solution walk pin below
  data per_corner   Poisson kernel of the disk (indicator g), cube around a
                    Neumann sphere (quad3 g and h), per-vertex equivalence
  data per_vertex   linear u on a square (2D) and on a cube with a Neumann
                    face (3D): exact; equal to per-corner walk for walk
  data grid         screened source on a grid (bilinear, clamped)
  double-sided      (App. B) slit square with g+ != g- (u = polar angle),
                    Neumann sheets inside a Dirichlet box (2D, 3D)
  fn zero           Poisson kernel of the disk
  fn exp_cos        pure Dirichlet disk, the 64-segment flower, convergence
  fn sin2x_cos3y    f = 13 u on a Dirichlet disk and with a Neumann half
  fn quad3          pure Dirichlet cube, cube around a Neumann sphere
  fn bump           -Lap u = 1 in 2D and 3D (sign and norm of the source)
  fn linear         square with Neumann sides, per-vertex pins, R13
  fn log_radial     annulus with a Neumann inner circle
  fn exp_plane      screened disks and cubes (Dirichlet, mixed, pure Neumann)
No function of the oracle is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wost_oracle.c")
_LIBPATH = os.path.join(_HERE, "liborc_wost.so")
_lib = None
_lock = threading.Lock()

DATA = {"none": 0, "per_vertex": 1, "per_corner": 2, "analytic": 3, "grid": 4}
FN = {"zero": 0, "exp_cos": 1, "sin2x_cos3y": 2, "quad3": 3, "bump": 4, "linear": 5, "log_radial": 6,
      "exp_plane": 7}
TRACE_COLS = ("x0", "x1", "x2", "onN", "dD", "dsil", "r", "hit", "t_boundary", "N", "S")

DEFAULT_OFFSET = 1e-6      # reading R4: relative ray-origin offset on the boundary
DEFAULT_VIS_TMAX = 1 - 1e-4  # reading R4: visibility ray end for the Neumann sample


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fused multiply-add)."""
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "wost_oracle.h"))):
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("values", C.POINTER(C.c_double)), ("fn", C.c_int),
                ("params", C.c_double * 8), ("origin", C.c_double * 3),
                ("spacing", C.c_double * 3), ("dims", C.c_int * 3)]


class _Params(C.Structure):
    _fields_ = [("epsilon", C.c_double), ("r_min", C.c_double), ("max_steps", C.c_int),
                ("seed", C.c_uint64), ("offset", C.c_double), ("vis_tmax", C.c_double),
                ("n_threads", C.c_int), ("sigma", C.c_double), ("screen_after", C.c_int)]


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIBPATH)
            P = C.c_void_p
            lib.orc_scene_new.restype = P
            lib.orc_scene_new.argtypes = [C.c_int, C.c_int, P, C.c_int, P, P, P, P, P]
            lib.orc_scene_free.argtypes = [P]
            lib.orc_scene_set_minus.argtypes = [P, P, P]
            lib.orc_scene_info.argtypes = [P, P]
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_closest_dirichlet.argtypes = [P, C.c_int64, P, P, P, P]
            lib.orc_silhouette_distance.argtypes = [P, C.c_int64, P, P, P, P]
            lib.orc_intersect_neumann.argtypes = [P, C.c_int64, P, P, P, P, P, P, P]
            lib.orc_silhouette_distance_tol.argtypes = [P, C.c_int64, P, P, C.c_double, P]
            lib.orc_intersect_neumann_tol.argtypes = [P, C.c_int64, P, P, P, P, C.c_double, P, P]
            lib.orc_neumann_sample.argtypes = [P, P, C.c_double, C.c_uint64, C.c_uint32,
                                               C.c_uint32, C.c_uint32, P, P, P, P]
            lib.orc_green_ball.restype = C.c_double
            lib.orc_green_ball.argtypes = [C.c_int, C.c_double, C.c_double]
            lib.orc_green_ball_norm.restype = C.c_double
            lib.orc_green_ball_norm.argtypes = [C.c_int, C.c_double]
            for nm in ("orc_bessel_i0e", "orc_bessel_i1e", "orc_bessel_k0e", "orc_bessel_k1e"):
                getattr(lib, nm).restype = C.c_double
                getattr(lib, nm).argtypes = [C.c_double]
            lib.orc_screened_green_ball.restype = C.c_double
            lib.orc_screened_green_ball.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
            lib.orc_screened_green_ball_norm.restype = C.c_double
            lib.orc_screened_green_ball_norm.argtypes = [C.c_int, C.c_double, C.c_double]
            lib.orc_screened_q.restype = C.c_double
            lib.orc_screened_q.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
            lib.orc_source_radius.restype = C.c_double
            lib.orc_source_radius.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
            lib.orc_solve.restype = C.c_int
            lib.orc_solve.argtypes = [P, C.c_int64, P, P, P, C.c_int, C.c_uint32, C.c_uint32, P, P, P, P, P, P]
            lib.orc_walk_trace.restype = C.c_int
            lib.orc_walk_trace.argtypes = [P, P, P, C.c_int, C.c_uint32, C.c_uint32, P, P,
                                           C.c_int, P, P]
            lib.orc_exact_u.argtypes = [C.c_int, C.c_int, P, C.c_int64, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _field(spec, keep):
    f = _Field()
    spec = spec or {"kind": "none"}
    f.kind = DATA[spec["kind"]]
    if spec["kind"] in ("per_vertex", "per_corner", "grid"):
        v = _d(spec["values"]).ravel()
        keep.append(v)
        f.values = v.ctypes.data_as(C.POINTER(C.c_double))
    if spec["kind"] == "analytic":
        f.fn = FN[spec["fn"]]
        for i, p in enumerate(spec.get("params", [])):
            f.params[i] = float(p)
    if spec["kind"] == "grid":
        for i, v in enumerate(spec["origin"]):
            f.origin[i] = float(v)
        for i, v in enumerate(spec["spacing"]):
            f.spacing[i] = float(v)
        for i, v in enumerate(spec["dims"]):
            f.dims[i] = int(v)
    return f


class Scene:
    """An oracle scene built from a scene dict (see the inputs module)."""

    def __init__(self, spec: dict):
        lib = _L()
        self.dim = int(spec["dim"])
        V = _d(spec["vertices"]).ravel()
        Pm = np.ascontiguousarray(spec["prims"], dtype=np.int32).ravel()
        Fl = np.ascontiguousarray(spec["flags"], dtype=np.uint8).ravel()
        keep = []
        g, h, f = (_field(spec.get(k), keep) for k in ("g", "h", "f"))
        self._h = lib.orc_scene_new(self.dim, len(V) // self.dim, _ptr(V), len(Pm) // self.dim,
                                    _ptr(Pm), _ptr(Fl), C.byref(g), C.byref(h), C.byref(f))
        if not self._h:
            raise ValueError("oracle rejected the scene")
        if "g_minus" in spec or "h_minus" in spec:
            gm, hm = (_field(spec.get(k), keep) for k in ("g_minus", "h_minus"))
            lib.orc_scene_set_minus(self._h, C.byref(gm), C.byref(hm))

    def info(self):
        out = np.zeros(8, np.int64)
        _L().orc_scene_info(self._h, _ptr(out))
        return dict(dim=int(out[0]), n_dirichlet=int(out[1]), n_neumann=int(out[2]),
                    n_silhouette=int(out[3]), n_nodes=int(out[4]))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_scene_free(self._h)
            self._h = None


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _L().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def green_ball(dim, rho, R):
    return _L().orc_green_ball(int(dim), float(rho), float(R))


def green_ball_norm(dim, R):
    return _L().orc_green_ball_norm(int(dim), float(R))


def source_radius(dim, R, u1, u2=0.5):
    return _L().orc_source_radius(int(dim), float(R), float(u1), float(u2))


def closest_dirichlet(scene: Scene, pts):
    x = _d(pts)
    n = len(x)
    d = np.zeros(n); xb = np.zeros((n, 3)); pr = np.zeros(n, np.int32)
    _L().orc_closest_dirichlet(scene._h, n, _ptr(x), _ptr(d), _ptr(xb), _ptr(pr))
    return d, xb[:, :scene.dim], pr


def silhouette_distance(scene: Scene, pts, rmax):
    x = _d(pts)
    n = len(x)
    rm = _d(np.broadcast_to(np.asarray(rmax, np.float64), (n,)))
    d = np.zeros(n); w = np.zeros(n, np.int32)
    _L().orc_silhouette_distance(scene._h, n, _ptr(x), _ptr(rm), _ptr(d), _ptr(w))
    return d, w


def intersect_neumann(scene: Scene, origins, dirs, tmax, skip=None):
    o = _d(origins); v = _d(dirs)
    n = len(o)
    tm = _d(np.broadcast_to(np.asarray(tmax, np.float64), (n,)))
    sk = None if skip is None else np.ascontiguousarray(np.broadcast_to(skip, (n,)), np.int32)
    hit = np.zeros(n, np.int32); t = np.zeros(n); pr = np.zeros(n, np.int32)
    _L().orc_intersect_neumann(scene._h, n, _ptr(o), _ptr(v), _ptr(tm), _ptr(sk), _ptr(hit),
                               _ptr(t), _ptr(pr))
    return hit.astype(bool), t, pr


def silhouette_distance_tol(scene: Scene, pts, rmax, tau):
    """Q.2 with the silhouette threshold moved to tau |v| (1 + |x|_inf)
    (tests only: brackets answers decided in single precision)."""
    x = _d(pts)
    n = len(x)
    rm = _d(np.broadcast_to(np.asarray(rmax, np.float64), (n,)))
    d = np.zeros(n)
    _L().orc_silhouette_distance_tol(scene._h, n, _ptr(x), _ptr(rm), float(tau), _ptr(d))
    return d


def intersect_neumann_tol(scene: Scene, origins, dirs, tmax, tol, skip=None):
    """Q.3 with the accepted segment-parameter / barycentric range widened
    by tol (tests only: brackets answers decided in single precision)."""
    o = _d(origins); v = _d(dirs)
    n = len(o)
    tm = _d(np.broadcast_to(np.asarray(tmax, np.float64), (n,)))
    sk = None if skip is None else np.ascontiguousarray(np.broadcast_to(skip, (n,)), np.int32)
    hit = np.zeros(n, np.int32); t = np.zeros(n)
    _L().orc_intersect_neumann_tol(scene._h, n, _ptr(o), _ptr(v), _ptr(tm), _ptr(sk), float(tol), _ptr(hit),
                                   _ptr(t))
    return hit.astype(bool), t


def neumann_sample(scene: Scene, x, r, seed=0, c0=0, c1=0, c2=0):
    xx = _d(x).ravel()
    z = np.zeros(3); nz = np.zeros(3); pdf = np.zeros(1); pr = np.zeros(1, np.int32)
    _L().orc_neumann_sample(scene._h, _ptr(xx), float(r), int(seed), int(c0), int(c1), int(c2),
                            _ptr(z), _ptr(nz), _ptr(pdf), _ptr(pr))
    return z[:scene.dim], nz[:scene.dim], float(pdf[0]), int(pr[0])


def _params(epsilon, r_min, max_steps, seed, offset, vis_tmax, threads, sigma=0.0, screen_after=0):
    p = _Params()
    p.sigma = float(sigma)
    p.screen_after = int(screen_after)
    p.epsilon = float(epsilon)
    p.r_min = float(epsilon if r_min is None else r_min)
    p.max_steps = int(max_steps)
    p.seed = int(seed)
    p.offset = float(offset)
    p.vis_tmax = float(vis_tmax)
    p.n_threads = int(threads)
    return p


def solve(scene: Scene, points, walks: int, epsilon: float, r_min=None, max_steps=1024, seed=0,
          normals=None, on_neumann=None, first_walk=0, offset=DEFAULT_OFFSET,
          vis_tmax=DEFAULT_VIS_TMAX, threads=0, per_walk=False, point_base=0, sigma=0.0,
          screen_after=0) -> dict:
    """Runs `walks` walks from every point; returns per-point FP64 statistics.
    Point i uses the random stream of point index point_base + i.  sigma > 0
    solves the screened equation -Lap u + sigma u = f from step screen_after
    on (App. A.2; the Tikhonov switch of Sec. 4.1)."""
    x = _d(points)
    n = len(x)
    nr = None if normals is None else _d(normals)
    on = None if on_neumann is None else np.ascontiguousarray(on_neumann, np.uint8)
    sm = np.zeros(n); sq = np.zeros(n)
    st = np.zeros(n, np.int64); cp = np.zeros(n, np.int64)
    pw = np.zeros(n * walks) if per_walk else None
    p = _params(epsilon, r_min, max_steps, seed, offset, vis_tmax, threads, sigma, screen_after)
    used = _L().orc_solve(scene._h, n, _ptr(x), _ptr(nr), _ptr(on), int(walks), int(first_walk),
                          int(point_base), C.byref(p), _ptr(sm), _ptr(sq), _ptr(st), _ptr(cp), _ptr(pw))
    mean = sm / walks
    var = np.maximum(sq / walks - mean**2, 0.0) * walks / max(walks - 1, 1)
    out = dict(mean=mean, se=np.sqrt(var / walks), sum=sm, sumsq=sq, steps=st, capped=cp,
               walks=walks, threads=used)
    if per_walk:
        out["per_walk"] = pw.reshape(n, walks)
    return out


def walk_trace(scene: Scene, x0, point_index=0, walk_index=0, epsilon=1e-3, r_min=None,
               max_steps=1024, seed=0, n0=None, on_neumann=False, offset=DEFAULT_OFFSET,
               vis_tmax=DEFAULT_VIS_TMAX, sigma=0.0, screen_after=0):
    """One walk with its per-step trace (rows of TRACE_COLS)."""
    x = _d(x0).ravel()
    nn = None if n0 is None else _d(n0).ravel()
    rows = np.zeros((max_steps, len(TRACE_COLS)))
    val = np.zeros(1); capped = np.zeros(1, np.int32)
    p = _params(epsilon, r_min, max_steps, seed, offset, vis_tmax, 1, sigma, screen_after)
    k = _L().orc_walk_trace(scene._h, _ptr(x), _ptr(nn), int(bool(on_neumann)), int(point_index),
                            int(walk_index), C.byref(p), _ptr(rows), max_steps, _ptr(val),
                            _ptr(capped))
    return float(val[0]), rows[:k], bool(capped[0])


def exact_u(dim, fn, params, pts):
    x = _d(pts)
    out = np.zeros(len(x))
    pr = np.zeros(8)
    pr[: len(params or [])] = params or []
    _L().orc_exact_u(int(dim), FN[fn], _ptr(pr), len(x), _ptr(x), _ptr(out))
    return out


def bessel_scaled(x):
    """(e^-x I0, e^-x I1, e^x K0, e^x K1) at each x > 0."""
    L = _L()
    return np.array([[L.orc_bessel_i0e(float(t)), L.orc_bessel_i1e(float(t)), L.orc_bessel_k0e(float(t)),
                      L.orc_bessel_k1e(float(t))] for t in np.ravel(x)])


def screened_green_ball(dim, rho, R, sigma):
    return _L().orc_screened_green_ball(int(dim), float(rho), float(R), float(sigma))


def screened_green_ball_norm(dim, R, sigma):
    return _L().orc_screened_green_ball_norm(int(dim), float(R), float(sigma))


def screened_q(dim, rho, R, sigma):
    return _L().orc_screened_q(int(dim), float(rho), float(R), float(sigma))
