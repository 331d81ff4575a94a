"""Python binding of libwost (include/wost.h): argument marshalling only.

Every function named ``wost_*`` here calls the C function of the same name;
all computation happens in the CUDA library.  If the library is missing or
cannot be loaded this module raises -- there is no fallback.

Arrays: host inputs are numpy arrays; device inputs/outputs are torch CUDA
tensors (PyTorch only provides device memory and streams).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libwost.so")
_lib = None
_lock = threading.Lock()

# status codes (include/wost.h)
OK, ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_BUDGET, ERR_CUDA, ERR_TIMEOUT, ERR_CANCELLED, ERR_INTERNAL = range(8)
STATUS_NAMES = ["OK", "INVALID_ARG", "OUT_OF_MEMORY", "BUDGET", "CUDA", "TIMEOUT", "CANCELLED", "INTERNAL"]
DATA = {"none": 0, "per_vertex": 1, "per_corner": 2, "analytic": 3, "grid": 4}
FN = {"zero": 0, "exp_cos": 1, "sin2x_cos3y": 2, "quad3": 3, "bump": 4, "linear": 5, "log_radial": 6,
      "exp_plane": 7}
ABI_VERSION = 4  # WOST_ABI_VERSION of the header these structures mirror
MEM_HOST, MEM_DEVICE = 0, 1
KERNEL = {"plain": 0, "persistent": 1, "counting": 2, "resumable": 3}
COUNT_NAMES = ("q1", "q2", "q3", "q4", "vis")


class WostError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class wost_field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("values", C.POINTER(C.c_float)), ("fn", C.c_int32),
                ("params", C.c_float * 8), ("origin", C.c_float * 3), ("spacing", C.c_float * 3),
                ("dims", C.c_int32 * 3)]


class wost_scene_desc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vertices", C.c_int64), ("vertices", C.POINTER(C.c_float)),
                ("n_prims", C.c_int64), ("prims", C.POINTER(C.c_int32)), ("flags", C.POINTER(C.c_uint8)),
                ("g", wost_field), ("h", wost_field), ("f", wost_field), ("device", C.c_int32),
                ("leaf_size", C.c_int32), ("g_minus", wost_field), ("h_minus", wost_field),
                ("silhouette_split", C.c_int32)]


class wost_scene_info(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_dirichlet", C.c_int64), ("n_neumann", C.c_int64),
                ("n_silhouette", C.c_int64), ("n_dropped", C.c_int64), ("nodes_dirichlet", C.c_int64),
                ("nodes_neumann", C.c_int64), ("nodes_silhouette", C.c_int64), ("depth_dirichlet", C.c_int32),
                ("depth_neumann", C.c_int32), ("depth_silhouette", C.c_int32), ("device_bytes", C.c_int64),
                ("build_seconds", C.c_double), ("bbox_lo", C.c_float * 3), ("bbox_hi", C.c_float * 3),
                ("lanes_per_walk", C.c_int32), ("node_bytes", C.c_int32), ("cone_bytes", C.c_int32),
                ("wide_nodes_dirichlet", C.c_int64), ("wide_nodes_neumann", C.c_int64),
                ("wide_nodes_silhouette", C.c_int64), ("wide_depth_dirichlet", C.c_int32),
                ("wide_depth_neumann", C.c_int32), ("wide_depth_silhouette", C.c_int32), ("device", C.c_int32),
                ("stack_depth", C.c_int32)]


class wost_solve_desc(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("points", C.c_void_p), ("normals", C.c_void_p),
                ("on_neumann", C.c_void_p), ("memory", C.c_int32), ("walks_per_point", C.c_int32),
                ("epsilon", C.c_float), ("r_min", C.c_float), ("max_steps", C.c_int32), ("seed", C.c_uint64),
                ("first_walk", C.c_uint32), ("kernel", C.c_int32), ("block_size", C.c_int32),
                ("stream", C.c_void_p), ("sigma", C.c_float), ("screen_after", C.c_int32),
                ("stack_depth", C.c_int32), ("visit_limit", C.c_int32), ("lanes_per_walk", C.c_int32)]


class wost_progress(C.Structure):
    _fields_ = [("done", C.c_int32), ("walks_done", C.c_uint64), ("total_steps", C.c_uint64),
                ("capped_walks", C.c_uint64), ("guard_flags", C.c_uint32), ("elapsed_seconds", C.c_double),
                ("steps_run", C.c_uint64), ("launches", C.c_uint64)]


_SIGS = {
    "wost_scene_create": [C.POINTER(wost_scene_desc), C.POINTER(C.c_void_p)],
    "wost_scene_destroy": [C.c_void_p],
    "wost_scene_validate": [C.POINTER(wost_scene_desc), C.POINTER(wost_scene_info)],
    "wost_scene_get_info": [C.c_void_p, C.POINTER(wost_scene_info)],
    "wost_solve": [C.c_void_p, C.POINTER(wost_solve_desc), C.POINTER(C.c_void_p)],
    "wost_poll": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(wost_progress)],
    "wost_wait": [C.c_void_p, C.c_double],
    "wost_solve_advance": [C.c_void_p, C.c_int32, C.c_void_p],
    "wost_cancel": [C.c_void_p],
    "wost_solve_destroy": [C.c_void_p],
    "wost_solve_device_accumulators": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "wost_solve_work_counts": [C.c_void_p, C.c_void_p],
    "wost_solve_batch": [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "wost_engine_create": [C.c_void_p, C.POINTER(C.c_void_p)],
    "wost_engine_submit": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(C.c_void_p)],
    "wost_engine_get_stats": [C.c_void_p, C.c_void_p],
    "wost_engine_destroy": [C.c_void_p],
    "wost_scene_autotune": [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_float, C.c_int32,
                            C.c_void_p],
    "wost_screened_kernels": [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_float, C.c_void_p, C.c_void_p,
                              C.c_void_p],
    "wost_solve_static": [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_float, C.c_float, C.c_int32, C.c_uint64,
                          C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p],
    "wost_read_probe": [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p],
    "wost_query_closest_dirichlet": [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p],
    "wost_query_silhouette": [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "wost_query_intersect_neumann": [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "wost_query_neumann_sample": [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint32,
                                  C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
}


def load(path: str | None = None):
    """Loads libwost.so (raises OSError if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIBPATH
            if not os.path.exists(p):
                raise OSError(f"libwost.so not built ({p}); run __graft_entry__.build()")
            lib = C.CDLL(p)
            # the version first: a library of another version may lack
            # symbols this binding declares
            lib.wost_abi_version.restype = C.c_int32
            lib.wost_abi_version.argtypes = []
            if lib.wost_abi_version() != ABI_VERSION:
                raise OSError(f"{p}: ABI version {lib.wost_abi_version()}, this binding needs {ABI_VERSION}; "
                              "rebuild the library")
            for name, argt in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = argt
                fn.restype = C.c_int
            lib.wost_last_error.restype = C.c_char_p
            lib.wost_last_error.argtypes = []
            _lib = lib
    return _lib


def _check(status):
    if status != OK:
        raise WostError(status, _lib.wost_last_error().decode())


def wost_last_error() -> str:
    return load().wost_last_error().decode()


def wost_abi_version() -> int:
    return load().wost_abi_version()


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _field(spec, keep):
    f = wost_field()
    spec = spec or {"kind": "none"}
    f.kind = DATA[spec["kind"]]
    if spec["kind"] in ("per_vertex", "per_corner", "grid"):
        v = np.ascontiguousarray(spec["values"], np.float32).ravel()
        keep.append(v)
        f.values = _fptr(v)
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


def _dptr(t):
    """Device pointer of a torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ---------------------------------------------------------------------------
# C calls with the same names
# ---------------------------------------------------------------------------
def _scene_desc(spec: dict, device: int, leaf_size: int, keep: list):
    dim = int(spec["dim"])
    V = np.ascontiguousarray(spec["vertices"], np.float32)
    P = np.ascontiguousarray(spec["prims"], np.int32)
    Fl = np.ascontiguousarray(spec["flags"], np.uint8)
    keep += [V, P, Fl]
    d = wost_scene_desc()
    d.dim = dim
    d.n_vertices = V.size // dim
    d.vertices = _fptr(V)
    d.n_prims = P.size // dim
    d.prims = P.ctypes.data_as(C.POINTER(C.c_int32))
    d.flags = Fl.ctypes.data_as(C.POINTER(C.c_uint8))
    d.g = _field(spec.get("g"), keep)
    d.h = _field(spec.get("h"), keep)
    d.f = _field(spec.get("f"), keep)
    d.g_minus = _field(spec.get("g_minus"), keep)
    d.h_minus = _field(spec.get("h_minus"), keep)
    d.device = device
    d.leaf_size = leaf_size
    d.silhouette_split = int(spec.get("silhouette_split", 0))
    return d


def wost_scene_create(spec: dict, device: int = 0, leaf_size: int = 0):
    """Creates a scene from a scene dict (see scenes.py); returns the handle."""
    lib = load()
    keep = []
    d = _scene_desc(spec, device, leaf_size, keep)
    h = C.c_void_p()
    _check(lib.wost_scene_create(C.byref(d), C.byref(h)))
    return h


def wost_scene_validate(spec: dict, leaf_size: int = 0) -> dict:
    """Builds a scene's hierarchies on the host only and checks their
    structure; returns the scene info (raises WostError on a violation)."""
    lib = load()
    keep = []
    d = _scene_desc(spec, 0, leaf_size, keep)
    info = wost_scene_info()
    _check(lib.wost_scene_validate(C.byref(d), C.byref(info)))
    out = {k: getattr(info, k) for k, _ in wost_scene_info._fields_}
    out["bbox_lo"] = list(info.bbox_lo)
    out["bbox_hi"] = list(info.bbox_hi)
    return out


def wost_scene_destroy(h):
    _check(load().wost_scene_destroy(h))


def wost_scene_get_info(h) -> dict:
    info = wost_scene_info()
    _check(load().wost_scene_get_info(h, C.byref(info)))
    out = {k: getattr(info, k) for k, _ in wost_scene_info._fields_}
    out["bbox_lo"] = list(info.bbox_lo)
    out["bbox_hi"] = list(info.bbox_hi)
    return out


def wost_solve(scene, points, walks_per_point, epsilon, r_min=0.0, max_steps=1024, seed=0, first_walk=0,
               kernel="plain", block_size=0, normals=None, on_neumann=None, stream=None, sigma=0.0,
               screen_after=0, stack_depth=0, visit_limit=0, lanes_per_walk=0):
    """Starts a solve.  `points` is a numpy array (host) or a torch CUDA
    tensor (device); normals/on_neumann likewise.  sigma > 0 solves the
    screened equation from step screen_after on.  stack_depth / visit_limit
    (0 = defaults) bound the traversals (guards).  Returns the handle."""
    lib = load()
    keep = []
    d = _solve_desc(keep, points, walks_per_point, epsilon, r_min, max_steps, seed, first_walk, kernel, block_size,
                    normals, on_neumann, stream, sigma, screen_after, stack_depth, visit_limit, lanes_per_walk)
    h = C.c_void_p()
    _check(lib.wost_solve(scene, C.byref(d), C.byref(h)))
    return h


def wost_solve_batch(scenes, requests, stream=None):
    """One batched persistent launch (per dimension) for many solves.
    `requests` is a list of dicts with the keyword arguments of wost_solve.
    Returns one handle per request."""
    lib = load()
    n = len(requests)
    keep = []
    arr = (wost_solve_desc * n)()
    for i, rq in enumerate(requests):
        rq = dict(rq)
        pts = rq.pop("points")
        arr[i] = _solve_desc(keep, pts, **rq)
    sc = (C.c_void_p * n)(*[s.value if isinstance(s, C.c_void_p) else s for s in scenes])
    out = (C.c_void_p * n)()
    _check(lib.wost_solve_batch(n, sc, arr, _stream_ptr(stream), out))
    return [C.c_void_p(h) for h in out]


class wost_engine_desc(C.Structure):
    _fields_ = [("device", C.c_int32), ("memory_budget_bytes", C.c_int64), ("round_seconds", C.c_double),
                ("min_walks", C.c_int32), ("max_walks_per_point", C.c_int32), ("block_size", C.c_int32),
                ("max_wait_seconds", C.c_double)]


class wost_engine_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("cancelled", C.c_uint64), ("rejected", C.c_uint64), ("capped", C.c_uint64), ("queued", C.c_int32),
                ("active", C.c_int32), ("rounds", C.c_uint64), ("graph_launches", C.c_uint64),
                ("gpu_seconds", C.c_double),
                ("budget_bytes", C.c_int64), ("used_bytes", C.c_int64), ("round_budget_steps", C.c_double),
                ("walk_steps", C.c_uint64)]


def wost_engine_create(device=0, memory_budget_bytes=0, round_seconds=0.0, min_walks=0, max_walks_per_point=0,
                       block_size=0, max_wait_seconds=0.0):
    lib = load()
    d = wost_engine_desc(device, memory_budget_bytes, round_seconds, min_walks, max_walks_per_point, block_size,
                         max_wait_seconds)
    h = C.c_void_p()
    _check(lib.wost_engine_create(C.byref(d), C.byref(h)))
    return h


def wost_engine_submit(engine, scene, points, target_se, walks_cap=0, epsilon=1e-3, r_min=0.0, max_steps=1024,
                       seed=0, first_walk=0, normals=None, on_neumann=None):
    lib = load()
    keep = []
    d = _solve_desc(keep, points, walks_cap, epsilon, r_min, max_steps, seed, first_walk, "persistent", 0, normals,
                    on_neumann, None)
    h = C.c_void_p()
    _check(lib.wost_engine_submit(engine, scene, C.byref(d), float(target_se), C.byref(h)))
    return h


class wost_tune_result(C.Structure):
    _fields_ = [("block_size", C.c_int32), ("steps_per_second", C.c_double), ("n_tried", C.c_int32),
                ("tried_block", C.c_int32 * 8), ("tried_steps_per_second", C.c_double * 8),
                ("lanes_per_walk", C.c_int32), ("tried_lanes", C.c_int32 * 8)]


def wost_scene_autotune(scene, points, walks_per_point=32, epsilon=1e-3, r_min=0.0, max_steps=1024) -> dict:
    """Times block sizes on a sample of the (device) points; the fastest
    becomes the scene's default."""
    r = wost_tune_result()
    _check(load().wost_scene_autotune(scene, _dptr(points), points.shape[0], int(walks_per_point), float(epsilon),
                                      float(r_min), int(max_steps), C.byref(r)))
    return {"block_size": r.block_size, "lanes_per_walk": r.lanes_per_walk, "steps_per_second": r.steps_per_second,
            "tried": {(int(r.tried_lanes[i]), int(r.tried_block[i])): float(r.tried_steps_per_second[i])
                      for i in range(r.n_tried)}}


def wost_engine_get_stats(engine) -> dict:
    s = wost_engine_stats()
    _check(load().wost_engine_get_stats(engine, C.byref(s)))
    return {k: getattr(s, k) for k, _ in wost_engine_stats._fields_}


def wost_engine_destroy(engine):
    _check(load().wost_engine_destroy(engine))


def _solve_desc(keep, points, walks_per_point, epsilon, r_min=0.0, max_steps=1024, seed=0, first_walk=0,
                kernel="plain", block_size=0, normals=None, on_neumann=None, stream=None, sigma=0.0,
                screen_after=0, stack_depth=0, visit_limit=0, lanes_per_walk=0):
    d = wost_solve_desc()
    d.lanes_per_walk = int(lanes_per_walk)
    d.sigma = float(sigma)
    d.screen_after = int(screen_after)
    d.stack_depth = int(stack_depth)
    d.visit_limit = int(visit_limit)
    if isinstance(points, np.ndarray):
        pts = np.ascontiguousarray(points, np.float32)
        keep.append(pts)
        d.points = pts.ctypes.data_as(C.c_void_p)
        d.memory = MEM_HOST
        n = pts.shape[0]
        if normals is not None:
            nn = np.ascontiguousarray(normals, np.float32)
            on = np.ascontiguousarray(on_neumann, np.uint8)
            keep += [nn, on]
            d.normals = nn.ctypes.data_as(C.c_void_p)
            d.on_neumann = on.ctypes.data_as(C.c_void_p)
    else:
        d.points = _dptr(points)
        d.memory = MEM_DEVICE
        n = points.shape[0]
        if normals is not None:
            d.normals = _dptr(normals)
            d.on_neumann = _dptr(on_neumann)
    d.n_points = n
    d.walks_per_point = int(walks_per_point)
    d.epsilon = float(epsilon)
    d.r_min = float(r_min or 0.0)
    d.max_steps = int(max_steps)
    d.seed = int(seed)
    d.first_walk = int(first_walk)
    d.kernel = KERNEL[kernel] if isinstance(kernel, str) else int(kernel)
    d.block_size = int(block_size)
    d.stream = _stream_ptr(stream)
    return d


def wost_poll(solve, n_points):
    """Returns (mean, stderr, walks_done, progress dict)."""
    mean = np.zeros(n_points)
    se = np.zeros(n_points)
    wd = np.zeros(n_points, np.uint64)
    pr = wost_progress()
    _check(load().wost_poll(solve, mean.ctypes.data_as(C.c_void_p), se.ctypes.data_as(C.c_void_p),
                            wd.ctypes.data_as(C.c_void_p), C.byref(pr)))
    prog = {k: getattr(pr, k) for k, _ in wost_progress._fields_}
    return mean, se, wd, prog


def wost_solve_advance(solve, iterations=2048, stream=None):
    """One launch of a resumable solve: every lane runs up to `iterations`
    walk steps and saves its unfinished walk."""
    _check(load().wost_solve_advance(solve, int(iterations), _stream_ptr(stream)))


def wost_wait(solve, timeout_s=-1.0):
    _check(load().wost_wait(solve, float(timeout_s)))


def wost_wait_status(solve, timeout_s=0.0):
    """wost_wait's status code, without raising (OK, TIMEOUT while it runs,
    CANCELLED, BUDGET, ...): a cheap completion check for many requests."""
    return int(load().wost_wait(solve, float(timeout_s)))


def wost_cancel(solve):
    _check(load().wost_cancel(solve))


def wost_solve_destroy(solve):
    _check(load().wost_solve_destroy(solve))


def wost_solve_device_accumulators(solve):
    ptrs = [C.c_void_p() for _ in range(4)]
    _check(load().wost_solve_device_accumulators(solve, *[C.byref(p) for p in ptrs]))
    return [p.value for p in ptrs]


def wost_solve_work_counts(solve) -> dict:
    c = np.zeros(10, np.uint64)
    _check(load().wost_solve_work_counts(solve, c.ctypes.data_as(C.c_void_p)))
    out = {f"{q}_nodes": int(c[i]) for i, q in enumerate(COUNT_NAMES)}
    out.update({f"{q}_prims": int(c[5 + i]) for i, q in enumerate(COUNT_NAMES)})
    return out


def wost_query_closest_dirichlet(scene, pts, stream=None):
    import torch
    n = pts.shape[0]
    dim = pts.shape[1]
    dist = torch.empty(n, device=pts.device, dtype=torch.float32)
    cl = torch.empty(n, dim, device=pts.device, dtype=torch.float32)
    prim = torch.empty(n, device=pts.device, dtype=torch.int32)
    _check(load().wost_query_closest_dirichlet(scene, n, _dptr(pts), _dptr(dist), _dptr(cl), _dptr(prim),
                                               _stream_ptr(stream)))
    return dist, cl, prim


def wost_query_silhouette(scene, pts, rmax, stream=None):
    import torch
    n = pts.shape[0]
    dist = torch.empty(n, device=pts.device, dtype=torch.float32)
    _check(load().wost_query_silhouette(scene, n, _dptr(pts), _dptr(rmax), _dptr(dist), _stream_ptr(stream)))
    return dist


def wost_query_intersect_neumann(scene, origins, dirs, tmax, skip=None, stream=None):
    import torch
    n = origins.shape[0]
    hit = torch.empty(n, device=origins.device, dtype=torch.int32)
    t = torch.empty(n, device=origins.device, dtype=torch.float32)
    prim = torch.empty(n, device=origins.device, dtype=torch.int32)
    _check(load().wost_query_intersect_neumann(scene, n, _dptr(origins), _dptr(dirs), _dptr(tmax), _dptr(skip),
                                               _dptr(hit), _dptr(t), _dptr(prim), _stream_ptr(stream)))
    return hit, t, prim


def wost_query_neumann_sample(scene, pts, r, seed=0, ctr1=0, ctr2=0, stream=None):
    import torch
    n, dim = pts.shape
    z = torch.empty(n, dim, device=pts.device, dtype=torch.float32)
    pdf = torch.empty(n, device=pts.device, dtype=torch.float32)
    prim = torch.empty(n, device=pts.device, dtype=torch.int32)
    _check(load().wost_query_neumann_sample(scene, n, _dptr(pts), _dptr(r), int(seed), int(ctr1), int(ctr2),
                                            _dptr(z), _dptr(pdf), _dptr(prim), _stream_ptr(stream)))
    return z, pdf, prim


# ---------------------------------------------------------------------------
# small object wrappers
# ---------------------------------------------------------------------------
class Scene:
    def __init__(self, spec: dict, device: int = 0, leaf_size: int = 0):
        self.dim = int(spec["dim"])
        self.handle = wost_scene_create(spec, device, leaf_size)

    def info(self):
        return wost_scene_get_info(self.handle)

    def close(self):
        if self.handle:
            wost_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(scene: Scene, points, walks, epsilon, r_min=0.0, max_steps=1024, seed=0, first_walk=0, kernel="plain",
          block_size=0, normals=None, on_neumann=None, stream=None, timeout=-1.0, sigma=0.0, screen_after=0,
          stack_depth=0, visit_limit=0, lanes_per_walk=0):
    """Runs a solve to completion; returns a dict of per-point statistics."""
    h = wost_solve(scene.handle, points, walks, epsilon, r_min, max_steps, seed, first_walk, kernel, block_size,
                   normals, on_neumann, stream, sigma, screen_after, stack_depth, visit_limit, lanes_per_walk)
    try:
        wost_wait(h, timeout)
        mean, se, wd, prog = wost_poll(h, points.shape[0])
        if kernel == "counting":
            prog["counts"] = wost_solve_work_counts(h)
    finally:
        wost_solve_destroy(h)
    return dict(mean=mean, se=se, walks=wd, **prog)


# ---------------------------------------------------------------------------
# solve without allocation
# ---------------------------------------------------------------------------
WOST_STATIC_MAX_POINTS = 65536


def wost_solve_static(scene, points, walks_per_point, epsilon, r_min, max_steps, seed, first_walk, mean_out,
                      stderr_out=None, stream=None):
    """wost_solve_static: the walks of wost_solve (persistent kernel) with no
    allocation anywhere, for callers that cannot allocate device memory while
    they solve.  points (n x dim), mean_out and stderr_out (n) are CUDA
    float32 tensors owned by the caller; the call returns once the work is
    enqueued on `stream`."""
    info = wost_scene_get_info(scene)
    for name, t in (("points", points), ("mean_out", mean_out), ("stderr_out", stderr_out)):
        if t is not None and not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 4
                                  and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        if t is not None and t.device.index != info["device"]:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the scene on cuda:{info['device']}")
    # the C entry point takes raw pointers and cannot check sizes itself
    if points.dim() != 2 or points.shape[1] != info["dim"]:
        raise ValueError(f"points must be (n, {info['dim']}) for this scene, got {tuple(points.shape)}")
    n = int(points.shape[0])
    for name, t in (("mean_out", mean_out), ("stderr_out", stderr_out)):
        if t is not None and t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} values, fewer than the {n} points")
    _check(load().wost_solve_static(scene, int(points.shape[0]), points.data_ptr(), int(walks_per_point),
                                    float(epsilon), float(r_min), int(max_steps), int(seed), int(first_walk),
                                    mean_out.data_ptr(), None if stderr_out is None else stderr_out.data_ptr(),
                                    _stream_ptr(stream)))


def wost_read_probe(buf, passes, sink, stream=None):
    """One read sweep kernel over a contiguous CUDA tensor `buf` (passes
    sweeps of 16-byte loads that bypass L1); the caller times it."""
    _check(load().wost_read_probe(_dptr(buf), int(buf.numel() * buf.element_size()), int(passes), _dptr(sink),
                                  _stream_ptr(stream)))


def wost_screened_kernels(dim, rho, R, sigma, stream=None):
    """G^sigma_B and Q^sigma_B (App. A.2) at CUDA float32 tensors rho, R;
    returns (G, Q) as new CUDA tensors."""
    import torch

    G = torch.empty_like(rho)
    Q = torch.empty_like(rho)
    _check(load().wost_screened_kernels(int(dim), int(rho.numel()), _dptr(rho), _dptr(R), float(sigma), _dptr(G),
                                        _dptr(Q), _stream_ptr(stream)))
    return G, Q
