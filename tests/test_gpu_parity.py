"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
and against exact solutions.

Tolerances (FP32 walks and queries against FP64):
  * query distances: |d_gpu - d_oracle| <= 1e-5 d + 4e-7 (relative 1e-5 with
    an absolute floor of a few single-precision ulps at unit scale); the same
    primitive except at ties;
  * silhouette predicates and ray hits decided within float rounding of their
    threshold may differ: at most 0.2% of the queries, and every such answer
    lies between the oracle's answers with the threshold moved by the size
    of single-precision rounding either way (Q.3: also by the 1e-4 edge
    margin of the GPU's hit test);
  * walks: both sides draw the same Philox4x32-10 numbers, so per-point
    estimates are strongly correlated; against the exact solution the
    multiple-comparisons z test of statcheck.py; RMS error of the GPU at most
    1.1x the oracle's at equal walk counts.
"""
import numpy as np
import pytest

import oracle
from paper_2302_11815_gb300 import scenes
from statcheck import check_z, kurtosis

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ABS = 4e-7
REL = 1e-5
# silhouette threshold bracket: tau |v| (1 + |x|_inf), a few times the
# rounding of the single-precision product (v.n0)(v.n1) (3D closest points on
# edges carry errors of order 1e-7 (1 + |x|))
SIL_TAU = 4e-6
# Q.3 on the GPU accepts hits within 1e-4 of a segment end / triangle edge
RAY_TOL_WIDE = 1.1e-4
RAY_TOL_NARROW = 1e-6


@pytest.fixture(scope="module")
def wost():
    from paper_2302_11815_gb300 import build as libbuild
    from paper_2302_11815_gb300 import wost as w

    assert torch.cuda.is_available()
    libbuild.build()
    w.load()
    return w


def _scenes():
    return {
        "flower": scenes.config1(),
        "koch3": scenes.config2(grid=48, level=3),
        "box_sphere": scenes.box_sphere_scene(m=6, n_lat=16, n_lon=32),
        "cube_torus": scenes.config3(grid=24, nu=120, nv=48, cube_m=8),
    }


SCENES = _scenes()


def _rand_points(sc, n, seed):
    rng = np.random.default_rng(seed)
    V = sc["vertices"]
    lo, hi = V.min(0), V.max(0)
    pad = 0.1 * (hi - lo)
    return (lo - pad + (hi - lo + 2 * pad) * rng.random((n, sc["dim"]))).astype(np.float32)


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


# ---------------------------------------------------------------------------
# queries
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(SCENES))
def test_q1_closest_point_matches_brute_force(wost, name):
    sc = SCENES[name]
    S = wost.Scene(sc)
    O = oracle.Scene(sc)
    pts = _rand_points(sc, 20000, 1)
    d, cl, pr = wost.wost_query_closest_dirichlet(S.handle, _dev(pts))
    d, cl, pr = d.cpu().numpy(), cl.cpu().numpy(), pr.cpu().numpy()
    od, ocl, opr = oracle.closest_dirichlet(O, pts.astype(np.float64))
    assert np.all(np.abs(d - od) <= REL * od + ABS), np.max(np.abs(d - od) / (od + 1e-9))
    same = pr == opr
    # the closest point is unique where the primitive is
    assert np.all(np.abs(cl - ocl)[same] <= 1e-5 + 1e-5 * np.abs(ocl)[same])
    diff = ~same
    if diff.any():
        # ties: the oracle's distance to the GPU's primitive equals the minimum
        sub = {"dim": sc["dim"], "vertices": sc["vertices"], "prims": sc["prims"][pr[diff]],
               "flags": np.zeros(diff.sum(), np.uint8), "g": {"kind": "none"}, "h": {"kind": "none"}}
        for i, k in enumerate(np.nonzero(diff)[0]):
            one = dict(sub, prims=sc["prims"][pr[k]][None], flags=np.zeros(1, np.uint8))
            dk, _, _ = oracle.closest_dirichlet(oracle.Scene(one), pts[k:k + 1].astype(np.float64))
            assert abs(dk[0] - od[k]) <= 1e-5 * od[k] + ABS
            if i > 50:
                break
    S.close()


@pytest.mark.parametrize("name", list(SCENES))
def test_q2_silhouette_distance_matches_brute_force(wost, name):
    sc = SCENES[name]
    S = wost.Scene(sc)
    O = oracle.Scene(sc)
    pts = _rand_points(sc, 20000, 2)
    od, _, _ = oracle.closest_dirichlet(O, pts.astype(np.float64))
    rmax = np.minimum(od, 10.0).astype(np.float32)
    d = wost.wost_query_silhouette(S.handle, _dev(pts), _dev(rmax)).cpu().numpy()
    ods, _ = oracle.silhouette_distance(O, pts.astype(np.float64), rmax.astype(np.float64))
    bad = np.abs(d - ods) > REL * ods + ABS
    assert bad.mean() <= 2e-3, (bad.sum(), len(bad))
    assert (ods < rmax).mean() > 0.05  # the test does see silhouettes
    if bad.any():
        # each disagreement is a predicate decided within rounding: the GPU's
        # distance lies between the oracle's with the silhouette threshold
        # relaxed (more silhouettes, nearer) and tightened (fewer, farther)
        x, rm = pts[bad].astype(np.float64), rmax[bad].astype(np.float64)
        lo = oracle.silhouette_distance_tol(O, x, rm, SIL_TAU)
        hi = oracle.silhouette_distance_tol(O, x, rm, -SIL_TAU)
        ok = (d[bad] >= lo * (1 - REL) - ABS) & (d[bad] <= hi * (1 + REL) + ABS)
        assert ok.all(), list(zip(d[bad][~ok], lo[~ok], hi[~ok]))
    S.close()


@pytest.mark.parametrize("name", list(SCENES))
def test_q3_ray_hits_match_brute_force(wost, name):
    sc = SCENES[name]
    S = wost.Scene(sc)
    O = oracle.Scene(sc)
    rng = np.random.default_rng(3)
    o = _rand_points(sc, 20000, 3)
    v = rng.normal(size=o.shape).astype(np.float32)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    tmax = np.full(len(o), 0.6, np.float32)
    hit, t, pr = (a.cpu().numpy() for a in wost.wost_query_intersect_neumann(S.handle, _dev(o), _dev(v), _dev(tmax)))
    oh, ot, opr = oracle.intersect_neumann(O, o.astype(np.float64), v.astype(np.float64), tmax.astype(np.float64))
    agree = (hit.astype(bool) == oh)
    assert agree.mean() >= 1 - 2e-3
    both = agree & oh
    assert both.sum() > 100
    close = np.abs(t - ot) <= REL * ot + ABS
    assert np.mean(close[both]) >= 1 - 2e-3
    assert np.mean(pr[both] == opr[both]) >= 1 - 2e-3
    _check_ray_brackets(O, o, v, tmax, hit, t, ~(agree & close))
    # skipping the primitive that was hit
    sk = np.where(oh, opr, -1).astype(np.int32)
    h2, t2, _ = (a.cpu().numpy() for a in wost.wost_query_intersect_neumann(
        S.handle, _dev(o), _dev(v), _dev(tmax), skip=torch.from_numpy(sk).cuda()))
    oh2, ot2, _ = oracle.intersect_neumann(O, o.astype(np.float64), v.astype(np.float64), tmax.astype(np.float64), skip=sk)
    agree2 = h2.astype(bool) == oh2
    assert agree2.mean() >= 1 - 2e-3
    _check_ray_brackets(O, o, v, tmax, h2, t2, ~(agree2 & (np.abs(t2 - ot2) <= REL * ot2 + ABS)), skip=sk)
    S.close()


def _check_ray_brackets(O, o, v, tmax, hit, t, which, skip=None):
    """Every ray answer that differs from the oracle's lies between the
    oracle's answers with the hit test widened by the GPU's edge margin
    (plus rounding) and tightened by rounding, and tmax moved by rounding."""
    if not which.any():
        return
    x, d, tm = o[which].astype(np.float64), v[which].astype(np.float64), tmax[which].astype(np.float64)
    sk = None if skip is None else skip[which]
    hl, tl = oracle.intersect_neumann_tol(O, x, d, tm * (1 + REL), RAY_TOL_WIDE, skip=sk)
    hh, th = oracle.intersect_neumann_tol(O, x, d, tm * (1 - REL), -RAY_TOL_NARROW, skip=sk)
    tg = np.where(hit[which].astype(bool), t[which], tm)
    ok = (tg >= np.where(hl, tl, tm) * (1 - REL) - ABS) & (tg <= np.where(hh, th, tm) * (1 + REL) + ABS)
    assert ok.all(), list(zip(tg[~ok], tl[~ok], th[~ok]))


def test_q4_sampler_is_unbiased_on_gpu(wost):
    # E[1{|z-x|<r}/pdf] = length (2D) or area (3D) of the Neumann boundary in
    # the ball (Algs. 5-6 give an unbiased estimate for any tree)
    k = 200
    xs = np.linspace(-2, 2, k + 1)
    V = np.c_[xs, np.zeros(k + 1)]
    P = np.c_[np.arange(k), np.arange(1, k + 1)]
    # one far Dirichlet segment (a scene needs one)
    V = np.r_[V, [[-2, 5], [2, 5]]]
    P = np.r_[P, [[k + 1, k + 2]]]
    sc = {"dim": 2, "vertices": V.astype(np.float32), "prims": P.astype(np.int32),
          "flags": np.r_[np.ones(k), 0].astype(np.uint8), "g": {"kind": "none"}, "h": {"kind": "none"},
          "f": {"kind": "none"}}
    S = wost.Scene(sc)
    n = 200000
    x = np.tile(np.array([[0.1, 0.3]], np.float32), (n, 1))
    r = np.full(n, 0.5, np.float32)
    z, pdf, pr = (a.cpu().numpy() for a in wost.wost_query_neumann_sample(S.handle, _dev(x), _dev(r), seed=5))
    ok = (pr >= 0) & (pdf > 0) & (np.linalg.norm(z - x, axis=1) < 0.5)
    vals = np.where(ok, 1.0 / np.where(pdf > 0, pdf, 1), 0.0)
    want = 2 * np.sqrt(0.25 - 0.09)
    assert abs(vals.mean() - want) < 4 * vals.std() / np.sqrt(n)
    S.close()


# ---------------------------------------------------------------------------
# walks
# ---------------------------------------------------------------------------
def _gpu_solve(wost, sc, pts, walks, seed, kernel="plain", eps=None, max_steps=None, device_points=True):
    S = wost.Scene(sc)
    p = _dev(pts) if device_points else np.ascontiguousarray(pts, np.float32)
    res = wost.solve(S, p, walks, eps or sc["epsilon"], sc.get("r_min", 0.0), max_steps or sc["max_steps"],
                     seed=seed, kernel=kernel)
    S.close()
    return res


def _allow(sc, eps):
    fn, pr = sc["exact"]
    L = np.max(np.linalg.norm(scenes.exact_grad(fn, pr, sc["vertices"].astype(float)), axis=1))
    return eps * 1.05 * L


@pytest.mark.parametrize("kernel", ["plain", "persistent"])
def test_walk_config1_vs_exact_and_oracle(wost, kernel):
    sc = scenes.config1()
    pts = sc["points"]
    res = _gpu_solve(wost, sc, pts, 512, 11, kernel)
    assert res["done"] == 1 and int(res["walks"].sum()) == len(pts) * 512
    assert res["capped_walks"] == 0 and res["guard_flags"] == 0
    u = scenes.exact_u("exp_cos", (), pts)
    ref = oracle.solve(oracle.Scene(sc), pts, 512, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=11,
                       per_walk=True)
    check_z(res["mean"] - u, res["se"], _allow(sc, sc["epsilon"]), label="gpu", walks=512,
            kurt=kurtosis(ref["per_walk"]))
    rms_g = np.sqrt(np.mean((res["mean"] - u) ** 2))
    rms_o = np.sqrt(np.mean((ref["mean"] - u) ** 2))
    assert rms_g <= 1.1 * rms_o, (rms_g, rms_o)
    # same random streams: the GPU and oracle estimates track each other
    assert np.median(np.abs(res["mean"] - ref["mean"])) < 0.2 * np.median(ref["se"])


def test_walk_identical_streams_without_neumann_data(wost):
    """With h = 0 the Neumann sampler cannot change an estimate, so the GPU
    and the oracle follow the same walks: per-point means agree to float
    rounding except where a float-vs-double decision splits a walk."""
    sc = scenes.square_scene(8, fn="linear", params=(0.0, 0.0, 1.0, 0.0), neumann_sides=("left", "right"))
    rng = np.random.default_rng(31)
    pts = (0.05 + 0.9 * rng.random((128, 2))).astype(np.float32)
    res = _gpu_solve(wost, sc, pts, 256, 5, eps=1e-3, max_steps=4096)
    ref = oracle.solve(oracle.Scene(sc), pts, 256, 1e-3, None, 4096, seed=5)
    d = np.abs(res["mean"] - ref["mean"])
    assert np.median(d) < 1e-5, np.median(d)
    assert np.mean(d < 1e-4) > 0.8
    assert np.all(d < 4 * ref["se"] + 1e-4)


def test_walk_koch_poisson_small_vs_exact_and_oracle(wost):
    sc = scenes.config2(grid=16, level=3)
    pts = sc["points"]
    res = _gpu_solve(wost, sc, pts, 256, 21, "persistent")
    u = scenes.exact_u("sin2x_cos3y", (), pts)
    assert res["capped_walks"] <= 1e-3 * len(pts) * 256
    ref = oracle.solve(oracle.Scene(sc), pts, 256, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=21,
                       per_walk=True)
    check_z(res["mean"] - u, res["se"], _allow(sc, sc["epsilon"]), label="gpu koch", walks=256,
            kurt=kurtosis(ref["per_walk"]))
    rms_g = np.sqrt(np.mean((res["mean"] - u) ** 2))
    rms_o = np.sqrt(np.mean((ref["mean"] - u) ** 2))
    assert rms_g <= 1.1 * rms_o, (rms_g, rms_o)


def test_walk_3d_box_sphere_vs_exact_and_oracle(wost):
    sc = scenes.box_sphere_scene()
    rng = np.random.default_rng(25)
    p = rng.uniform(-0.9, 0.9, (400, 3))
    pts = p[np.linalg.norm(p, axis=1) > 0.5][:96].astype(np.float32)
    res = _gpu_solve(wost, sc, pts, 512, 7, "persistent", eps=1e-3, max_steps=4096)
    u = scenes.exact_u("quad3", (), pts)
    ref = oracle.solve(oracle.Scene(sc), pts, 512, 1e-3, None, 4096, seed=7, per_walk=True)
    check_z(res["mean"] - u, res["se"], _allow(sc, 1e-3), label="gpu 3d", walks=512, kurt=kurtosis(ref["per_walk"]))
    rms_g = np.sqrt(np.mean((res["mean"] - u) ** 2))
    rms_o = np.sqrt(np.mean((ref["mean"] - u) ** 2))
    assert rms_g <= 1.1 * rms_o, (rms_g, rms_o)


def test_walk_source_term_bump_2d(wost):
    sc = scenes.disk_scene(256, "bump", source=True)
    rng = np.random.default_rng(4)
    pts = scenes.ball_points(rng, 128, 2, 0.9)
    res = _gpu_solve(wost, sc, pts, 1024, 3, eps=1e-3, max_steps=1024)
    ref = oracle.solve(oracle.Scene(sc), pts, 1024, 1e-3, None, 1024, seed=3, per_walk=True)
    check_z(res["mean"] - scenes.exact_u("bump", (), pts), res["se"], _allow(sc, 1e-3), label="bump", walks=1024,
            kurt=kurtosis(ref["per_walk"]))


@pytest.mark.parametrize("where", ["square_2d", "cube_3d", "flower_2d"])
def test_walk_per_vertex_data_vs_exact_and_oracle(wost, where):
    """Per-vertex g and h (the layout the workloads specify), converted to
    primitive corners by the library: exact for a linear u on the square and
    on a cube with one Neumann face (against the exact solution), and on the
    curved mixed flower against the oracle on the same random streams (the
    oracle interpolates the vertex values itself)."""
    rng = np.random.default_rng(41)
    if where == "square_2d":
        sc = scenes.square_scene(8, fn="linear", params=(0.3, 0.7, -1.2, 0.0), neumann_sides=("bottom", "top"),
                                 data="per_vertex")
        pts = (0.05 + 0.9 * rng.random((256, 2))).astype(np.float32)
    elif where == "cube_3d":
        sc = scenes.cube_scene(4, fn="linear", params=(0.2, 0.5, -0.3, 0.8), neumann_faces=(5,), data="per_vertex")
        pts = rng.uniform(-0.85, 0.85, (128, 3)).astype(np.float32)
    else:
        sc = scenes.config1(data="per_vertex")
        pts = sc["points"]
    res = _gpu_solve(wost, sc, pts, 512, 13, "persistent", eps=1e-3, max_steps=4096)
    assert res["guard_flags"] == 0 and res["capped_walks"] == 0
    ref = oracle.solve(oracle.Scene(sc), pts, 512, 1e-3, None, 4096, seed=13, per_walk=True)
    # same streams: the estimates track the oracle's (loosely: the two Neumann
    # samplers descend different trees, so those terms differ walk by walk)
    assert np.median(np.abs(res["mean"] - ref["mean"])) < 0.5 * np.median(ref["se"])
    if where != "flower_2d":
        u = scenes.exact_u(*sc["exact"], pts)
        check_z(res["mean"] - u, res["se"], _allow(sc, 1e-3), label=f"per-vertex {where}", walks=512,
                kurt=kurtosis(ref["per_walk"]))
        rms_g = np.sqrt(np.mean((res["mean"] - u) ** 2))
        rms_o = np.sqrt(np.mean((ref["mean"] - u) ** 2))
        assert rms_g <= 1.1 * rms_o, (rms_g, rms_o)


@pytest.mark.parametrize("where", ["flower_mid", "flower_near_vertex", "sphere_3d"])
def test_walk_from_points_on_the_neumann_boundary(wost, where):
    """Evaluation points on the Neumann boundary with their normals (Alg. 1's
    Require: x0 may lie on the Neumann part): the first step samples the
    hemisphere about -n_x, starts its queries off the boundary (R4) and
    weights the Neumann term with alpha = 1/2 (R8).  Against the exact
    solution and against the oracle on the same random streams."""
    if where == "sphere_3d":
        sc = scenes.box_sphere_scene(data="analytic")
        V, P = sc["vertices"].astype(np.float64), sc["prims"]
        sel = np.nonzero(sc["flags"] == 1)[0][::37]
        pts = (V[P[sel, 0]] + V[P[sel, 1]] + V[P[sel, 2]]) / 3.0
        walks, fn = 2000, "quad3"
    else:
        sc = scenes.config1()
        V, P = sc["vertices"].astype(np.float64), sc["prims"]
        sel = np.nonzero(sc["flags"] == 1)[0][::4]
        s = 0.5 if where == "flower_mid" else 0.9
        pts = V[P[sel, 0]] * (1 - s) + V[P[sel, 1]] * s
        walks, fn = 3000, "exp_cos"
    nrm = scenes.prim_normals(sc)[sel]
    on = np.ones(len(sel), np.uint8)
    S = wost.Scene(sc)
    res = wost.solve(S, _dev(pts), walks, 1e-3, 0.0, 1024, seed=41, kernel="persistent",
                     normals=_dev(nrm), on_neumann=torch.from_numpy(on).cuda())
    S.close()
    assert res["guard_flags"] == 0 and res["capped_walks"] == 0
    ref = oracle.solve(oracle.Scene(sc), pts, walks, 1e-3, max_steps=1024, seed=41, normals=nrm, on_neumann=on,
                       per_walk=True)
    u = scenes.exact_u(fn, (), pts)
    check_z(res["mean"] - u, res["se"], 3e-3, label=f"gpu boundary starts {where}", walks=walks,
            kurt=kurtosis(ref["per_walk"]))
    rms_g = np.sqrt(np.mean((res["mean"] - u) ** 2))
    rms_o = np.sqrt(np.mean((ref["mean"] - u) ** 2))
    assert rms_g <= 1.1 * rms_o + 1e-3, (rms_g, rms_o)


def _app_b_case(name):
    rng = np.random.default_rng(60)
    if name in ("slit", "crack"):
        sc = scenes.slit_square_scene() if name == "slit" else scenes.crack_square_scene()
        p = rng.uniform(-0.95, 0.95, (1000, 2))
        pts = p[(np.abs(p[:, 1]) > 0.05) | (p[:, 0] < -0.05)][:192]
        return sc, pts, 1e-4, (1.05e-4 / 0.05 if name == "slit" else 1.05e-4 * 3.0), 4096
    if name == "plate_3d":
        sc = scenes.plate_cube_scene()
        p = rng.uniform(-0.85, 0.85, (1000, 3))
        pts = p[(np.abs(p[:, 2] - 0.1) > 0.04) | (np.abs(p[:, 0]) > 0.55) | (np.abs(p[:, 1]) > 0.55)][:128]
        return sc, pts, 1e-3, 1.05e-3 * 1.7, 16384
    sc = scenes.sheet_square_scene(data=name.split(":")[1])
    p = rng.uniform(-0.9, 0.9, (1000, 2))
    pts = p[(np.abs(p[:, 1] - 0.1) > 0.03) | (np.abs(p[:, 0]) > 0.55)][:192]
    return sc, pts, 1e-3, 1.05e-3 * 1.6, 4096


@pytest.mark.parametrize("name", ["slit", "crack", "sheet:analytic", "sheet:per_corner", "sheet:per_corner_minus",
                                  "plate_3d"])
def test_walk_double_sided_boundaries_vs_exact_and_oracle(wost, name):
    """App. B: double-sided Dirichlet data on a slit (u = polar angle, 0 above
    and 2 pi below), a zero-flux Neumann crack across which u jumps, and
    Neumann sheets / a 3D plate inside Dirichlet boxes with the flux of each
    side given analytically, per corner, or per corner for both sides.
    Against the exact solution and the oracle on the same random streams."""
    sc, pts, eps, allow, cap = _app_b_case(name)
    pts = pts.astype(np.float32)
    res = _gpu_solve(wost, sc, pts, 1024, 61, "persistent", eps=eps, max_steps=cap)
    assert res["guard_flags"] == 0 and res["capped_walks"] == 0
    ref = oracle.solve(oracle.Scene(sc), pts, 1024, eps, None, cap, seed=61, per_walk=True)
    u = scenes.exact_u(*sc["exact"], pts)
    check_z(res["mean"] - u, res["se"], allow, label=f"gpu {name}", walks=1024, kurt=kurtosis(ref["per_walk"]))
    assert np.median(np.abs(res["mean"] - ref["mean"])) < 0.5 * np.median(ref["se"])
    rms_g = np.sqrt(np.mean((res["mean"] - u) ** 2))
    rms_o = np.sqrt(np.mean((ref["mean"] - u) ** 2))
    assert rms_g <= 1.1 * rms_o + 1e-3, (rms_g, rms_o)


def test_walk_keyhole_neumann_dominated(wost):
    """The Neumann-dominated stress scene (two rooms, a narrow corridor, a
    small Dirichlet window; walks of hundreds of steps, the keyhole regime
    the paper describes among its limitations): the resumable kernel against
    the exact solution u = x, with the kurtosis of the walk estimates from
    the oracle at the same points."""
    sc = scenes.keyhole_scene(n_points=32)
    pts = sc["points"]
    S = wost.Scene(sc)
    res = wost.solve(S, _dev(pts), 8192, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=91, kernel="resumable")
    S.close()
    assert res["guard_flags"] == 0 and res["capped_walks"] == 0
    steps_per_walk = res["total_steps"] / (len(pts) * 8192)
    assert steps_per_walk > 200  # the regime of the scene
    ref = oracle.solve(oracle.Scene(sc), pts, 256, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=91,
                       per_walk=True)
    u = pts[:, 0].astype(np.float64)
    check_z(res["mean"] - u, res["se"], 1.05e-3, label="keyhole", walks=8192, kurt=kurtosis(ref["per_walk"]))


def test_plain_and_persistent_give_the_same_walks(wost):
    sc = scenes.config1(n_points=64)
    a = _gpu_solve(wost, sc, sc["points"], 256, 9, "plain")
    b = _gpu_solve(wost, sc, sc["points"], 256, 9, "persistent")
    # identical walks; only the order of the FP64 additions differs
    np.testing.assert_allclose(a["mean"], b["mean"], rtol=1e-9, atol=1e-12)
    assert a["total_steps"] == b["total_steps"]


@pytest.mark.parametrize("iters", [1, 7, 2048])
def test_resumable_gives_the_same_walks(wost, iters):
    # walks carried across many short launches (1 and 7 steps per launch)
    # end exactly as in one persistent launch
    sc = scenes.config2(grid=24)
    pts = sc["points"][:40]
    a = _gpu_solve(wost, sc, pts, 64, 9, "persistent", eps=sc["epsilon"], max_steps=512)
    S = wost.Scene(sc)
    h = wost.wost_solve(S.handle, _dev(pts), 64, sc["epsilon"], sc["r_min"], 512, seed=9, kernel="resumable")
    n_adv = 0
    while True:
        wost.wost_solve_advance(h, iters)
        n_adv += 1
        _, _, _, pr = wost.wost_poll(h, len(pts))
        if pr["walks_done"] == len(pts) * 64 or n_adv > 100000:
            break
    wost.wost_wait(h)  # completion check: no walk left in a slot
    mean, se, wd, pr = wost.wost_poll(h, len(pts))
    wost.wost_solve_destroy(h)
    S.close()
    assert pr["done"] == 1 and pr["launches"] >= n_adv
    assert int(wd.sum()) == len(pts) * 64
    np.testing.assert_allclose(mean, a["mean"], rtol=1e-9, atol=1e-12)
    assert pr["total_steps"] == a["total_steps"] and pr["capped_walks"] == a["capped_walks"]
    assert pr["steps_run"] == pr["total_steps"]


def test_resumable_wait_drives_the_launches(wost):
    sc = scenes.config1(n_points=64)
    a = _gpu_solve(wost, sc, sc["points"], 128, 4, "persistent")
    b = _gpu_solve(wost, sc, sc["points"], 128, 4, "resumable")
    np.testing.assert_allclose(a["mean"], b["mean"], rtol=1e-9, atol=1e-12)
    assert a["total_steps"] == b["total_steps"] and b["launches"] >= 1


@pytest.mark.parametrize("kernel", ["plain", "persistent", "resumable"])
def test_walk_outside_the_grown_bounding_box_ends_at_once(wost, kernel):
    # R13 on the GPU, against the oracle: one step, capped, g at the closest
    # Dirichlet point; a non-finite start ends with no boundary term
    sc = scenes.square_scene(m=4, fn="linear", params=(0.5, 1.0, 2.0, 0.0), neumann_sides=("bottom", "top"))
    pts = np.array([[2.5, 0.25], [-1.25, 0.75], [np.nan, 0.5]], np.float32)
    res = _gpu_solve(wost, sc, pts, 32, 3, kernel, eps=1e-3, max_steps=1024)
    assert res["total_steps"] == 3 * 32 and res["capped_walks"] == 3 * 32
    o = oracle.solve(oracle.Scene(sc), pts.astype(np.float64), 4, 1e-3, max_steps=1024, seed=3)
    np.testing.assert_allclose(res["mean"], o["mean"], rtol=1e-6, atol=1e-6)


def test_host_and_device_inputs_agree(wost):
    sc = scenes.config1(n_points=32)
    a = _gpu_solve(wost, sc, sc["points"], 64, 2, device_points=True)
    b = _gpu_solve(wost, sc, sc["points"], 64, 2, device_points=False)
    np.testing.assert_allclose(a["mean"], b["mean"], rtol=1e-9, atol=1e-12)


def test_edge_cases(wost):
    sc = scenes.config1(n_points=8)
    # one point, one walk
    r = _gpu_solve(wost, sc, sc["points"][:1], 1, 1)
    assert r["walks"][0] == 1 and np.isfinite(r["mean"][0])
    # step cap 1: every walk stops at once with g at the closest point
    S = wost.Scene(sc)
    r = wost.solve(S, _dev(sc["points"]), 16, 1e-3, 0.0, 1, seed=1)
    assert r["capped_walks"] == 8 * 16
    d, cl, _ = wost.wost_query_closest_dirichlet(S.handle, _dev(sc["points"]))
    g = scenes.exact_u("exp_cos", (), cl.cpu().numpy())
    np.testing.assert_allclose(r["mean"], g, rtol=1e-5, atol=1e-5)
    # a point on the Dirichlet boundary ends immediately with g there
    V = sc["vertices"]
    on = ((V[0] + V[1]) / 2)[None].astype(np.float32)
    r = wost.solve(S, _dev(on), 8, 1e-3, 0.0, 1024, seed=1)
    assert r["total_steps"] == 8
    np.testing.assert_allclose(r["mean"], scenes.exact_u("exp_cos", (), on), rtol=1e-5, atol=1e-5)
    # pure Dirichlet scene (empty Neumann set) = walk on spheres
    D = scenes.disk_scene(64, "exp_cos")
    rng = np.random.default_rng(0)
    pts = scenes.ball_points(rng, 32, 2, 0.8)
    r = _gpu_solve(wost, D, pts, 512, 4, eps=1e-3, max_steps=1024)
    o = oracle.solve(oracle.Scene(D), pts, 512, 1e-3, None, 1024, seed=4, per_walk=True)
    check_z(r["mean"] - scenes.exact_u("exp_cos", (), pts), r["se"], _allow(D, 1e-3), label="wos", walks=512,
            kurt=kurtosis(o["per_walk"]))
    # invalid solve arguments
    for kw in (dict(walks=0), dict(eps=0.0), dict(rmin=1e-2), dict(steps=0)):
        with pytest.raises(wost.WostError) as ei:
            wost.wost_solve(S.handle, _dev(sc["points"]), kw.get("walks", 4), kw.get("eps", 1e-3),
                            kw.get("rmin", 0.0), kw.get("steps", 16))
        assert ei.value.status == wost.ERR_INVALID_ARG
    S.close()


@pytest.mark.parametrize("kernel", ["plain", "persistent", "resumable"])
@pytest.mark.parametrize("knob, bit", [("stack_depth", 1), ("visit_limit", 2)])
def test_device_guards_fire_and_are_reported(wost, kernel, knob, bit):
    """A traversal stack of 2 entries (the scene's trees are 13-15 deep) or
    a limit of 3 node visits per traversal: the bounded device guards stop
    the traversal, record their bit, and wost_wait / wost_poll return
    INTERNAL promptly (a limit running out, no fault)."""
    import time
    sc = SCENES["koch3"]
    S = wost.Scene(sc)
    assert S.info()["stack_depth"] > 4
    pts = _dev(sc["points"][:64])
    h = wost.wost_solve(S.handle, pts, 16, sc["epsilon"], sc["r_min"], 256, seed=3, kernel=kernel,
                        **{knob: 2 if knob == "stack_depth" else 3})
    t0 = time.perf_counter()
    with pytest.raises(wost.WostError) as ei:
        wost.wost_wait(h, 120.0)
    assert ei.value.status == wost.ERR_INTERNAL
    assert time.perf_counter() - t0 < 60
    with pytest.raises(wost.WostError) as ei:
        wost.wost_poll(h, 64)
    assert ei.value.status == wost.ERR_INTERNAL
    wost.wost_solve_destroy(h)
    # the same solve with the defaults: no guard
    r = wost.solve(S, pts, 16, sc["epsilon"], sc["r_min"], 256, seed=3, kernel=kernel)
    assert r["guard_flags"] == 0
    S.close()


def test_autotune_picks_a_tried_block_and_keeps_the_walks(wost):
    sc = scenes.config2(grid=32, level=3)
    S = wost.Scene(sc)
    pts = _dev(sc["points"])
    before = wost.solve(S, pts, 32, sc["epsilon"], sc["r_min"], 4096, seed=8, kernel="persistent")
    t = wost.wost_scene_autotune(S.handle, pts, 16, sc["epsilon"], sc["r_min"], 4096)
    assert (t["lanes_per_walk"], t["block_size"]) in t["tried"] and len(t["tried"]) == 8
    assert {k[0] for k in t["tried"]} == {1, 8}
    assert t["steps_per_second"] == max(t["tried"].values()) > 0
    assert S.info()["lanes_per_walk"] == t["lanes_per_walk"]
    after = wost.solve(S, pts, 32, sc["epsilon"], sc["r_min"], 4096, seed=8, kernel="persistent",
                       lanes_per_walk=1)
    # the tuned block size runs the same walks
    np.testing.assert_allclose(after["mean"], before["mean"], rtol=1e-9, atol=1e-12)
    assert after["total_steps"] == before["total_steps"]
    S.close()


@pytest.mark.parametrize("kernel", ["persistent", "resumable"])
def test_team_layout_runs_the_same_walks(wost, kernel):
    """8 lanes per walk over the 8-wide trees (the layout the autotuner can
    pick at run time): with h = 0 the Neumann sampler cannot change an
    estimate, and every other query returns the same nearest answer as the
    one-lane traversal of the binary trees, so the walks are the same (up to
    single-precision rounding); with h != 0 against the exact solution."""
    sc = scenes.square_scene(8, fn="linear", params=(0.0, 0.0, 1.0, 0.0), neumann_sides=("left", "right"))
    rng = np.random.default_rng(71)
    pts = _dev((0.05 + 0.9 * rng.random((256, 2))).astype(np.float32))
    S = wost.Scene(sc)
    a = wost.solve(S, pts, 64, 1e-3, 0.0, 4096, seed=3, kernel=kernel, lanes_per_walk=1)
    b = wost.solve(S, pts, 64, 1e-3, 0.0, 4096, seed=3, kernel=kernel, lanes_per_walk=8)
    S.close()
    assert b["guard_flags"] == 0
    np.testing.assert_allclose(b["mean"], a["mean"], rtol=1e-5, atol=1e-6)
    fl = scenes.config1()
    S = wost.Scene(fl)
    r = wost.solve(S, _dev(fl["points"]), 512, fl["epsilon"], fl["r_min"], fl["max_steps"], seed=4, kernel=kernel,
                   lanes_per_walk=8)
    S.close()
    ref = oracle.solve(oracle.Scene(fl), fl["points"], 512, fl["epsilon"], fl["r_min"], fl["max_steps"], seed=4,
                       per_walk=True)
    u = scenes.exact_u("exp_cos", (), fl["points"])
    check_z(r["mean"] - u, r["se"], _allow(fl, fl["epsilon"]), label="team layout", walks=512,
            kurt=kurtosis(ref["per_walk"]))
    with pytest.raises(wost.WostError):  # teams serve persistent and resumable Poisson solves only
        wost.solve(wost.Scene(fl), _dev(fl["points"]), 4, fl["epsilon"], fl["r_min"], 64, kernel="plain",
                   lanes_per_walk=8)


def test_cancel_and_progressive_poll(wost):
    sc = scenes.config2(grid=64, level=4)
    S = wost.Scene(sc)
    n = len(sc["points"])
    h = wost.wost_solve(S.handle, _dev(sc["points"]), 4096, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=1,
                        kernel="persistent")
    m, se, wd, pr = wost.wost_poll(h, n)
    assert pr["walks_done"] <= n * 4096
    wost.wost_cancel(h)
    with pytest.raises(wost.WostError) as ei:
        wost.wost_wait(h, 120.0)
    assert ei.value.status == wost.ERR_CANCELLED
    m, se, wd, pr = wost.wost_poll(h, n)
    assert pr["done"] == 1 and pr["walks_done"] < n * 4096
    wost.wost_solve_destroy(h)
    S.close()
