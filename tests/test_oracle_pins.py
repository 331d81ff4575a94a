"""Pins for the FP64 CPU oracle: checks against facts fixed by the paper and by
mathematics, not against the oracle itself.

  * Philox4x32-10 against the published known-answer vectors;
  * App. A: Green's function of the ball (normalisation by its flux, zero on
    the sphere, harmonic away from the centre) and its printed integrals;
  * Sec. 4.6 source sampling against the radial CDF of the normalised G_B
    (obtained by quadrature of G_B, not by retyping the sampler);
  * Q.1-Q.3 on tiny shapes with hand-derived answers;
  * Q.4 (Algs. 5-6): E[1{|z-x|<r}/pdf] equals the measure of the Neumann
    boundary inside the ball;
  * the walk: exact harmonic and Poisson solutions, the Poisson kernel of the
    disk (pure Dirichlet = walk on spheres), mixed Dirichlet/Neumann problems
    in 2D and 3D, 1/sqrt(N) convergence, and per-step invariants.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from statcheck import check_z, kurtosis
from paper_2302_11815_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split(":")
            w = [int(t, 16) for t in lhs.split()]
            want = [int(t, 16) for t in rhs.split()]
            got = oracle.philox(w[:4], w[4:6])
            assert [int(v) for v in got] == want
            rows += 1
    assert rows == 3


# ---------------------------------------------------------------------------
# App. A: Green's function of the ball
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_green_ball_is_the_dirichlet_green_function(dim):
    R = 0.7
    G = lambda rho: oracle.green_ball(dim, rho, R)
    # vanishes on the sphere
    assert abs(G(R)) < 1e-15
    # unit flux of -grad G through every sphere around the pole (delta source)
    area = (lambda rho: 2 * math.pi * rho) if dim == 2 else (lambda rho: 4 * math.pi * rho**2)
    for rho in (0.05, 0.3, 0.6):
        h = 1e-6 * rho
        dG = (G(rho + h) - G(rho - h)) / (2 * h)
        assert abs(-dG * area(rho) - 1.0) < 1e-6
    # harmonic away from the pole: radial Laplacian by finite differences
    for rho in (0.1, 0.4):
        h = 1e-4
        d2 = (G(rho + h) - 2 * G(rho) + G(rho - h)) / h**2
        d1 = (G(rho + h) - G(rho - h)) / (2 * h)
        assert abs(d2 + (dim - 1) / rho * d1) < 1e-4 * abs(d2)


def test_green_ball_integrals_match_app_a():
    want = {}
    with open(os.path.join(GOLDEN, "green_ball_app_a.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            d, c = line.split()
            want[int(d)] = float(c)
    for dim in (2, 3):
        for R in (0.25, 1.0, 3.0):
            shell = (lambda rho: 2 * math.pi * rho) if dim == 2 else (lambda rho: 4 * math.pi * rho**2)
            quad, _ = integrate.quad(lambda rho: oracle.green_ball(dim, rho, R) * shell(rho), 0, R,
                                     limit=200)
            assert abs(quad - want[dim] * R * R) < 1e-9 * R * R
            assert abs(oracle.green_ball_norm(dim, R) - want[dim] * R * R) < 1e-14 * R * R


@pytest.mark.parametrize("dim", [2, 3])
def test_source_radius_follows_normalised_green_function(dim):
    """Sec. 4.6: t ~ G_B(x, x + t v) along v.  The CDF of t/R is obtained
    here by quadrature of G_B times the shell measure."""
    R = 1.0
    shell = (lambda rho: rho) if dim == 2 else (lambda rho: rho**2)
    norm, _ = integrate.quad(lambda s: oracle.green_ball(dim, s, R) * shell(s), 0, R)
    grid = np.linspace(1e-9, 1.0, 2001)
    cdf_vals = np.array([integrate.quad(lambda s: oracle.green_ball(dim, s, R) * shell(s), 0, g)[0]
                         for g in grid]) / norm
    rng = np.random.default_rng(5)
    u = rng.random((20000, 2))
    t = np.array([oracle.source_radius(dim, R, a, b) for a, b in u])
    assert np.all((t > 0) & (t < R))
    res = stats.kstest(t, lambda q: np.interp(q, grid, cdf_vals))
    assert res.pvalue > 1e-3


# ---------------------------------------------------------------------------
# queries on tiny shapes
# ---------------------------------------------------------------------------
def _scene(dim, V, P, flags):
    return oracle.Scene({"dim": dim, "vertices": np.array(V, float), "prims": np.array(P, np.int32),
                         "flags": np.array(flags, np.uint8),
                         "g": {"kind": "analytic", "fn": "zero"}, "h": {"kind": "analytic", "fn": "zero"},
                         "f": {"kind": "none"}})


def test_q1_closest_point_2d_square():
    S = _scene(2, [[0, 0], [1, 0], [1, 1], [0, 1]], [[0, 1], [1, 2], [2, 3], [3, 0]], [0, 0, 0, 0])
    d, xb, pr = oracle.closest_dirichlet(S, [[0.3, 0.2], [0.9, 0.5], [2.0, 2.0], [-1.0, 0.5]])
    np.testing.assert_allclose(d, [0.2, 0.1, math.sqrt(2), 1.0], atol=1e-14)
    np.testing.assert_allclose(xb, [[0.3, 0], [1, 0.5], [1, 1], [0, 0.5]], atol=1e-14)
    assert list(pr[[0, 1, 3]]) == [0, 1, 3]


def test_q1_closest_point_3d_triangle_regions():
    S = _scene(3, [[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]], [0])
    q = [[0.2, 0.2, 0.5], [-1, -1, 0], [0.5, -1, 0], [1, 1, 0], [0.1, 0.1, -2]]
    d, xb, _ = oracle.closest_dirichlet(S, q)
    np.testing.assert_allclose(d, [0.5, math.sqrt(2), 1.0, math.sqrt(0.5), 2.0], atol=1e-14)
    np.testing.assert_allclose(xb[3], [0.5, 0.5, 0], atol=1e-14)


def test_q2_convex_neumann_polygon_has_no_silhouette_from_inside():
    # Sec. 4.4 / Sec. 5.1: from inside a convex region the Neumann boundary is
    # never a visibility silhouette, so d_sil = r_max
    V = scenes.regular_polygon(64)
    P = scenes.closed_polyline(V)
    S = _scene(2, V, P, np.ones(64))
    rng = np.random.default_rng(1)
    pts = scenes.ball_points(rng, 200, 2, 0.9)
    d, w = oracle.silhouette_distance(S, pts, 10.0)
    assert np.all(d == 10.0) and np.all(w == -1)


def test_q2_reflex_vertex_is_the_silhouette():
    # L-shaped room (all Neumann).  Seen from inside an arm, the reflex
    # corner (1,1) is the only silhouette point: one of its walls faces the
    # viewer and the other turns away.  From the square where the arms
    # overlap both walls face the viewer: no silhouette.
    V = [[0, 0], [2, 0], [2, 1], [1, 1], [1, 2], [0, 2]]
    P = scenes.closed_polyline(np.array(V, float))
    S = _scene(2, V, P, np.ones(6))
    q = np.array([[0.5, 1.5], [1.5, 0.5], [0.3, 0.4]])
    d, w = oracle.silhouette_distance(S, q, 100.0)
    want = np.linalg.norm(q - np.array([1.0, 1.0]), axis=1)
    want[2] = 100.0
    np.testing.assert_allclose(d, want, atol=1e-14)
    assert list(w[:2]) == [3, 3] and w[2] == -1


def test_q2_straight_wall_independent_of_subdivision():
    # Sec. 1: steps are independent of the tessellation; interior vertices of
    # a straight wall are never silhouettes, its two ends always are
    rng = np.random.default_rng(2)
    q = np.c_[rng.uniform(-2, 2, 100), rng.uniform(0.05, 1.5, 100)]
    ref = None
    for k in (1, 3, 16, 101):
        xs = np.linspace(-1, 1, k + 1)
        V = np.c_[xs, np.zeros(k + 1)]
        P = np.c_[np.arange(k), np.arange(1, k + 1)]
        S = _scene(2, V, P, np.ones(k))
        d, _ = oracle.silhouette_distance(S, q, 100.0)
        want = np.minimum(np.linalg.norm(q - [-1, 0], axis=1), np.linalg.norm(q - [1, 0], axis=1))
        np.testing.assert_allclose(d, want, atol=1e-13)
        ref = d if ref is None else ref
        np.testing.assert_allclose(d, ref, atol=1e-13)


def test_q2_3d_closed_cube_from_inside_and_open_triangle():
    V, P = scenes.cube_mesh(3)
    S = _scene(3, V, P, np.ones(len(P)))
    rng = np.random.default_rng(3)
    pts = rng.uniform(-0.9, 0.9, (100, 3))
    d, _ = oracle.silhouette_distance(S, pts, 7.0)
    assert np.all(d == 7.0)
    # a lone triangle: all three edges are boundary edges, hence silhouettes
    T = _scene(3, [[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]], [1])
    d, _ = oracle.silhouette_distance(T, [[0.2, 0.2, 0.3], [0.25, -0.5, 0.0]], 10.0)
    np.testing.assert_allclose(d, [math.sqrt(0.2**2 + 0.3**2), 0.5], atol=1e-14)


def test_q2_3d_sphere_silhouette_is_the_tangent_circle():
    V, P = scenes.sphere_mesh(48, 96, 1.0)
    S = _scene(3, V, P, np.ones(len(P)))
    for D in (1.5, 2.0, 4.0):
        d, _ = oracle.silhouette_distance(S, [[0.0, 0.3 * D, math.sqrt(1 - 0.09) * D]], 100.0)
        # within the angular resolution of the inscribed mesh (pi/48)
        assert abs(d[0] - math.sqrt(D * D - 1)) < 0.06 and d[0] > D - 1


def test_q3_ray_hits_2d_and_3d():
    S = _scene(2, [[0, 0], [1, 0], [1, 1], [0, 1]], [[0, 1], [1, 2], [2, 3], [3, 0]], [1, 1, 1, 0])
    hit, t, pr = oracle.intersect_neumann(S, [[0.5, 0.5], [0.5, 0.5], [0.5, 0.5]],
                                          [[0, -1], [1, 0], [-1, 0]], [1.0, 0.4, 1.0])
    assert list(hit) == [True, False, False]  # the left wall is Dirichlet
    assert abs(t[0] - 0.5) < 1e-15 and pr[0] == 0
    T = _scene(3, [[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]], [1])
    hit, t, _ = oracle.intersect_neumann(T, [[0.2, 0.2, 1.0]] * 4,
                                         [[0, 0, -1], [0, 0, -1], [0, 0, 1], [0, 0, -1]],
                                         [2.0, 0.5, 2.0, 2.0], skip=[-1, -1, -1, 0])
    assert list(hit) == [True, False, False, False]
    assert abs(t[0] - 1.0) < 1e-15


# ---------------------------------------------------------------------------
# Q.4: hierarchical Neumann sampling (Algs. 5-6) is unbiased
# ---------------------------------------------------------------------------
def _sample_measure(S, x, r, n, seed):
    vals = np.zeros(n)
    for i in range(n):
        z, _, pdf, pr = oracle.neumann_sample(S, x, r, seed, i, 0, 0)
        if pr >= 0 and pdf > 0 and np.linalg.norm(z - np.asarray(x)) < r:
            vals[i] = 1.0 / pdf
    return vals


def test_query_threshold_brackets_reduce_to_the_exact_queries():
    """The test-only bracket queries: at 0 they are Q.2 and Q.3; a larger
    threshold never gives a farther silhouette point or a farther hit."""
    for sc in (scenes.config1(), scenes.box_sphere_scene(m=3, n_lat=8, n_lon=16)):
        O = oracle.Scene(sc)
        rng = np.random.default_rng(5)
        d = sc["dim"]
        x = rng.uniform(-1.2, 1.2, (400, d))
        rm = np.full(len(x), 0.7)
        d0, _ = oracle.silhouette_distance(O, x, rm)
        np.testing.assert_array_equal(oracle.silhouette_distance_tol(O, x, rm, 0.0), d0)
        lo, hi = oracle.silhouette_distance_tol(O, x, rm, 1e-3), oracle.silhouette_distance_tol(O, x, rm, -1e-3)
        assert np.all(lo <= d0) and np.all(d0 <= hi)
        v = rng.normal(size=x.shape)
        h0, t0, _ = oracle.intersect_neumann(O, x, v, 0.8)
        h, t = oracle.intersect_neumann_tol(O, x, v, 0.8, 0.0)
        np.testing.assert_array_equal(h, h0)
        np.testing.assert_array_equal(t, t0)
        hl, tl = oracle.intersect_neumann_tol(O, x, v, 0.8, 1e-2)
        hh, th = oracle.intersect_neumann_tol(O, x, v, 0.8, -1e-2)
        assert np.all(tl <= t0) and np.all(t0 <= th) and np.all(hl >= h0) and np.all(hh <= h0)


def test_q4_measure_of_wall_in_ball_2d():
    k = 200
    xs = np.linspace(-2, 2, k + 1)
    S = _scene(2, np.c_[xs, 0.05 * np.sin(0 * xs)], np.c_[np.arange(k), np.arange(1, k + 1)], np.ones(k))
    x, r = [0.1, 0.3], 0.5
    vals = _sample_measure(S, x, r, 20000, 11)
    want = 2 * math.sqrt(r * r - 0.3**2)
    assert abs(vals.mean() - want) < 4 * vals.std() / math.sqrt(len(vals))
    # ball covering the whole boundary: E[1/pdf] = total length
    vals = _sample_measure(S, [0.0, 0.5], 10.0, 4000, 12)
    assert abs(vals.mean() - 4.0) < 1e-9 * 4 + 4 * vals.std() / math.sqrt(len(vals))


def test_q4_measure_of_plate_in_ball_3d():
    m = 24
    g = np.linspace(-1, 1, m + 1)
    A, B = np.meshgrid(g, g, indexing="ij")
    V = np.c_[A.ravel(), B.ravel(), np.zeros(A.size)]
    idx = np.arange((m + 1) ** 2).reshape(m + 1, m + 1)
    a, b, c, d = idx[:-1, :-1].ravel(), idx[1:, :-1].ravel(), idx[1:, 1:].ravel(), idx[:-1, 1:].ravel()
    P = np.concatenate([np.c_[a, b, c], np.c_[a, c, d]])
    S = _scene(3, V, P, np.ones(len(P)))
    x, r = [0.1, -0.2, 0.3], 0.5
    vals = _sample_measure(S, x, r, 20000, 13)
    want = math.pi * (r * r - 0.09)
    assert abs(vals.mean() - want) < 4 * vals.std() / math.sqrt(len(vals))


# ---------------------------------------------------------------------------
# the walk (Alg. 1) against exact solutions
# ---------------------------------------------------------------------------
def _check_exact(sc, pts, walks, eps, seed=7, z=4.0, r_min=None, chi2=True, max_steps=1024):
    S = oracle.Scene(sc)
    res = oracle.solve(S, pts, walks, eps, r_min, max_steps, seed=seed, per_walk=True)
    fn, pr = sc["exact"]
    u = scenes.exact_u(fn, pr, pts)
    # epsilon-shell bias bound: |u(xbar) - u(x)| <= eps * max|grad u|
    L = np.max(np.linalg.norm(scenes.exact_grad(fn, pr, sc["vertices"].astype(float)), axis=1))
    allow = eps * 1.05 * L
    err = res["mean"] - u
    assert res["capped"].sum() == 0
    check_z(err, res["se"], allow, zthr=z, band=chi2, walks=walks, kurt=kurtosis(res["per_walk"]))
    return res, u


def test_walk_pure_dirichlet_harmonic_disk():
    # pure Dirichlet: WoSt reduces to walk on spheres (Sec. 3.4, Sec. 4.3)
    rng = np.random.default_rng(21)
    pts = scenes.ball_points(rng, 64, 2, 0.9)
    _check_exact(scenes.disk_scene(256, "exp_cos"), pts, 1024, 1e-3)


def test_walk_poisson_kernel_of_the_disk():
    """Dirichlet data = indicator of the arc [0, pi/2] on the unit circle:
    u(x) is the harmonic measure, the integral of the disk's Poisson kernel
    (1 - |x|^2) / (2 pi |x - z|^2) over the arc."""
    n = 1024
    sc = scenes.disk_scene(n, "zero")
    ind = (np.arange(n) < n // 4).astype(np.float32)
    sc["g"] = {"kind": "per_corner", "values": np.c_[ind, ind]}
    S = oracle.Scene(sc)
    rng = np.random.default_rng(22)
    pts = scenes.ball_points(rng, 48, 2, 0.85)
    res = oracle.solve(S, pts, 2048, 1e-4, None, 1024, seed=3, per_walk=True)

    def hm(x):
        f = lambda th: (1 - x @ x) / (2 * np.pi * ((x[0] - np.cos(th)) ** 2 + (x[1] - np.sin(th)) ** 2))
        return integrate.quad(f, 0, np.pi / 2, limit=200)[0]

    want = np.array([hm(p.astype(float)) for p in pts])
    check_z(res["mean"] - want, res["se"], 0.0, walks=2048, kurt=kurtosis(res["per_walk"]))
    # the centre sees a quarter of the circle
    c = oracle.solve(S, np.zeros((1, 2)), 8192, 1e-4, None, 1024, seed=4)
    assert abs(c["mean"][0] - 0.25) < 4 * c["se"][0]


def test_walk_source_term_sign_and_norm_2d_3d():
    # -Lap u = 1 with u = (1 - |x|^2)/(2 dim): pins the sign of S and |G_B|
    rng = np.random.default_rng(23)
    _check_exact(scenes.disk_scene(256, "bump", source=True), scenes.ball_points(rng, 48, 2, 0.9), 1024, 1e-3)
    _check_exact(scenes.cube_scene(4, "bump", source=True), rng.uniform(-0.8, 0.8, (32, 3)), 512, 1e-3)


def test_walk_mixed_flower_exp_cos():
    # the 64-segment flower with alternating Dirichlet/Neumann segments and
    # u = e^x cos y: pins the sign of the Neumann term, alpha and the hemisphere
    sc = scenes.config1()
    res, u = _check_exact(sc, sc["points"], 512, 1e-3)
    rel = np.sqrt(np.mean((res["mean"] - u) ** 2) / np.mean(u**2))
    assert rel < 0.05


def test_walk_mixed_square_and_annulus():
    rng = np.random.default_rng(24)
    pts = (0.05 + 0.9 * rng.random((48, 2))).astype(np.float32)
    _check_exact(scenes.square_scene(8), pts, 1024, 1e-3)  # u = y, Neumann top/bottom
    ann = scenes.annulus_scene()
    r = np.sqrt(rng.uniform(0.35**2, 0.95**2, 48))
    th = rng.uniform(0, 2 * np.pi, 48)
    _check_exact(ann, np.c_[r * np.cos(th), r * np.sin(th)].astype(np.float32), 1024, 1e-3)


def test_walk_sin2x_cos3y_poisson_with_neumann_arc():
    """The bench workload's data: u = sin 2x cos 3y with f = -Lap u = 13 u
    (analytic g = u, h = grad u . n, f) on a disk, all Dirichlet and then
    with a Neumann upper half.  A wrong factor in f (12 u), a wrong sign of
    a term of grad u (h) or a wrong frequency in u (g) fails it (each
    planted in the oracle and checked)."""
    n = 256
    rng = np.random.default_rng(31)
    # all Dirichlet first: low variance, so the source term (a third of the
    # size of u here) is resolved to about 1/30 of its size
    _check_exact(scenes.disk_scene(n, "sin2x_cos3y", source=True), scenes.ball_points(rng, 48, 2, 0.9), 8192, 1e-4)
    th = 2 * np.pi * (np.arange(n) + 0.5) / n
    sc = scenes.disk_scene(n, "sin2x_cos3y", neumann=(np.sin(th) > 0).astype(np.uint8), source=True)
    _check_exact(sc, scenes.ball_points(rng, 64, 2, 0.9), 2048, 1e-4)


def _linear_square(data):
    return scenes.square_scene(8, fn="linear", params=(0.3, 0.7, -1.2, 0.0), neumann_sides=("bottom", "top"),
                               data=data)


def test_walk_per_vertex_data_exact_for_linear_u_2d():
    """Per-vertex g and h (the layout the workloads specify) interpolated
    linearly on each segment are exact for a linear u on a polygon whose
    Neumann sides are straight, so the walk must reach the exact solution;
    and with the corner values taken from the vertices, the per-vertex path
    must reproduce the per-corner path walk for walk (same streams).  A
    vertex read by corner position instead of by the primitive's vertex
    index fails both."""
    sc = _linear_square("per_vertex")
    rng = np.random.default_rng(32)
    pts = (0.05 + 0.9 * rng.random((48, 2))).astype(np.float32)
    res, _ = _check_exact(sc, pts, 1024, 1e-3)
    P = sc["prims"]
    corner = dict(sc, g={"kind": "per_corner", "values": sc["g"]["values"][P]},
                  h={"kind": "per_corner", "values": sc["h"]["values"][P]})
    a = oracle.solve(oracle.Scene(sc), pts, 64, 1e-3, None, 1024, seed=5)
    b = oracle.solve(oracle.Scene(corner), pts, 64, 1e-3, None, 1024, seed=5)
    np.testing.assert_allclose(a["mean"], b["mean"], rtol=0, atol=1e-12)
    # per-vertex data on a curved, mixed boundary: still the per-corner
    # path walk for walk
    fl = scenes.config1(data="per_vertex")
    fc = dict(fl, g={"kind": "per_corner", "values": fl["g"]["values"][fl["prims"]]},
              h={"kind": "per_corner", "values": fl["h"]["values"][fl["prims"]]})
    a = oracle.solve(oracle.Scene(fl), fl["points"][:32], 32, 1e-3, None, 1024, seed=6)
    b = oracle.solve(oracle.Scene(fc), fl["points"][:32], 32, 1e-3, None, 1024, seed=6)
    np.testing.assert_allclose(a["mean"], b["mean"], rtol=0, atol=1e-12)


def test_walk_per_vertex_data_exact_for_linear_u_3d():
    """3D: a cube with one Neumann face (+z) and per-vertex data of a linear
    u; per-vertex h is averaged over the Neumann triangles at a vertex, all
    of which lie in that face, so the data are exact."""
    sc = scenes.cube_scene(4, fn="linear", params=(0.2, 0.5, -0.3, 0.8), neumann_faces=(5,), data="per_vertex")
    rng = np.random.default_rng(33)
    _check_exact(sc, rng.uniform(-0.85, 0.85, (32, 3)).astype(np.float32), 1024, 1e-3)


# ---------------------------------------------------------------------------
# double-sided boundaries (App. B)
# ---------------------------------------------------------------------------
def _slit_points(rng, n):
    p = rng.uniform(-0.95, 0.95, (4 * n, 2))
    keep = (np.abs(p[:, 1]) > 0.05) | (p[:, 0] < -0.05)
    return p[keep][:n].astype(np.float32)


def test_walk_double_sided_dirichlet_slit():
    """App. B, double-sided Dirichlet data: the square with a slit from the
    centre to the right side, u = polar angle in [0, 2 pi): 0 on the slit's
    upper side, 2 pi on its lower side.  A walk ending at the slit must take
    the data of the side it is on; the wrong side is off by 2 pi."""
    sc = scenes.slit_square_scene()
    rng = np.random.default_rng(51)
    pts = _slit_points(rng, 64)
    S = oracle.Scene(sc)
    res = oracle.solve(S, pts, 1024, 1e-4, None, 1024, seed=5, per_walk=True)
    u = scenes.exact_u("polar_angle", (), pts)
    # shell bias: |grad u| = 1/rho is large only near the slit's tip
    check_z(res["mean"] - u, res["se"], 1e-4 * 1.05 / 0.05, walks=1024, kurt=kurtosis(res["per_walk"]))


def test_walk_double_sided_neumann_crack():
    """App. B at a Neumann crack: the square with a zero-flux crack from the
    centre to the right side, u = sqrt(rho) cos(theta/2), which jumps by
    2 sqrt(rho) across the crack.  A walk that hits the crack must leave on
    the side it came from; one that crossed would carry the other side's
    value (the rule that keeps it on its side is checked by planting it
    out of the oracle)."""
    sc = scenes.crack_square_scene()
    rng = np.random.default_rng(54)
    pts = _slit_points(rng, 64)
    S = oracle.Scene(sc)
    res = oracle.solve(S, pts, 1024, 1e-4, None, 4096, seed=6, per_walk=True)
    assert res["capped"].sum() == 0
    u = scenes.exact_u("crack_mode", (), pts)
    # |grad u| = 1 / (2 sqrt(rho)), large only next to the tip
    check_z(res["mean"] - u, res["se"], 1e-4 * 1.05 * 3.0, walks=1024, kurt=kurtosis(res["per_walk"]))


@pytest.mark.parametrize("data", ["analytic", "per_corner", "per_corner_minus"])
def test_walk_double_sided_neumann_sheet_2d(data):
    """App. B, double-sided Neumann data: a Neumann sheet inside a Dirichlet
    square, u linear with du/dy = 1.5 across the sheet: h+ = -1.5 on the
    upper (+) side, h- = +1.5 below.  Sheet hits must keep the walk on its
    side and Neumann samples must use the data of the side facing the walk;
    either mistake biases the means by many SE."""
    sc = scenes.sheet_square_scene(data=data)
    rng = np.random.default_rng(52)
    p = rng.uniform(-0.9, 0.9, (400, 2))
    pts = p[(np.abs(p[:, 1] - 0.1) > 0.03) | (np.abs(p[:, 0]) > 0.55)][:64].astype(np.float32)
    _check_exact(sc, pts, 1024, 1e-3)


def test_walk_double_sided_neumann_plate_3d():
    sc = scenes.plate_cube_scene()
    rng = np.random.default_rng(53)
    p = rng.uniform(-0.85, 0.85, (400, 3))
    pts = p[(np.abs(p[:, 2] - 0.1) > 0.04) | (np.abs(p[:, 0]) > 0.55) | (np.abs(p[:, 1]) > 0.55)][:48]
    _check_exact(sc, pts.astype(np.float32), 1024, 1e-3, max_steps=16384)


def test_walk_3d_cube_around_neumann_sphere():
    sc = scenes.box_sphere_scene()
    rng = np.random.default_rng(25)
    p = rng.uniform(-0.9, 0.9, (200, 3))
    p = p[np.linalg.norm(p, axis=1) > 0.5][:32].astype(np.float32)
    _check_exact(sc, p, 512, 1e-3)


def test_walk_3d_pure_dirichlet_cube_quad():
    rng = np.random.default_rng(26)
    _check_exact(scenes.cube_scene(4, "quad3"), rng.uniform(-0.9, 0.9, (32, 3)).astype(np.float32), 512, 1e-3)


def test_walk_rmse_converges_as_one_over_sqrt_n():
    # Sec. 6.2: error of magnitude O(1/sqrt(N))
    sc = scenes.disk_scene(256, "exp_cos", neumann=(np.arange(256) < 64).astype(np.uint8))
    S = oracle.Scene(sc)
    rng = np.random.default_rng(27)
    pts = scenes.ball_points(rng, 64, 2, 0.8)
    u = scenes.exact_u("exp_cos", (), pts)
    Ns = [16, 64, 256, 1024]
    rmse = []
    for i, N in enumerate(Ns):
        res = oracle.solve(S, pts, N, 1e-4, None, 1024, seed=100 + i)
        rmse.append(np.sqrt(np.mean((res["mean"] - u) ** 2)))
    slope = np.polyfit(np.log(Ns), np.log(rmse), 1)[0]
    assert -0.65 < slope < -0.35, slope


# ---------------------------------------------------------------------------
# per-step invariants of the walk
# ---------------------------------------------------------------------------
def _silhouette_vertices_2d(sc):
    V = sc["vertices"].astype(float)
    n = scenes.prim_normals(sc)
    adj = {}
    for p in np.nonzero(sc["flags"])[0]:
        for k in range(2):
            adj.setdefault(int(sc["prims"][p, k]), []).append(n[p])
    return V, adj


@pytest.mark.parametrize("which", ["flower", "koch"])
def test_walk_step_invariants(which):
    sc = scenes.config1() if which == "flower" else scenes.config2(grid=24, level=3)
    eps = sc["epsilon"]
    S = oracle.Scene(sc)
    V, adj = _silhouette_vertices_2d(sc)
    Nseg = np.nonzero(sc["flags"])[0]
    A = V[sc["prims"][Nseg, 0]]
    B = V[sc["prims"][Nseg, 1]]
    checked = 0
    npts, nw = (40, 4) if which == "flower" else (12, 2)
    for i, x0 in enumerate(sc["points"][:npts]):
        for j in range(nw):
            val, rows, capped = oracle.walk_trace(S, x0, i, j, eps, sc["r_min"], sc["max_steps"], seed=9)
            assert not capped and np.isfinite(val)
            for k in range(len(rows) - 1):
                x, onN, dD, dsil, r, hit, tb = rows[k, [0, 1]], rows[k, 3], rows[k, 4], rows[k, 5], rows[k, 6], rows[k, 7], rows[k, 8]
                assert dD >= eps and r <= dD and r >= min(sc["r_min"], dD) - 1e-15
                xn = rows[k + 1, [0, 1]]
                assert np.linalg.norm(xn - x) <= r * (1 + 1e-9) + 1e-9
                if rows[k + 1, 3]:  # next point lies on the Neumann boundary
                    e = B - A
                    t = np.clip(np.sum((xn - A) * e, 1) / np.sum(e * e, 1), 0, 1)
                    assert np.min(np.linalg.norm(A + t[:, None] * e - xn, axis=1)) < 1e-9
                if not onN and r > sc["r_min"] * (1 + 1e-12):
                    # no visibility-silhouette vertex strictly inside the star ball
                    for vid, ns in adj.items():
                        v = V[vid] - x
                        dv = np.linalg.norm(v)
                        if dv < r * (1 - 1e-12):
                            assert len(ns) == 2 and (v @ ns[0]) * (v @ ns[1]) > 0
                    checked += 1
    assert checked > 100


def test_walk_outside_the_grown_bounding_box_ends_at_once():
    # R13: the unit square's box grown by its side is [-1, 2]^2.  A walk
    # started outside it ends in its first step as a capped walk with g at the
    # closest Dirichlet point (R5); one started outside the domain but inside
    # the grown box is not stopped by the rule; a non-finite start ends with
    # no boundary term.
    sc = scenes.square_scene(m=4, fn="linear", params=(0.5, 1.0, 2.0, 0.0), neumann_sides=("bottom", "top"))
    O = oracle.Scene(sc)
    far = np.array([[2.5, 0.25], [-1.25, 0.75]])
    r = oracle.solve(O, far, 8, 1e-3, max_steps=1024, seed=3)
    assert np.all(r["steps"] == 8) and np.all(r["capped"] == 8)
    # closest Dirichlet points: (1, 0.25) on the right side, (0, 0.75) on the left
    expect = 0.5 + 1.0 * np.array([1.0, 0.0]) + 2.0 * np.array([0.25, 0.75])
    np.testing.assert_allclose(r["mean"], expect, rtol=0, atol=1e-12)
    near = oracle.solve(O, np.array([[1.5, 0.5]]), 8, 1e-3, max_steps=1024, seed=3)
    assert near["steps"][0] > 8
    nan = oracle.solve(O, np.array([[np.nan, 0.5]]), 4, 1e-3, max_steps=1024, seed=3)
    assert nan["steps"][0] == 4 and nan["capped"][0] == 4 and nan["mean"][0] == 0.0


# ---------------------------------------------------------------------------
# screened Poisson equation (App. A.2) and the Tikhonov switch (Sec. 4.1)
# ---------------------------------------------------------------------------
def test_scaled_bessel_functions_match_scipy():
    from scipy import special

    x = np.logspace(-4, 3, 29)
    b = oracle.bessel_scaled(x)
    ref = np.stack([special.i0e(x), special.i1e(x), special.k0e(x), special.k1e(x)], 1)
    np.testing.assert_allclose(b, ref, rtol=1e-10, atol=0)


def _dG(dim, rho, R, sig, h):
    return (oracle.screened_green_ball(dim, rho + h, R, sig) - oracle.screened_green_ball(dim, rho - h, R, sig)) / (2 * h)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("R,sig", [(0.3, 0.5), (1.5, 10.0), (0.8, 400.0)])
def test_screened_green_function_of_the_ball(dim, R, sig):
    G = lambda r: oracle.screened_green_ball(dim, r, R, sig)  # noqa: E731
    sphere = 2 * math.pi if dim == 2 else 4 * math.pi
    # zero on the sphere
    assert abs(G(R)) < 1e-12 * abs(G(0.5 * R))
    # -G'' - (dim-1)/r G' + sigma G = 0 away from the centre
    for rho in (0.2 * R, 0.5 * R, 0.9 * R):
        h = 1e-4 * rho
        d2 = (G(rho + h) - 2 * G(rho) + G(rho - h)) / h**2
        d1 = (G(rho + h) - G(rho - h)) / (2 * h)
        res = -d2 - (dim - 1) / rho * d1 + sig * G(rho)
        assert abs(res) < 1e-5 * (abs(d2) + abs(sig * G(rho))), (rho, res)
    # unit source: the flux through a small sphere around the centre is 1
    rho = 1e-6 * R
    assert abs(-sphere * rho ** (dim - 1) * _dG(dim, rho, R, sig, 1e-3 * rho) - 1.0) < 1e-4
    # Q = P^sigma_B / P^free = -|S^(dim-1)| rho^(dim-1) dG/drho at every rho
    for rho in (0.1 * R, 0.5 * R, R):
        q = oracle.screened_q(dim, rho, R, sig)
        fd = -sphere * rho ** (dim - 1) * _dG(dim, rho, R, sig, 1e-5 * rho)
        assert abs(q - fd) < 1e-6 * abs(fd), (rho, q, fd)
        assert 0.0 <= q < 1.0
    # |G^sigma_B| is the integral of G over the ball
    quad, _ = integrate.quad(lambda r: G(r) * sphere * r ** (dim - 1), 0, R, limit=200, points=[1e-6 * R])
    norm = oracle.screened_green_ball_norm(dim, R, sig)
    assert abs(norm - quad) < 1e-8 * norm


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_green_function_tends_to_the_unscreened_one(dim):
    R, sig = 0.7, 1e-9
    for rho in (0.05, 0.3, 0.6):
        assert abs(oracle.screened_green_ball(dim, rho, R, sig) / oracle.green_ball(dim, rho, R) - 1) < 1e-6
        assert abs(oracle.screened_q(dim, rho, R, sig) - 1) < 1e-6
    # (the closed form of the norm cancels at tiny sigma: checked at 1e-6,
    # where the true relative difference is O(R^2 sigma))
    assert abs(oracle.screened_green_ball_norm(dim, R, 1e-6) / (R * R / (4 if dim == 2 else 6)) - 1) < 1e-5


def _exp_plane_disk(neumann_frac, a=(1.2, -0.7)):
    n = 128
    mask = np.arange(n) < int(round(neumann_frac * n))
    sc = scenes.disk_scene(n, "exp_plane", (1.0, a[0], a[1], 0.0), neumann=mask)
    return sc, a[0] ** 2 + a[1] ** 2


@pytest.mark.parametrize("neumann_frac", [0.0, 0.5, 1.0])
def test_walk_screened_disk_exp_plane(neumann_frac):
    # -Lap u + sigma u = 0 for u = exp(a.x), sigma = |a|^2: Dirichlet, mixed
    # and pure Neumann (the screened problem is well posed without any
    # Dirichlet boundary; walks end by Russian roulette)
    sc, sig = _exp_plane_disk(neumann_frac)
    rng = np.random.default_rng(5)
    pts = scenes.ball_points(rng, 24, 2, 0.85)
    O = oracle.Scene(sc)
    # pure Neumann walks sum many heavy-tailed Neumann terms: more walks for
    # a trustworthy standard error
    walks = 2000 if neumann_frac == 1.0 else 600
    r = oracle.solve(O, pts, walks, 1e-3, max_steps=4096, seed=17, sigma=sig, per_walk=True)
    u = scenes.exact_u("exp_plane", (1.0, 1.2, -0.7, 0.0), pts)
    check_z(r["mean"] - u, r["se"], 1e-3 * 3.0, label=f"screened disk N={neumann_frac}", walks=walks, kurt=kurtosis(r["per_walk"]))
    assert r["capped"].sum() == 0


def test_walk_screened_source_and_tikhonov_switch():
    # u = exp(a.x) with sigma = 2|a|^2 needs f = -Lap u + sigma u = |a|^2 u,
    # given here on a fine grid (bilinear interpolation error ~1e-5)
    a = (0.9, 0.4)
    sig0 = a[0] ** 2 + a[1] ** 2
    sc = scenes.disk_scene(128, "exp_plane", (1.0, a[0], a[1], 0.0))
    ng = 513
    xs = np.linspace(-1.05, 1.05, ng)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    fv = sig0 * np.exp(a[0] * X + a[1] * Y)
    sc["f"] = {"kind": "grid", "origin": [xs[0], xs[0], 0.0], "spacing": [xs[1] - xs[0]] * 2 + [1.0],
               "dims": [ng, ng, 1], "values": fv.astype(np.float32).ravel()}
    O = oracle.Scene(sc)
    rng = np.random.default_rng(6)
    pts = scenes.ball_points(rng, 16, 2, 0.8)
    r = oracle.solve(O, pts, 800, 1e-3, max_steps=4096, seed=19, sigma=2 * sig0, per_walk=True)
    u = scenes.exact_u("exp_plane", (1.0, a[0], a[1], 0.0), pts)
    check_z(r["mean"] - u, r["se"], 3e-3, label="screened source", walks=800, kurt=kurtosis(r["per_walk"]))
    # a switch beyond every walk's length leaves the Poisson walks unchanged
    sc0 = scenes.disk_scene(128, "exp_plane", (1.0, a[0], a[1], 0.0))
    O0 = oracle.Scene(sc0)
    p0 = oracle.solve(O0, pts[:8], 64, 1e-3, max_steps=4096, seed=23)
    p1 = oracle.solve(O0, pts[:8], 64, 1e-3, max_steps=4096, seed=23, sigma=5.0, screen_after=100000)
    np.testing.assert_array_equal(p0["mean"], p1["mean"])
    np.testing.assert_array_equal(p0["steps"], p1["steps"])
    # screening from step 0 shortens the walks (roulette)
    p2 = oracle.solve(O0, pts[:8], 64, 1e-3, max_steps=4096, seed=23, sigma=50.0)
    assert p2["steps"].sum() < p0["steps"].sum()


def test_walk_screened_cube_exp_plane_3d():
    a = (0.8, -0.5, 0.6)
    sig = sum(t * t for t in a)
    sc = scenes.cube_scene(m=4, fn="exp_plane", params=(1.0, *a), neumann_faces=(0, 3))
    O = oracle.Scene(sc)
    rng = np.random.default_rng(7)
    pts = rng.uniform(-0.8, 0.8, size=(24, 3))
    r = oracle.solve(O, pts, 1500, 1e-3, max_steps=4096, seed=29, sigma=sig, per_walk=True)
    u = scenes.exact_u("exp_plane", (1.0, *a), pts)
    check_z(r["mean"] - u, r["se"], 1e-3 * 4.0, label="screened cube", walks=1500, kurt=kurtosis(r["per_walk"]))


@pytest.mark.parametrize("where", ["mid", "near_end"])
def test_walk_from_points_on_the_neumann_boundary(where):
    # Alg. 1 admits x0 on the Neumann boundary (its normal n_x given): the
    # first step samples the hemisphere about -n_x and weights the Neumann
    # term with alpha = 1/2 (R8).  Points on Neumann segments of the flower
    # scene, against the exact solution.
    sc = scenes.config1()
    V = sc["vertices"].astype(np.float64)
    P = sc["prims"]
    nrm = scenes.prim_normals(sc)
    odd = np.nonzero(sc["flags"] == 1)[0][::4]
    s = 0.5 if where == "mid" else 0.9
    pts = V[P[odd, 0]] * (1 - s) + V[P[odd, 1]] * s
    O = oracle.Scene(sc)
    r = oracle.solve(O, pts, 3000, 1e-3, max_steps=1024, seed=41, normals=nrm[odd], on_neumann=np.ones(len(odd)), per_walk=True)
    u = scenes.exact_u("exp_cos", (), pts)
    # (alpha = 1 instead of 1/2 at these points fails this check)
    check_z(r["mean"] - u, r["se"], 1e-3 * 3.0, label=f"boundary points {where}", walks=3000, kurt=kurtosis(r["per_walk"]))


def test_walk_screened_pure_neumann_cube_3d():
    # every face Neumann: well posed only for sigma > 0; walks end by roulette
    a = (0.7, 0.3, -0.5)
    sig = sum(t * t for t in a)
    sc = scenes.cube_scene(m=4, fn="exp_plane", params=(1.0, *a), neumann_faces=(0, 1, 2, 3, 4, 5))
    O = oracle.Scene(sc)
    pts = np.random.default_rng(8).uniform(-0.8, 0.8, size=(16, 3))
    r = oracle.solve(O, pts, 2000, 1e-3, max_steps=4096, seed=31, sigma=sig, per_walk=True)
    assert r["capped"].sum() == 0
    check_z(r["mean"] - scenes.exact_u("exp_plane", (1.0, *a), pts), r["se"], 0.0, label="screened Neumann cube", walks=2000, kurt=kurtosis(r["per_walk"]))


def test_walk_from_points_on_a_neumann_sphere_3d():
    # starts on the inner Neumann sphere of the box-sphere scene (normals out
    # of the domain, i.e. into the sphere), against the exact solution
    sc = scenes.box_sphere_scene(data="analytic")
    nrm = scenes.prim_normals(sc)
    V = sc["vertices"].astype(np.float64)
    P = sc["prims"]
    sphere = np.nonzero(sc["flags"] == 1)[0][::37]
    pts = (V[P[sphere, 0]] + V[P[sphere, 1]] + V[P[sphere, 2]]) / 3.0
    O = oracle.Scene(sc)
    r = oracle.solve(O, pts, 2000, 1e-3, max_steps=1024, seed=43, normals=nrm[sphere],
                     on_neumann=np.ones(len(sphere)), per_walk=True)
    u = scenes.exact_u("quad3", (), pts)
    check_z(r["mean"] - u, r["se"], 1e-3 * 3.0, label="boundary points on a sphere", walks=2000, kurt=kurtosis(r["per_walk"]))
