"""The screened Poisson equation on the GPU (App. A.2; Tikhonov switch and
Russian roulette of Sec. 4.1; readings R14, R15): the single-precision
Green's function and step weight against the FP64 oracle, and walks against
exact screened solutions and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2302_11815_gb300 import scenes
from statcheck import check_z

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wost():
    from paper_2302_11815_gb300 import build as libbuild
    from paper_2302_11815_gb300 import wost as w

    assert torch.cuda.is_available()
    libbuild.build()
    w.load()
    return w


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sigma", [1e-3, 0.7, 30.0, 4000.0])
def test_screened_green_function_and_weight_match_the_oracle(wost, dim, sigma):
    rng = np.random.default_rng(11)
    R = rng.uniform(1e-3, 1.5, 400)
    rho = R * rng.uniform(1e-3, 1.0, 400)
    rho[:20] = R[:20]  # on the sphere: G = 0, Q = the walk-on-spheres weight
    G, Q = (t.cpu().numpy().astype(np.float64) for t in wost.wost_screened_kernels(dim, _dev(rho), _dev(R), sigma))
    rho32, R32 = rho.astype(np.float32).astype(np.float64), R.astype(np.float32).astype(np.float64)
    Go = np.array([oracle.screened_green_ball(dim, a, b, sigma) for a, b in zip(rho32, R32)])
    Qo = np.array([oracle.screened_q(dim, a, b, sigma) for a, b in zip(rho32, R32)])
    # Q is in [0, 1): absolute error; G: relative to its value at half the radius
    # (G -> 0 at the sphere, where the two terms of the formula cancel)
    np.testing.assert_allclose(Q, Qo, rtol=0, atol=3e-5)
    scale = np.array([abs(oracle.screened_green_ball(dim, 0.5 * b, b, sigma)) for b in R32])
    assert np.max(np.abs(G - Go) / (np.abs(Go) + scale)) < 3e-5


def _disk(neumann_frac, a):
    n = 128
    mask = np.arange(n) < int(round(neumann_frac * n))
    return scenes.disk_scene(n, "exp_plane", (1.0, a[0], a[1], 0.0), neumann=mask)


@pytest.mark.parametrize("kernel", ["persistent", "resumable"])
@pytest.mark.parametrize("neumann_frac", [0.0, 0.5, 1.0])
def test_walk_screened_disk_against_exact_and_oracle(wost, kernel, neumann_frac):
    a = (1.2, -0.7)
    sig = a[0] ** 2 + a[1] ** 2
    sc = _disk(neumann_frac, a)
    rng = np.random.default_rng(5)
    pts = scenes.ball_points(rng, 96, 2, 0.85)
    S = wost.Scene(sc)
    res = wost.solve(S, _dev(pts), 4096, 1e-3, 1e-3, 4096, seed=17, kernel=kernel, sigma=sig)
    S.close()
    assert res["done"] == 1 and res["capped_walks"] == 0 and res["guard_flags"] == 0
    u = scenes.exact_u("exp_plane", (1.0, a[0], a[1], 0.0), pts)
    check_z(res["mean"] - u, res["se"], 3e-3, label=f"gpu screened disk N={neumann_frac}")
    o = oracle.solve(oracle.Scene(sc), pts[:16], 600, 1e-3, max_steps=4096, seed=3, sigma=sig)
    se = np.hypot(o["se"], res["se"][:16])
    # 16 points: the outlier rule only (their mean z^2 scatters too much for a band)
    check_z(res["mean"][:16] - o["mean"], se, 0.0, band=None, label="gpu vs oracle screened")


def test_walk_screened_cube_3d(wost):
    a = (0.8, -0.5, 0.6)
    sig = sum(t * t for t in a)
    sc = scenes.cube_scene(m=4, fn="exp_plane", params=(1.0, *a), neumann_faces=(0, 3))
    rng = np.random.default_rng(7)
    pts = rng.uniform(-0.8, 0.8, size=(64, 3))
    S = wost.Scene(sc)
    res = wost.solve(S, _dev(pts), 4096, 1e-3, 1e-3, 4096, seed=29, kernel="persistent", sigma=sig)
    S.close()
    u = scenes.exact_u("exp_plane", (1.0, *a), pts)
    check_z(res["mean"] - u, res["se"], 4e-3, label="gpu screened cube")


def test_tikhonov_switch_and_pure_neumann_rules(wost):
    a = (0.9, 0.4)
    sc = _disk(0.5, a)
    pts = scenes.ball_points(np.random.default_rng(9), 32, 2, 0.8)
    S = wost.Scene(sc)
    # a switch beyond every walk leaves the Poisson walks (the same streams)
    p0 = wost.solve(S, _dev(pts), 256, 1e-3, 1e-3, 4096, seed=23, kernel="persistent")
    p1 = wost.solve(S, _dev(pts), 256, 1e-3, 1e-3, 4096, seed=23, kernel="persistent", sigma=5.0,
                    screen_after=100000)
    np.testing.assert_allclose(p1["mean"], p0["mean"], rtol=1e-5, atol=1e-6)
    assert p1["total_steps"] == p0["total_steps"]
    # screening from the first step shortens the walks
    p2 = wost.solve(S, _dev(pts), 256, 1e-3, 1e-3, 4096, seed=23, kernel="persistent", sigma=50.0)
    assert p2["total_steps"] < p0["total_steps"]
    S.close()
    # a pure Neumann scene needs sigma > 0
    pure = _disk(1.0, a)
    S = wost.Scene(pure)
    with pytest.raises(wost.WostError, match="sigma"):
        wost.solve(S, _dev(pts), 16, 1e-3, 1e-3, 64, seed=1)
    S.close()
