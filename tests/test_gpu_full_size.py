"""The benchmark workload at full size, in the launch configuration bench.py
times (persistent kernel, device-resident points, the full geometry and
parameters of the 512 x 512 Koch-snowflake grid).

  * the whole grid (141,021 points) at 16 walks per point: every walk
    accounted for, no guard fired, capped walks below 1e-3, and sampled
    points recomputed by the FP64 oracle with the same random streams agree
    within their standard errors;
  * a 2% random subsample of the grid at the benchmark's 256 walks per point:
    per-point z scores against the exact solution (multiple-comparisons test
    of statcheck.py), its mean z^2 band widened by the kurtosis of the walk
    estimates measured on the GPU from single-walk replicates of a subset;
  * the per-walk variance of the GPU estimator against the oracle's on the
    same points (the RMS error at equal walk counts is its square root);
  * the 3D workload (cube around the 200k-triangle noisy torus) at full
    geometry: a seeded subsample against the exact solution, and sampled
    points against the oracle on the same random streams.
"""
import numpy as np
import pytest

import oracle
from paper_2302_11815_gb300 import scenes
from statcheck import check_z, kurtosis

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WALKS_GRID = 16


@pytest.fixture(scope="module")
def setup():
    from paper_2302_11815_gb300 import build as libbuild
    from paper_2302_11815_gb300 import wost

    assert torch.cuda.is_available()
    libbuild.build()
    wost.load()
    sc = scenes.config2()
    S = wost.Scene(sc)
    yield wost, sc, S
    S.close()


@pytest.fixture(scope="module")
def grid(setup):
    wost, sc, S = setup
    res = wost.solve(S, torch.from_numpy(sc["points"]).cuda(), WALKS_GRID, sc["epsilon"], sc["r_min"],
                     sc["max_steps"], seed=777, kernel="persistent")
    return sc, res


def test_full_grid_accounting(grid):
    sc, res = grid
    n = len(sc["points"])
    assert n > 130000
    assert res["done"] == 1 and res["guard_flags"] == 0
    assert int(res["walks"].min()) == WALKS_GRID and int(res["walks"].sum()) == n * WALKS_GRID
    assert res["capped_walks"] <= 1e-3 * n * WALKS_GRID
    assert np.all(np.isfinite(res["mean"]))


def test_full_grid_sampled_points_against_oracle(grid):
    sc, res = grid
    rng = np.random.default_rng(12)
    idx = rng.choice(len(sc["points"]), 6, replace=False)
    O = oracle.Scene(sc)
    for i in idx:
        # walk j of point i draws the counters (j, i, step, slot): the oracle
        # recomputes point i with the same streams as the full-grid launch
        o = oracle.solve(O, sc["points"][i:i + 1], WALKS_GRID, sc["epsilon"], sc["r_min"], sc["max_steps"],
                         seed=777, point_base=int(i))
        se = np.hypot(o["se"][0], res["se"][i])
        assert abs(res["mean"][i] - o["mean"][0]) <= 4 * se + 1e-6, (i, res["mean"][i], o["mean"][0], se)


def test_subsample_at_benchmark_walks_against_exact(setup):
    wost, sc, S = setup
    rng = np.random.default_rng(13)
    idx = np.sort(rng.choice(len(sc["points"]), len(sc["points"]) // 50, replace=False))
    pts = sc["points"][idx]
    res = wost.solve(S, torch.from_numpy(pts).cuda(), sc["walks"], sc["epsilon"], sc["r_min"], sc["max_steps"],
                     seed=778, kernel="persistent")
    assert int(res["walks"].sum()) == len(pts) * sc["walks"]
    u = scenes.exact_u("sin2x_cos3y", (), pts)
    L = np.max(np.linalg.norm(scenes.exact_grad("sin2x_cos3y", (), sc["vertices"].astype(float)), axis=1))
    k = _replicate_kurtosis(wost, S, sc, pts[::8], sc["walks"], seed=779)
    check_z(res["mean"] - u, res["se"], sc["epsilon"] * 1.05 * L, label="subsample", walks=sc["walks"],
            kurt=np.full(len(pts), np.mean(k)))


def _replicate_kurtosis(wost, S, sc, pts, walks, seed):
    """Per-point kurtosis of single-walk estimates: each point repeated
    `walks` times with one walk each (independent streams by point index)."""
    rep = np.repeat(np.ascontiguousarray(pts, np.float32), walks, axis=0)
    r = wost.solve(S, torch.from_numpy(rep).cuda(), 1, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=seed,
                   kernel="persistent")
    return kurtosis(r["mean"].reshape(len(pts), walks))


def test_full_grid_walk_variance_against_oracle(setup):
    """Pooled per-walk variance of the GPU estimator against the oracle's on
    the same 32 points: the GPU may not be noisier (the RMS error at equal
    walks scales with its square root).  The allowance is the RMS ratio of
    1.1 squared plus the 99.9% spread of the ratio of two variance
    estimates, Var(ratio) ~ (kappa - 1)(1/n_gpu + 1/n_oracle)."""
    wost, sc, S = setup
    rng = np.random.default_rng(14)
    pts = sc["points"][rng.choice(len(sc["points"]), 32, replace=False)]
    g = wost.solve(S, torch.from_numpy(pts).cuda(), 256, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=31,
                   kernel="persistent")
    o = oracle.solve(oracle.Scene(sc), pts, 32, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=32, per_walk=True)
    var_g = float(np.mean(g["se"] ** 2 * 256))
    var_o = float(np.mean(np.var(o["per_walk"], axis=1, ddof=1)))
    kap = float(np.mean(kurtosis(o["per_walk"])))
    sd = np.sqrt(max(kap - 1.0, 2.0) * (1.0 / (32 * 256) + 1.0 / (32 * 32)))
    assert var_g <= var_o * (1.21 + 3.29 * sd), (var_g, var_o, kap)


@pytest.fixture(scope="module")
def torus():
    from paper_2302_11815_gb300 import wost

    sc = scenes.config3()
    S = wost.Scene(sc)
    yield wost, sc, S
    S.close()


def test_cube_torus_full_geometry_against_exact(torus):
    """2048 seeded slice points at least 0.01 from the noisy torus (nearer,
    the walks start amid the bumps' concave hollows, where hemispherical
    sampling and the r_min clamp carry the bias Sec. 4.4 acknowledges) at
    512 walks (at the workload's 128 the sample SE of the heavy-tailed
    estimates understates the spread at a few points)."""
    wost, sc, S = torus
    assert len(sc["prims"]) > 200000
    _, _, tube = scenes.torus_mesh(500, 200, seed=3001)
    rho, rs = tube(sc["points"].astype(np.float64))
    far = sc["points"][rho > rs + 0.01]
    rng = np.random.default_rng(15)
    pts = far[rng.choice(len(far), 2048, replace=False)]
    walks = 512
    res = wost.solve(S, torch.from_numpy(pts).cuda(), walks, sc["epsilon"], sc["r_min"], sc["max_steps"],
                     seed=41, kernel="resumable")
    assert res["guard_flags"] == 0 and res["capped_walks"] <= 1e-4 * len(pts) * walks
    u = scenes.exact_u("quad3", (), pts)
    k = _replicate_kurtosis(wost, S, sc, pts[::16], walks, seed=42)
    # per-corner data: g interpolated linearly on 1/16-wide cube faces (u
    # quadratic: bias up to h^2/8 |u''| = 1e-3) plus the epsilon shell
    check_z(res["mean"] - u, res["se"], 1e-3 + sc["epsilon"] * 1.05 * 3.0, label="cube torus", walks=walks,
            kurt=np.full(len(pts), np.mean(k)))


def test_cube_torus_full_geometry_sampled_points_against_oracle(torus):
    wost, sc, S = torus
    rng = np.random.default_rng(16)
    idx = rng.choice(len(sc["points"]), 4, replace=False)
    pts = np.ascontiguousarray(sc["points"][idx])
    g = wost.solve(S, torch.from_numpy(pts).cuda(), 16, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=43,
                   kernel="persistent")
    o = oracle.solve(oracle.Scene(sc), pts, 16, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=43)
    se = np.hypot(o["se"], g["se"])
    assert np.all(np.abs(g["mean"] - o["mean"]) <= 4 * se + 1e-6), (g["mean"], o["mean"], se)
