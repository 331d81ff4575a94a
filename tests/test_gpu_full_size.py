"""The benchmark workload at full size, in the launch configuration bench.py
times (persistent kernel, device-resident points): every point of the
512 x 512 Koch-snowflake grid, the full geometry and parameters, at 16 walks
per point (a sixteenth of the benchmark's 256, which keeps the test near a
minute: the full solve is about 1.1e11 walk steps).

  * whole grid: every walk accounted for, no guard fired, capped walks
    below 1e-3, per-point z scores against the exact solution (multiple-
    comparisons test of statcheck.py);
  * sampled points: the FP64 oracle recomputes a few points with the same
    random streams; per-point means agree within their standard errors.
"""
import numpy as np
import pytest

import oracle
from paper_2302_11815_gb300 import scenes
from statcheck import check_z

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    from paper_2302_11815_gb300 import build as libbuild
    from paper_2302_11815_gb300 import wost

    assert torch.cuda.is_available()
    libbuild.build()
    wost.load()
    sc = scenes.config2()
    sc["walks"] = WALKS
    S = wost.Scene(sc)
    res = wost.solve(S, torch.from_numpy(sc["points"]).cuda(), sc["walks"], sc["epsilon"], sc["r_min"],
                     sc["max_steps"], seed=777, kernel="persistent")
    S.close()
    return sc, res


WALKS = 16


def test_full_grid_accounting(run):
    sc, res = run
    n = len(sc["points"])
    assert n > 130000
    assert res["done"] == 1 and res["guard_flags"] == 0
    assert int(res["walks"].min()) == sc["walks"] and int(res["walks"].sum()) == n * sc["walks"]
    assert res["capped_walks"] <= 1e-3 * n * sc["walks"]


def test_full_grid_against_exact_solution(run):
    sc, res = run
    u = scenes.exact_u("sin2x_cos3y", (), sc["points"])
    L = np.max(np.linalg.norm(scenes.exact_grad("sin2x_cos3y", (), sc["vertices"].astype(float)), axis=1))
    check_z(res["mean"] - u, res["se"], sc["epsilon"] * 1.05 * L, band=(0.5, 2.0), label="full grid",
            dof=WALKS - 1, zthr=6.0)


def test_sampled_points_against_oracle(run):
    sc, res = run
    rng = np.random.default_rng(12)
    idx = rng.choice(len(sc["points"]), 4, replace=False)
    O = oracle.Scene(sc)
    for i in idx:
        # walk j of point i draws the counters (j, i, step, slot): the oracle
        # recomputes point i with the same streams as the full-grid launch
        o = oracle.solve(O, sc["points"][i:i + 1], sc["walks"], sc["epsilon"], sc["r_min"], sc["max_steps"],
                         seed=777, point_base=int(i))
        se = np.hypot(o["se"][0], res["se"][i])
        assert abs(res["mean"][i] - o["mean"][0]) <= 4 * se, (i, res["mean"][i], o["mean"][0], se)
