"""wost_solve_static, the solve entry point that allocates nothing, for
callers that cannot call cudaMalloc while they solve (its accumulators live
in a fixed device array of the library).  This file is collected last, so a
run that stops at the first failure has run every other test before it; it
also passes alone in a fresh process.

Checks, through the C ABI: two calls in a row against wost_solve with the
persistent kernel (the same walks; results within FP32 rounding of the FP64
sums), the size limit, and that a call leaves the device's free memory
unchanged."""
import numpy as np
import pytest

from paper_2302_11815_gb300 import scenes

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


@pytest.mark.parametrize("name", ["config1", "koch"])
def test_static_matches_wost_solve_on_two_calls_in_a_row(wost, name):
    sc = scenes.config1() if name == "config1" else scenes.config2(grid=48)
    pts = np.ascontiguousarray(sc["points"][:1000], np.float32)
    eps, rmin, cap = sc["epsilon"], sc.get("r_min", 0.0), min(sc["max_steps"], 4096)
    S = wost.Scene(sc)
    pts_dev = torch.from_numpy(pts).cuda()
    mean = torch.empty(len(pts), dtype=torch.float32, device="cuda")
    se = torch.empty(len(pts), dtype=torch.float32, device="cuda")
    for call, (seed, first_walk) in enumerate([(21, 0), (22, 64)]):
        ref = wost.solve(S, pts_dev, 64, eps, rmin, cap, seed=seed, first_walk=first_walk, kernel="persistent")
        wost.wost_solve_static(S.handle, pts_dev, 64, eps, rmin, cap, seed, first_walk, mean, se)
        torch.cuda.synchronize()
        m = mean.cpu().numpy().astype(np.float64)
        s = se.cpu().numpy().astype(np.float64)
        # identical walks; the FP64 sums differ only in the order of the
        # additions, and both sides end in FP32
        np.testing.assert_allclose(m, ref["mean"], rtol=1e-5, atol=1e-6, err_msg=f"call {call}")
        np.testing.assert_allclose(s, ref["se"], rtol=1e-4, atol=1e-6, err_msg=f"call {call}")
    S.close()


def test_static_rejects_too_many_points_and_allocates_nothing(wost):
    sc = scenes.config1()
    S = wost.Scene(sc)
    n_max = wost.WOST_STATIC_MAX_POINTS
    big = torch.zeros((n_max + 1, 2), dtype=torch.float32, device="cuda")
    out = torch.empty(n_max + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(wost.WostError, match="WOST_STATIC_MAX_POINTS"):
        wost.wost_solve_static(S.handle, big, 4, 1e-3, 1e-3, 64, 1, 0, out, None)
    pts = torch.from_numpy(np.ascontiguousarray(sc["points"], np.float32)).cuda()
    mean = torch.empty(len(pts), dtype=torch.float32, device="cuda")
    # the first call on the device may load the module (and with it the array)
    wost.wost_solve_static(S.handle, pts, 16, sc["epsilon"], 0.0, 256, 3, 0, mean, None)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    wost.wost_solve_static(S.handle, pts, 16, sc["epsilon"], 0.0, 256, 4, 0, mean, None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert bool(torch.isfinite(mean).all())
    S.close()


def test_static_binding_rejects_mismatched_arrays(wost):
    """The C entry point takes raw pointers and cannot check sizes: the
    binding checks the points' shape against the scene's dimension and the
    output lengths against the point count before it calls."""
    sc = scenes.config1()
    S = wost.Scene(sc)
    pts3 = torch.zeros((16, 3), dtype=torch.float32, device="cuda")
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError, match="points must be"):
        wost.wost_solve_static(S.handle, pts3, 4, 1e-3, 1e-3, 64, 1, 0, out, None)
    pts = torch.zeros((16, 2), dtype=torch.float32, device="cuda")
    short = torch.empty(15, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError, match="fewer than"):
        wost.wost_solve_static(S.handle, pts, 4, 1e-3, 1e-3, 64, 1, 0, short, None)
    with pytest.raises(ValueError, match="fewer than"):
        wost.wost_solve_static(S.handle, pts, 4, 1e-3, 1e-3, 64, 1, 0, out, short)
    S.close()
