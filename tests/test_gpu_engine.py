"""Batched launches and the serving engine on the GPU.

Every walk draws Philox numbers keyed by (seed, point, walk, step), so a
solve gives the same walks whether it runs alone, in a batch or in the
engine's mix.  Between runs of one kernel only the order of the FP64
additions differs (compared to 1e-9); the batched kernel is a separately
compiled instantiation (it also serves screened solves), whose single-
precision arithmetic may round differently in the last bit (fused
multiply-adds), so against the one-solve kernels walks agree to FP32
rounding (compared to 1e-6; a different walk would differ by O(1)).
"""
FP32_WALKS = dict(rtol=1e-6, atol=1e-7)
import time

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


@pytest.fixture(scope="module")
def mix(wost):
    a = scenes.config1(n_points=48)
    b = scenes.config2(grid=20, level=3, max_steps=8192)
    c = scenes.box_sphere_scene()
    rng = np.random.default_rng(8)
    p = rng.uniform(-0.9, 0.9, (400, 3))
    c["points"] = p[np.linalg.norm(p, axis=1) > 0.5][:40].astype(np.float32)
    c["epsilon"], c["r_min"], c["max_steps"] = 1e-3, 1e-3, 4096
    S = [wost.Scene(s) for s in (a, b, c)]
    yield [a, b, c], S
    for s in S:
        s.close()


def _alone(wost, S, sc, walks, seed, first_walk=0):
    return wost.solve(S, torch.from_numpy(sc["points"]).cuda(), walks, sc["epsilon"], sc["r_min"],
                      sc["max_steps"], seed=seed, first_walk=first_walk, kernel="persistent")


def test_batch_equals_solves_alone(wost, mix):
    specs, S = mix
    walks = [64, 32, 48]
    reqs = [dict(points=torch.from_numpy(sc["points"]).cuda(), walks_per_point=w, epsilon=sc["epsilon"],
                 r_min=sc["r_min"], max_steps=sc["max_steps"], seed=10 + i)
            for i, (sc, w) in enumerate(zip(specs, walks))]
    hs = wost.wost_solve_batch([s.handle for s in S], reqs)
    try:
        for h in hs:
            wost.wost_wait(h, 300)
        got = [wost.wost_poll(h, len(sc["points"])) for h, sc in zip(hs, specs)]
    finally:
        for h in hs:
            wost.wost_solve_destroy(h)
    for i, (sc, s) in enumerate(zip(specs, S)):
        ref = _alone(wost, s, sc, walks[i], 10 + i)
        np.testing.assert_allclose(got[i][0], ref["mean"], **FP32_WALKS)
        assert got[i][3]["done"] == 1 and int(got[i][2].sum()) == len(sc["points"]) * walks[i]


def test_batch_with_a_screened_job_equals_solves_alone(wost, mix):
    """A batch holding a screened job runs the screened form of the batched
    kernel for its dimension (the Poisson-only form for the other): every
    job's result is still its result alone."""
    specs, S = mix
    walks, sig = [32, 16, 24], [0.5, 0.0, 2.0]
    reqs = [dict(points=torch.from_numpy(sc["points"]).cuda(), walks_per_point=w, epsilon=sc["epsilon"],
                 r_min=sc["r_min"], max_steps=sc["max_steps"], seed=40 + i, sigma=g)
            for i, (sc, w, g) in enumerate(zip(specs, walks, sig))]
    hs = wost.wost_solve_batch([s.handle for s in S], reqs)
    try:
        for h in hs:
            wost.wost_wait(h, 300)
        got = [wost.wost_poll(h, len(sc["points"])) for h, sc in zip(hs, specs)]
    finally:
        for h in hs:
            wost.wost_solve_destroy(h)
    for i, (sc, s) in enumerate(zip(specs, S)):
        ref = wost.solve(s, torch.from_numpy(sc["points"]).cuda(), walks[i], sc["epsilon"], sc["r_min"],
                         sc["max_steps"], seed=40 + i, kernel="persistent", sigma=sig[i])
        np.testing.assert_allclose(got[i][0], ref["mean"], **FP32_WALKS)
        assert got[i][3]["total_steps"] == ref["total_steps"]


def _run_engine(wost, S, specs, targets, seeds, caps, **kw):
    eng = wost.wost_engine_create(**kw)
    hs = []
    try:
        for s, sc, t, sd, cap in zip(S, specs, targets, seeds, caps):
            hs.append(wost.wost_engine_submit(eng, s.handle, sc["points"], t, cap, sc["epsilon"], sc["r_min"],
                                              sc["max_steps"], seed=sd))
        for h in hs:
            wost.wost_wait(h, 600)
        res = [wost.wost_poll(h, len(sc["points"])) for h, sc in zip(hs, specs)]
        stats = wost.wost_engine_get_stats(eng)
    finally:
        for h in hs:
            wost.wost_solve_destroy(h)
        wost.wost_engine_destroy(eng)
    return res, stats


def test_engine_results_same_alone_and_in_the_mix(wost, mix):
    specs, S = mix
    targets = [0.02, 0.05, 0.02]
    caps = [4096, 2048, 4096]
    alone = []
    for i in range(3):
        r, _ = _run_engine(wost, [S[i]], [specs[i]], [targets[i]], [100 + i], [caps[i]])
        alone.append(r[0])
    both, stats = _run_engine(wost, S, specs, targets, [100, 101, 102], caps, round_seconds=0.005)
    assert stats["completed"] == 3 and stats["rounds"] >= 3
    # the rounds' device count of walk steps is the requests' own, walk for walk
    assert stats["walk_steps"] == sum(int(r[3]["total_steps"]) for r in both)
    for i in range(3):
        m_a, se_a, w_a, _ = alone[i]
        m_b, se_b, w_b, _ = both[i]
        np.testing.assert_array_equal(w_a, w_b)          # same stopping point
        np.testing.assert_allclose(m_a, m_b, rtol=1e-9, atol=1e-12)
        assert np.all(se_b <= targets[i] * (1 + 1e-6)) or int(w_b.min()) >= caps[i]


def test_engine_target_and_cap(wost, mix):
    specs, S = mix
    sc = specs[0]
    res, stats = _run_engine(wost, [S[0]], [sc], [0.0], [5], [40])  # target 0: exactly the cap
    m, se, w, pr = res[0]
    assert np.all(w == 40)
    ref = _alone(wost, S[0], sc, 40, 5)
    np.testing.assert_allclose(m, ref["mean"], **FP32_WALKS)


def test_engine_device_inputs_and_early_poll(wost, mix):
    """A request whose points are device memory (copied on the engine's own
    stream at submission) gives the walks of the same request from host
    memory; a poll right after submission reports no walks rather than
    reading buffers still being set up."""
    specs, S = mix
    sc = specs[1]
    eng = wost.wost_engine_create()
    hs = []
    try:
        for pts in (sc["points"], torch.from_numpy(sc["points"]).cuda()):
            h = wost.wost_engine_submit(eng, S[1].handle, pts, 0.0, 24, sc["epsilon"], sc["r_min"],
                                        sc["max_steps"], seed=77)
            hs.append(h)
            m0, se0, w0, pr0 = wost.wost_poll(h, len(sc["points"]))
            assert int(w0.sum()) == pr0["walks_done"] and pr0["walks_done"] <= len(sc["points"]) * 24
        for h in hs:
            wost.wost_wait(h, 300)
        res = [wost.wost_poll(h, len(sc["points"])) for h in hs]
    finally:
        for h in hs:
            wost.wost_solve_destroy(h)
        wost.wost_engine_destroy(eng)
    assert np.all(res[0][2] == 24) and np.all(res[1][2] == 24)
    np.testing.assert_allclose(res[1][0], res[0][0], **FP32_WALKS)
    assert res[1][3]["total_steps"] == res[0][3]["total_steps"]


def test_engine_budget_admission_and_rejection(wost, mix):
    specs, S = mix
    sc = specs[0]
    per_request = len(sc["points"]) * (2 * 4 + 32) + 64
    eng = wost.wost_engine_create(memory_budget_bytes=int(per_request * 1.5))
    try:
        big = np.concatenate([sc["points"]] * 2)
        with pytest.raises(wost.WostError) as ei:
            wost.wost_engine_submit(eng, S[0].handle, big, 0.05, 64, sc["epsilon"], sc["r_min"], sc["max_steps"])
        assert ei.value.status == wost.ERR_BUDGET
        h1 = wost.wost_engine_submit(eng, S[0].handle, sc["points"], 0.0, 32, sc["epsilon"], sc["r_min"],
                                     sc["max_steps"], seed=1)
        h2 = wost.wost_engine_submit(eng, S[0].handle, sc["points"], 0.0, 32, sc["epsilon"], sc["r_min"],
                                     sc["max_steps"], seed=2)
        wost.wost_wait(h1, 120)
        time.sleep(0.2)
        st = wost.wost_engine_get_stats(eng)
        assert st["queued"] == 1 and st["admitted"] == 1  # h1 keeps its memory until destroyed
        with pytest.raises(wost.WostError) as ei:
            wost.wost_wait(h2, 0.2)
        assert ei.value.status == wost.ERR_TIMEOUT
        wost.wost_solve_destroy(h1)
        wost.wost_wait(h2, 120)
        assert wost.wost_engine_get_stats(eng)["rejected"] == 1
        wost.wost_solve_destroy(h2)
    finally:
        wost.wost_engine_destroy(eng)


def test_engine_cancel_and_progressive_poll(wost, mix):
    specs, S = mix
    sc = specs[1]
    eng = wost.wost_engine_create(round_seconds=0.005)
    try:
        h = wost.wost_engine_submit(eng, S[1].handle, sc["points"], 1e-6, 1 << 20, sc["epsilon"], sc["r_min"],
                                    sc["max_steps"], seed=3)
        seen = []
        for _ in range(20):
            time.sleep(0.05)
            seen.append(wost.wost_poll(h, len(sc["points"]))[3]["walks_done"])
        assert seen[-1] > 0 and seen == sorted(seen)
        wost.wost_cancel(h)
        with pytest.raises(wost.WostError) as ei:
            wost.wost_wait(h, 120)
        assert ei.value.status == wost.ERR_CANCELLED
        wost.wost_solve_destroy(h)
        assert wost.wost_engine_get_stats(eng)["cancelled"] == 1
    finally:
        wost.wost_engine_destroy(eng)


def test_engine_sheds_requests_that_wait_too_long(wost, mix):
    """Overload shedding: with memory for one request, a second one queued
    behind a long-running first is finished with BUDGET once it has waited
    max_wait_seconds for its first walks, and counted as rejected; the first
    is unaffected."""
    specs, S = mix
    sc = specs[0]
    per_request = len(sc["points"]) * (2 * 4 + 32) + 64
    eng = wost.wost_engine_create(memory_budget_bytes=int(per_request * 1.5), max_wait_seconds=0.3)
    try:
        h1 = wost.wost_engine_submit(eng, S[0].handle, sc["points"], 0.0, 1 << 16, sc["epsilon"], sc["r_min"],
                                     sc["max_steps"], seed=1)
        h2 = wost.wost_engine_submit(eng, S[0].handle, sc["points"], 0.0, 32, sc["epsilon"], sc["r_min"],
                                     sc["max_steps"], seed=2)
        t0 = time.perf_counter()
        with pytest.raises(wost.WostError) as ei:
            wost.wost_wait(h2, 60)
        assert ei.value.status == wost.ERR_BUDGET and time.perf_counter() - t0 < 30
        st = wost.wost_engine_get_stats(eng)
        assert st["rejected"] == 1 and st["admitted"] == 1
        assert wost.wost_poll(h1, len(sc["points"]))[3]["walks_done"] > 0
        wost.wost_cancel(h1)
        try:  # finished by now or cancelled
            wost.wost_wait(h1, 120)
        except wost.WostError as e:
            assert e.status == wost.ERR_CANCELLED
        wost.wost_solve_destroy(h1)
        wost.wost_solve_destroy(h2)
    finally:
        wost.wost_engine_destroy(eng)
