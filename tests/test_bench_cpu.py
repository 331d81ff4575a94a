"""Host logic of bench.py on the CPU: the clock-sample summary, the
algorithmic work model and the arithmetic of the roofline figure, and the
record of profiled DRAM traffic it draws on."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_clock_summary_uses_loaded_samples_and_collects_reasons():
    lines = [
        "0, 345, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # idle sample
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.parse_clock_samples(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 4
    assert bench.parse_clock_samples([])["sm_mhz"] is None


def _counts(**kw):
    c = {f"{q}_{k}": 0.0 for q in ("q1", "q2", "q3", "q4", "vis") for k in ("nodes", "prims")}
    c.update(kw)
    return c


@pytest.mark.parametrize("lanes,node_bytes,cone_bytes,children", [(1, 48, 32, 2), (8, 256, 128, 8)])
def test_work_model_bytes_and_flops(lanes, node_bytes, cone_bytes, children):
    info = {"lanes_per_walk": lanes, "node_bytes": node_bytes, "cone_bytes": cone_bytes}
    # 10 steps: 30 Q.1 node visits, 20 Q.2 node visits (with cones), 5 Q.3 segment tests
    b, f = bench.work_per_step(_counts(q1_nodes=30, q2_nodes=20, q3_prims=5), 10, 2, info)
    assert b == pytest.approx((30 * node_bytes + 20 * (node_bytes + cone_bytes) + 5 * 16) / 10)
    expect_f = (30 * children * bench.CHILD_FLOPS[2]["q1"] + 20 * children * bench.CHILD_FLOPS[2]["q2"]
                + 5 * bench.PRIM_FLOPS[2]["q3"]) / 10 + bench.STEP_FLOPS[2]
    assert f == pytest.approx(expect_f)


def test_roofline_fraction_traffic_and_per_launch_bytes():
    peaks = {"hbm_gbs": 6000.0}
    # 3 launches of 1e9 walk steps in 2 s at 3,000 algorithmic bytes and 2,000 flops per step
    r = bench.roofline_block("k", 3000.0, 2000.0, 3e9, 2.0, 3, peaks, "measured", 20000.0, 7000.0, 80.0, "x",
                             0.5, {})
    assert r["achieved"] == pytest.approx(3000.0 * 3e9 / 2.0 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0) and r["peak"] == 6000.0
    assert r["l2_frac"] == pytest.approx(r["achieved"] / 20000.0)
    assert r["achieved_tflops"] == pytest.approx(2000.0 * 3e9 / 2.0 / 1e12)
    assert r["fp32_frac"] == pytest.approx(r["achieved_tflops"] / 80.0)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(3000.0 * 1e9)
    assert r["traffic"] == pytest.approx(0.5 * 1e9)  # DRAM bytes per step x the steps of one launch
    assert bench.roofline_block("k", 1.0, 1.0, 1.0, 1.0, 1, peaks, "m", 1.0, 1.0, 1.0, "x", None, {})["traffic"] is None


def test_traffic_record_format_and_lookup():
    """Every record of profiles/traffic.txt names a kernel, a 16-digit source
    hash and DRAM bytes per walk step; the lookup returns a record's figure
    only for its own hash."""
    path = os.path.join(bench.ROOT, "profiles", "traffic.txt")
    recs = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert recs
    for f in recs:
        assert f[0].startswith("k_walk_") and len(f[1]) == 16 and int(f[1], 16) >= 0 and float(f[2]) >= 0
        assert bench.profiled_traffic(f[0], f[1]) == float(f[2])
    assert bench.profiled_traffic(recs[0][0], "0" * 16) is None
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
