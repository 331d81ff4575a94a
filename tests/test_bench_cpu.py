"""Host logic of bench.py on the CPU: the clock-sample summary and the
algorithmic work model behind the roofline figure."""
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
