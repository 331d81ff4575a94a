"""The multi-GPU form of the benchmark is replicas: every rank solves its own
copy of the workload with its own seed and only the timings and step counts
are combined (max of the times, sum of the steps).  These tests run that
host logic as two gloo ranks on the CPU: the environment handling of
bench._dist_init, the barrier, the max/sum reductions, and that the ranks'
walks are independent (per-rank seeds) while each rank's result does not
depend on the other rank (it equals a single-process solve with its seed)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import bench
    import oracle
    from paper_2302_11815_gb300 import scenes

    r, w, local = bench._dist_init(world)
    assert (r, w, local) == (rank, world, rank)
    import torch.distributed as dist

    assert dist.get_backend() == "gloo"
    # each replica solves the same points with its own seed (as bench.py does)
    sc = scenes.config1(n_points=8)
    res = oracle.solve(oracle.Scene(sc), sc["points"], 64, sc["epsilon"], sc["r_min"], sc["max_steps"],
                       seed=1000 * (rank + 1))
    steps = float(res["steps"].sum())
    bench._barrier(world)
    t_max = bench._max_over_ranks(1.0 + rank, world)
    steps_all = bench._sum_over_ranks(steps, world)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), mean=res["mean"], steps=steps, t_max=t_max,
             steps_all=steps_all)
    dist.destroy_process_group()


def test_two_gloo_replicas_reduce_times_and_steps(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    a = np.load(tmp_path / "rank0.npz")
    b = np.load(tmp_path / "rank1.npz")
    # max over ranks of the time, sum over ranks of the steps, same on both
    assert float(a["t_max"]) == float(b["t_max"]) == 2.0
    assert float(a["steps_all"]) == float(b["steps_all"]) == float(a["steps"]) + float(b["steps"])
    # independent walks: different seeds give different estimates
    assert not np.allclose(a["mean"], b["mean"])
    # and rank 0's estimates are those of a single-process solve with its seed
    import oracle
    from paper_2302_11815_gb300 import scenes

    sc = scenes.config1(n_points=8)
    one = oracle.solve(oracle.Scene(sc), sc["points"], 64, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=1000)
    np.testing.assert_array_equal(a["mean"], one["mean"])
