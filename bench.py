"""Benchmark: walk-on-stars walk-steps/s on one or more GPUs.

Headline workload: 2D Poisson on a level-5 Koch snowflake (3072 segments,
half Dirichlet, half Neumann by arc length) with a 1024-segment random-walk
hole (all Neumann); exact u = sin 2x cos 3y, f = 13 u; the interior cell
centres of a 512 x 512 raster (141,021 points), 256 walks per point,
eps = r_min = 1e-4.  The whole workload is about 1.1e11 walk steps (walks
average ~3,000 steps: most of the boundary reflects; the longest reach the
65,536-step cap).  It runs as one resumable solve over the whole grid, and a
step is one launch of it: every resident lane runs up to --iters walk steps,
drawing new walks as its walks end and carrying unfinished ones to the next
launch, so no launch waits for the longest walks.  The e2e figure is a
complete solve of every 16th grid point from host memory, the longest walks
included.

After the timed headline (N = 1 only) the same line carries the other
workloads, measured outside the timed region: the 64-segment flower (plain
and persistent launches), the 3D cube around a noisy 200k-triangle torus
(resumable launches, its own work model and roofline), the batched
multi-scene workload (one batched launch against one launch per scene, same
walks) and the serving workload (a Poisson request stream into the engine:
p50/p99 latency, offered against served load); plus the walks per point and
points/s at which the headline workload reaches 1% relative RMS error.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are replicas: every rank solves
the whole workload with its own seed (independent walks), no collective is on
the data path; the timing is the max over ranks.  --impl reference times the
FP64 brute-force CPU oracle (the only reference this project has) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walk_steps_per_s"
UNIT = "walk-steps/s"
WORKLOAD = "koch5_hole_poisson_2d_grid512_w256"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2: written between timed solves


_T0 = time.perf_counter()


def _log(msg):
    """Progress on stderr (stdout carries only the JSON line)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def _config_block(sc, extra=None):
    cfg = {"workload": WORKLOAD, "n_points": int(len(sc["points"])), "walks_per_point": sc["walks"],
           "prims": int(len(sc["prims"])), "neumann_prims": int(sc["flags"].sum()), "epsilon": sc["epsilon"],
           "r_min": sc["r_min"], "max_steps": sc["max_steps"], "precision": "fp32 walks, fp64 accumulators",
           "l2": "flushed between timed steps (512 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def _dist_init(n_gpus):
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        out = os.environ.get("WOST_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, f"wost_clocks_gpu{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            return parse_clock_samples(fh)


def parse_clock_samples(lines):
    """Summary of nvidia-smi samples in ClockSampler.FIELDS order: median SM
    clock over the loaded samples (above half the highest), the highest max
    clock, and every throttle reason seen Active."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    load = [s for s in sm if s > 0.5 * max(sm)] or sm
    return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# algorithmic cost of one node visit / primitive test, per query: bytes read
# from the memory hierarchy and FP32 operations (an FMA counted as 2).  A node
# visit reads one node record (plus its child cones in Q.2) of the layout the
# kernels traverse, as reported in the scene info; its flops are per child
# box test (2 children in a binary node, 8 in a wide one).
PRIM_BYTES = {2: {"q1": 16, "q2": 32, "q3": 16, "q4": 16, "vis": 16},
              3: {"q1": 48, "q2": 48, "q3": 48, "q4": 48, "vis": 48}}
CHILD_FLOPS = {2: {"q1": 12, "q2": 35, "q3": 17, "q4": 22, "vis": 17},
               3: {"q1": 18, "q2": 45, "q3": 25, "q4": 30, "vis": 25}}
PRIM_FLOPS = {2: {"q1": 16, "q2": 12, "q3": 16, "q4": 22, "vis": 16},
              3: {"q1": 45, "q2": 30, "q3": 34, "q4": 50, "vis": 34}}
STEP_FLOPS = {2: 60, 3: 80}  # per-step bookkeeping: radius, direction, Green's function, source


def work_per_step(counts, steps, dim, info):
    children = 2 if info["lanes_per_walk"] == 1 else 8
    b = f = 0.0
    for q in ("q1", "q2", "q3", "q4", "vis"):
        nb = info["node_bytes"] + (info["cone_bytes"] if q == "q2" else 0)
        b += counts[f"{q}_nodes"] * nb + counts[f"{q}_prims"] * PRIM_BYTES[dim][q]
        f += counts[f"{q}_nodes"] * children * CHILD_FLOPS[dim][q] + counts[f"{q}_prims"] * PRIM_FLOPS[dim][q]
    return b / steps, f / steps + STEP_FLOPS[dim]


def measure_read_gbs(torch, wost, stream, nbytes, passes, reps=5):
    """Read bandwidth of the level a buffer of `nbytes` lives in, measured with
    the library's read probe (16-byte loads that bypass L1, resident grid):
    best of `reps` launches of `passes` sweeps, the first sweep of each
    included, CUDA events on the launching stream."""
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    best = 0.0
    with torch.cuda.stream(stream):
        wost.wost_read_probe(buf, passes, sink, stream)
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            wost.wost_read_probe(buf, passes, sink, stream)
            b.record(stream)
            b.synchronize()
            best = max(best, passes * nbytes / (a.elapsed_time(b) * 1e-3) / 1e9)
    del buf
    return best


KERNEL_SOURCES = ("wost_device.cuh", "wost_walk.cuh", "wost_kernels.cu", "wost_internal.h")


def kernel_source_hash():
    """sha256 (first 16 hex digits) of the sources the walk kernels compile
    from: a profile taken of other sources does not describe this build."""
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2302_11815_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, src_hash):
    """DRAM bytes per walk step of `kernel` from the ncu capture recorded in
    profiles/traffic.txt (lines: kernel, source hash, dram bytes per walk
    step, the capture), or None if none was taken of these sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            f = line.split()
            if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[1] == src_hash:
                return float(f[2])
    return None


def roofline_block(kernel, bytes_step, flops_step, steps, seconds, launches, peaks, peak_src, l2_gbs, hbm_probe_gbs,
                   fp32, fp32_src, traffic_per_step, counts_per_step):
    """Roofline of one kernel: the algorithmic bytes and flops per walk step
    times the steps of the timed launches over their device time, against
    the measured HBM copy bandwidth (the contract's memory roof), the L2 read
    bandwidth measured here (the level the scenes live in, the stricter roof)
    and the FP32 peak."""
    achieved_b = bytes_step * steps / seconds / 1e9
    achieved_f = flops_step * steps / seconds / 1e12
    return {"bound": "hbm", "achieved": achieved_b, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved_b / peaks["hbm_gbs"],
            "traffic": None if traffic_per_step is None else traffic_per_step * steps / launches,
            "traffic_src": "DRAM bytes per launch: ncu dram__bytes_read + dram__bytes_write per walk step of this"
                           " source build (profiles/traffic.txt) x the walk steps of an average timed launch",
            "algorithmic_bytes_per_launch": bytes_step * steps / launches,
            "kernel": kernel, "unit_of_work": "walk step", "bytes_per_step": bytes_step, "flops_per_step": flops_step,
            "peak_src": peak_src, "l2_peak_gbs": l2_gbs, "l2_frac": achieved_b / l2_gbs,
            "l2_peak_src": "measured in this run: read probe over a 48 MiB buffer (L2-resident)",
            "hbm_probe_gbs": hbm_probe_gbs, "fp32_frac": achieved_f / fp32, "fp32_peak_tflops": fp32,
            "fp32_peak_src": fp32_src, "achieved_tflops": achieved_f, "seconds": seconds, "steps": steps,
            "counts_per_step": counts_per_step}


def cpu_baseline(sc, walks=48, seed=1):
    """The FP64 oracle as it stands on all host cores (one thread per point),
    on a bounded sample: `cores` random grid points x `walks` of their walks
    (about 10-30 s of CPU work on the workload)."""
    import oracle
    O = oracle.Scene(sc)
    rng = np.random.default_rng(seed)
    cores = os.cpu_count() or 1
    idx = rng.choice(len(sc["points"]), cores, replace=False)
    t0 = time.perf_counter()
    r = oracle.solve(O, sc["points"][idx], walks, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=seed,
                     threads=cores)
    dt = time.perf_counter() - t0
    steps = int(r["steps"].sum())
    return {"value": steps / dt, "unit": UNIT, "cores": int(r["threads"]), "kind": "oracle",
            "sample": f"{cores} random grid points x {walks} of their {sc['walks']} walks ({steps} steps, {dt:.1f} s)",
            "points_per_s": cores * walks / sc["walks"] / dt}


def run_reference(args):
    rank, world, local = _dist_init(args.gpus)
    if rank != 0:
        return 0
    from paper_2302_11815_gb300 import scenes
    sc = scenes.config2()
    for _ in range(args.warmup):
        cpu_baseline(sc, walks=2, seed=99)
    vals = []
    t0 = time.perf_counter()
    for i in range(args.steps):
        vals.append(cpu_baseline(sc, walks=args.cpu_walks, seed=i + 1))
    elapsed = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config_block(sc, {"sample": "bounded random subsample per step",
                                         "precision": "fp64 oracle (brute-force queries)", "l2": "n/a (CPU)"}),
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "sample": vals[0]["sample"], "value": v,
                             "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _resumable_launches(wost, torch, S, pts_dev, sc, stream, flush, iters, warmup, steps, seed, block=0):
    """A resumable solve of every point x the workload's walks; `warmup`
    untimed launches, then `steps` timed launches of `iters` walk steps per
    lane, L2 flushed before each (outside the events).  Returns the solve
    handle (open), the walk steps of the timed launches, their device
    seconds and the per-launch milliseconds."""
    job = wost.wost_solve(S.handle, pts_dev, sc["walks"], sc["epsilon"], sc["r_min"], sc["max_steps"], seed=seed,
                          kernel="resumable", block_size=block, stream=stream)
    n = pts_dev.shape[0]

    def steps_run():
        return wost.wost_poll(job, n)[3]["steps_run"]

    for _ in range(warmup):
        wost.wost_solve_advance(job, iters, stream)
        stream.synchronize()
    total = 0
    dev_ms = []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))  # evict the scene and the walk state from L2
        s0 = steps_run()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        wost.wost_solve_advance(job, iters, stream)
        ev1.record(stream)
        ev1.synchronize()
        dev_ms.append(ev0.elapsed_time(ev1))
        total += steps_run() - s0
    return job, total, sum(dev_ms) * 1e-3, dev_ms


def _rel_rms(mean, u):
    return float(np.sqrt(np.sum((np.asarray(mean) - u) ** 2) / np.sum(u**2)))


def error_condition(steps_per_s, steps_per_walk, walks, rel_rms, target=0.01):
    """Walks per point for `target` relative RMS error and points/s there,
    from an error measured at `walks` walks: the error of a mean of
    independent walks falls as walks^-1/2 (the epsilon-shell bias, below
    1e-3 relative here, is neglected)."""
    need = walks * (rel_rms / target) ** 2
    return {"target_rel_rms": target, "measured_rel_rms": rel_rms, "at_walks_per_point": walks,
            "walks_per_point_needed": need, "points_per_s_at_target": steps_per_s / (need * steps_per_walk),
            "model": "rel RMS ~ walks^-1/2 from the measured point"}


def sub_flower(wost, torch, stream):
    """Workload 1: the 64-segment flower, 256 points x 512 walks, one launch
    of the plain and of the persistent kernel (device time), RMS against
    the exact solution."""
    from paper_2302_11815_gb300 import scenes

    sc = scenes.config1()
    S = wost.Scene(sc)
    pts = torch.from_numpy(sc["points"]).cuda()
    u = scenes.exact_u("exp_cos", (), sc["points"])
    out = {"workload": "flower64_laplace_2d_256pts_w512", "points": len(pts), "walks_per_point": sc["walks"]}
    for kernel in ("plain", "persistent"):
        best = None
        for rep in range(3):
            r = wost.solve(S, pts, sc["walks"], sc["epsilon"], sc["r_min"], sc["max_steps"], seed=17 + rep,
                           kernel=kernel, stream=stream)
            if best is None or r["elapsed_seconds"] < best["elapsed_seconds"]:
                best = r
        out[kernel] = {"seconds": best["elapsed_seconds"], "walk_steps_per_s": best["total_steps"] / best["elapsed_seconds"],
                       "points_per_s": len(pts) / best["elapsed_seconds"], "rel_rms_vs_exact": _rel_rms(best["mean"], u),
                       "steps": int(best["total_steps"]), "capped_walks": int(best["capped_walks"])}
    S.close()
    return out


def sub_cube_torus(wost, torch, args, stream, flush, peaks, peak_src, l2_gbs, hbm_gbs, fp32, fp32_src):
    """Workload 3: cube around a noisy 200k-triangle torus, ~850k slice points
    x 128 walks.  Timed like the headline (resumable launches of the whole
    job), with its own work model and roofline; the RMS error against the
    exact solution from a complete solve of a seeded subsample."""
    from paper_2302_11815_gb300 import scenes

    sc = scenes.config3()
    S = wost.Scene(sc)
    info = S.info()
    pts = np.ascontiguousarray(sc["points"], np.float32)
    rng = np.random.default_rng(3)
    sub = pts[rng.choice(len(pts), 4096, replace=False)]
    r = wost.solve(S, torch.from_numpy(sub[:512]).cuda(), 32, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=3,
                   kernel="counting")
    b_step, f_step = work_per_step(r["counts"], r["total_steps"], 3, dict(info, lanes_per_walk=1, node_bytes=64,
                                                                         cone_bytes=32))
    pts_dev = torch.from_numpy(pts).cuda()
    job, steps, secs, ms = _resumable_launches(wost, torch, S, pts_dev, sc, stream, flush, args.iters3, 2,
                                               args.steps3, seed=31)
    wost.wost_solve_destroy(job)
    full = wost.solve(S, torch.from_numpy(sub).cuda(), sc["walks"], sc["epsilon"], sc["r_min"], sc["max_steps"],
                      seed=33, kernel="resumable", stream=stream)
    u = scenes.exact_u("quad3", (), sub)
    spw = full["total_steps"] / max(1, int(full["walks"].sum()))
    rate = steps / secs
    rel = _rel_rms(full["mean"], u)
    roof = roofline_block("k_walk_resume<3>", b_step, f_step, steps, secs, args.steps3, peaks, peak_src, l2_gbs,
                          hbm_gbs, fp32, fp32_src, profiled_traffic("k_walk_resume<3>", kernel_source_hash()),
                          {k: v / r["total_steps"] for k, v in r["counts"].items()})
    out = {"workload": "cube_torus200k_laplace_3d_slices578_w128", "points": len(pts), "walks_per_point": sc["walks"],
           "prims": int(len(sc["prims"])), "walk_steps_per_s": rate, "launches": args.steps3,
           "iters_per_launch": args.iters3, "launch_ms": ms, "mean_steps_per_walk": spw,
           "points_per_s": rate / (spw * sc["walks"]),
           "rel_rms_vs_exact": rel, "rms_sample": f"{len(sub)} seeded points x {sc['walks']} walks, complete solve",
           "capped_walks": int(full["capped_walks"]), "roofline": roof,
           "error_condition": error_condition(rate, spw, sc["walks"], rel)}
    S.close()
    return out


def sub_keyhole(wost, torch, stream):
    """The Neumann-dominated stress scene (two rooms, a corridor, a small
    Dirichlet window: hundreds of steps per walk): one complete resumable
    solve of 64 points x 4096 walks, device time and error against u = x."""
    from paper_2302_11815_gb300 import scenes

    sc = scenes.keyhole_scene()
    S = wost.Scene(sc)
    pts = torch.from_numpy(sc["points"]).cuda()
    r = wost.solve(S, pts, 4096, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=19, kernel="resumable",
                   stream=stream)
    S.close()
    u = sc["points"][:, 0].astype(np.float64)
    spw = r["total_steps"] / max(1, int(r["walks"].sum()))
    return {"workload": "keyhole_neumann_2d_64pts_w4096", "prims": int(len(sc["prims"])),
            "dirichlet_prims": int((sc["flags"] == 0).sum()), "seconds": r["elapsed_seconds"],
            "walk_steps_per_s": r["total_steps"] / r["elapsed_seconds"], "mean_steps_per_walk": spw,
            "rel_rms_vs_exact": _rel_rms(r["mean"], u), "capped_walks": int(r["capped_walks"])}


def sub_batch(wost, torch, args):
    """Workload 4: many scenes in one batched persistent launch per dimension
    against one launch per scene (persistent and plain kernels).  The three
    forms run the same walks (same seeds), so their RMS errors are equal by
    construction (checked: the largest relative difference of the means)."""
    from paper_2302_11815_gb300 import scenes

    t0 = time.perf_counter()
    specs = scenes.config4(n_scenes=args.batch_scenes, points=(1, args.batch_max_points),
                           walks=(16, args.batch_max_walks), max_scene=args.batch_max_prims)
    gen_s = time.perf_counter() - t0
    S = [wost.Scene(s) for s in specs]
    pts = [torch.from_numpy(s["points"]).cuda() for s in specs]
    reqs = [dict(points=p, walks_per_point=s["walks"], epsilon=s["epsilon"], r_min=s["r_min"],
                 max_steps=s["max_steps"], seed=s["seed"]) for p, s in zip(pts, specs)]
    stream = torch.cuda.Stream()

    def batched():
        hs = wost.wost_solve_batch([s.handle for s in S], reqs, stream=stream)
        for h in hs:
            wost.wost_wait(h)
        out = [wost.wost_poll(h, len(s["points"])) for h, s in zip(hs, specs)]
        for h in hs:
            wost.wost_solve_destroy(h)
        return out

    def per_scene(kernel):
        out = []
        for s, sc, p in zip(S, specs, pts):
            h = wost.wost_solve(s.handle, p, sc["walks"], sc["epsilon"], sc["r_min"], sc["max_steps"],
                                seed=sc["seed"], kernel=kernel, stream=stream)
            wost.wost_wait(h)
            out.append(wost.wost_poll(h, len(sc["points"])))
            wost.wost_solve_destroy(h)
        return out

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = fn()
        b.record(stream)
        b.synchronize()
        return res, a.elapsed_time(b) * 1e-3

    rb, tb = timed(batched)
    _log(f"batched: {tb:.1f} s")
    rp, tp = timed(lambda: per_scene("persistent"))
    _log(f"one persistent launch per scene: {tp:.1f} s")
    rq, tq = timed(lambda: per_scene("plain"))
    _log(f"one plain launch per scene: {tq:.1f} s")
    steps = sum(r[3]["total_steps"] for r in rb)
    walks = sum(r[3]["walks_done"] for r in rb)
    maxdiff = max(float(np.max(np.abs(a[0] - b[0]) / (np.abs(b[0]) + 1e-9))) for a, b in zip(rb, rq))
    err2 = ref2 = 0.0
    for r, sc in zip(rb, specs):
        u = scenes.exact_u(*sc["exact"], sc["points"])
        err2 += float(np.sum((r[0] - u) ** 2))
        ref2 += float(np.sum(u**2))
    # roofline of the batched launches: each scene's algorithmic bytes per
    # walk step from the counting kernel on 2 of its walks per point (the
    # binary-tree records: 48-byte nodes in 2D, 64 in 3D, 32-byte cones)
    # times the walk steps the scene ran in the batch, over the batch time
    b_scene = []
    for s, sc, p in zip(S, specs, pts):
        rc = wost.solve(s, p, min(2, sc["walks"]), sc["epsilon"], sc["r_min"], sc["max_steps"], seed=sc["seed"],
                        kernel="counting", stream=stream)
        b_scene.append(work_per_step(rc["counts"], rc["total_steps"], sc["dim"],
                                     dict(s.info(), lanes_per_walk=1, node_bytes=48 if sc["dim"] == 2 else 64,
                                          cone_bytes=32))[0] if rc["total_steps"] > 0 else 0.0)
    peaks, peak_src = _measured_peaks()

    def roofline(res, secs):
        alg = sum(b * r[3]["total_steps"] for b, r in zip(b_scene, res))
        n = sum(r[3]["total_steps"] for r in res)
        return {"bound": "hbm", "achieved": alg / secs / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": alg / secs / 1e9 / peaks["hbm_gbs"], "bytes_per_step": alg / max(n, 1), "peak_src": peak_src,
                "kernel": "k_walk_batch<2/3, Poisson> (2D and 3D launches, concurrent)",
                "model": "per-scene counting-kernel bytes per walk step x the scene's walk steps in the batch"}

    roof = roofline(rb, tb)
    _log(f"batched roofline: {roof['achieved']:.0f} GB/s, {roof['frac']:.3f} of HBM")
    # the same scenes and points with 8x the walks: ~24 walks per resident
    # lane, so the launch is no longer one wave as long as its longest walks
    reqs = [dict(r, walks_per_point=8 * r["walks_per_point"]) for r in reqs]
    r8, t8 = timed(batched)
    steps8 = sum(r[3]["total_steps"] for r in r8)
    roof8 = roofline(r8, t8)
    _log(f"batched, 8x walks: {t8:.1f} s, {steps8 / t8:.3e} steps/s, {roof8['frac']:.3f} of HBM")
    for s in S:
        s.close()
    return {"workload": f"batched_{len(specs)}_scenes", "n_scenes": len(specs),
            "scenes_2d": sum(1 for s in specs if s["dim"] == 2), "total_walks": int(walks), "total_steps": int(steps),
            "total_points": int(sum(len(s["points"]) for s in specs)),
            "total_prims": int(sum(len(s["prims"]) for s in specs)),
            "batched": {"seconds": tb, "walk_steps_per_s": steps / tb, "launches": len({s["dim"] for s in specs}),
                        "roofline": roof},
            "batched_8x_walks": {"seconds": t8, "total_steps": int(steps8), "walk_steps_per_s": steps8 / t8,
                                 "walks_per_point": [128, 8 * args.batch_max_walks], "roofline": roof8},
            "per_scene_persistent": {"seconds": tp, "walk_steps_per_s": steps / tp, "launches": len(specs)},
            "per_scene_plain": {"seconds": tq, "walk_steps_per_s": steps / tq, "launches": len(specs)},
            "speedup_vs_plain": tq / tb, "speedup_vs_per_scene_persistent": tp / tb,
            "rel_rms_error_all_forms": float(np.sqrt(err2 / ref2)), "max_rel_diff_batched_vs_plain": maxdiff,
            "generation_seconds": gen_s,
            "sizes": {"points": [1, args.batch_max_points], "walks": [16, args.batch_max_walks],
                      "prims": [1e3, args.batch_max_prims]},
            "note": "same walks in all three forms (keyed random streams), so equal RMS error by construction"}


_SERVE_SCENES = {}


def sub_serve_knee(wost, torch, args):
    """The serving workload at a rate the GPU keeps up with (near the knee
    of served against offered load) and with a smaller per-request walk
    cap, so that completed requests give latency percentiles."""
    import copy

    a = copy.copy(args)
    a.serve_rate, a.serve_seconds = args.knee_rate, args.knee_seconds
    a.serve_walk_cap, a.serve_drain = args.knee_walk_cap, args.knee_drain
    out = sub_serve(wost, torch, a)
    out["workload"] = "serve_8_scenes_3d_knee"
    return out


def sub_serve(wost, torch, args):
    """Workload 5: 8 resident 3D scenes (cube + noisy torus, ~5M triangles
    together), a Poisson stream of requests into the serving engine
    (continuous batching): p50/p99 latency of the completed requests, offered
    against served load, rejections (memory budget, wait limit)."""
    import threading

    from paper_2302_11815_gb300 import scenes

    t0 = time.perf_counter()
    key = (args.serve_total_prims, args.serve_max_points)
    if key not in _SERVE_SCENES:  # resident scenes and point pools, shared by both serving runs
        specs = scenes.config5_scenes(total=args.serve_total_prims)
        rng = np.random.default_rng(7)
        _SERVE_SCENES[key] = (specs, [wost.Scene(s) for s in specs],
                              [scenes.plane_points(rng, int(args.serve_max_points), s["tube"]) for s in specs])
    specs, S, pools = _SERVE_SCENES[key]
    reqs = scenes.config5_requests(duration_s=args.serve_seconds, rate=args.serve_rate,
                                   points=(1e3, args.serve_max_points))
    setup_s = time.perf_counter() - t0
    eng = wost.wost_engine_create(round_seconds=args.round_seconds, max_walks_per_point=args.serve_walk_cap,
                                  max_wait_seconds=args.serve_max_wait)
    lock = threading.Lock()
    live, done = [], []
    stop = threading.Event()

    def collector():
        while not stop.is_set() or live:
            with lock:
                cur = list(live)
            for item in cur:
                h, rq, t_sub = item
                st = wost.wost_wait_status(h, 0.0)
                if st == wost.ERR_TIMEOUT:  # not finished yet
                    continue
                status = "ok" if st == 0 else wost.STATUS_NAMES[st]  # BUDGET: shed; CANCELLED
                m, se, wd, pr = wost.wost_poll(h, rq["n_points"])
                wost.wost_solve_destroy(h)
                with lock:
                    live.remove(item)
                    done.append({"latency": pr["elapsed_seconds"], "status": status, "n": rq["n_points"],
                                 "walks": int(wd.min()), "se_max": float(se.max()), "target": rq["target_se"],
                                 "steps": pr["total_steps"]})
            time.sleep(0.01)

    # the submitting thread must not wait long for the interpreter lock
    # while the collector sweeps thousands of live requests
    switch = sys.getswitchinterval()
    sys.setswitchinterval(5e-4)
    th = threading.Thread(target=collector, daemon=True)
    th.start()
    start = time.perf_counter()
    offered = 0
    for rq in reqs:
        wait = rq["t"] - (time.perf_counter() - start)
        if wait > 0:
            time.sleep(wait)
        pts = pools[rq["scene"]][: rq["n_points"]]
        sc = specs[rq["scene"]]
        h = wost.wost_engine_submit(eng, S[rq["scene"]].handle, pts, rq["target_se"], 0, sc["epsilon"],
                                    sc["r_min"], sc["max_steps"], seed=rq["seed"])
        offered += 1
        with lock:
            live.append((h, rq, time.perf_counter()))
    window = time.perf_counter() - start
    _log(f"serve: {offered} requests offered in {window:.1f} s, {len(done)} finished")
    drain_deadline = time.perf_counter() + args.serve_drain
    while time.perf_counter() < drain_deadline:
        with lock:
            if not live:
                break
        time.sleep(0.05)
    with lock:
        for h, rq, _ in live:
            wost.wost_cancel(h)
        _log(f"serve: drained, {len(done)} finished, {len(live)} cancelled")
    stop.set()
    th.join(timeout=120)
    sys.setswitchinterval(switch)
    _log("serve: collector joined")
    stats = wost.wost_engine_get_stats(eng)
    wost.wost_engine_destroy(eng)
    total = time.perf_counter() - start
    ok = [d for d in done if d["status"] == "ok"]
    lat = np.array([d["latency"] for d in ok]) if ok else np.array([np.nan])
    return {"workload": "serve_8_scenes_3d", "metric": "p99_latency_s",
            "p50_latency_s": float(np.nanpercentile(lat, 50)) if ok else None,
            "p99_latency_s": float(np.nanpercentile(lat, 99)) if ok else None,
            "offered_requests": offered, "offered_rate_per_s": offered / max(window, 1e-9),
            "completed": len(ok), "served_rate_per_s": len(ok) / total,
            "rejected_wait_limit": sum(1 for d in done if d["status"] == "BUDGET"),
            "cancelled_at_end": sum(1 for d in done if d["status"] == "CANCELLED"),
            "met_target": sum(1 for d in ok if d["se_max"] <= d["target"] * (1 + 1e-6)),
            "reached_walk_cap": int(stats["capped"]),
            "served_points_per_s": sum(d["n"] for d in ok) / total,
            "served_walk_steps_per_s": sum(d["steps"] for d in ok) / total,
            "engine_walk_steps_per_s": stats["walk_steps"] / total,
            "engine": stats, "window_s": window, "total_s": total, "setup_s": setup_s,
            "scene_prims": [int(len(s["prims"])) for s in specs],
            "config": {"rate_per_s": args.serve_rate, "seconds": args.serve_seconds,
                       "points": [1e3, args.serve_max_points], "walk_cap": args.serve_walk_cap,
                       "max_wait_s": args.serve_max_wait, "drain_s": args.serve_drain,
                       "targets": "SE 1e-2 or 1e-3, p = 1/2"}}


def run_ours(args):
    import torch

    rank, world, local = _dist_init(args.gpus)
    torch.cuda.set_device(local)
    from paper_2302_11815_gb300 import scenes, wost

    wost.load()  # fails loudly when the CUDA library is missing
    sc = scenes.config2()
    grid_pts = np.ascontiguousarray(sc["points"], np.float32)
    walks = sc["walks"]
    S = wost.Scene(sc, device=local)
    _log(f"scene built: {S.info()['n_dirichlet']} D + {S.info()['n_neumann']} N prims, {len(grid_pts)} grid points")
    tune = None
    if not args.block:
        # the library's autotuner picks the layout (lanes per walk) and block
        # size on a sample of the grid at the workload's walks per point
        # (~8,200 points x 256 walks: ~13 walks per resident lane, so every
        # lane stays busy through the timed launches); the timed launches
        # use its choice
        sample = torch.from_numpy(grid_pts[:: max(1, len(grid_pts) // 8192)].copy()).cuda()
        tune = wost.wost_scene_autotune(S.handle, sample, walks, sc["epsilon"], sc["r_min"], sc["max_steps"])
        _log(f"autotune: {tune['lanes_per_walk']} lane(s) per walk, block {tune['block_size']}")
    info = S.info()
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    seed0 = 1000 * (rank + 1)

    # work counts per step from the counting kernel on a subsample (untimed)
    sub = torch.from_numpy(grid_pts[:: args.count_stride * 64].copy()).cuda()
    r = wost.solve(S, sub, walks, sc["epsilon"], sc["r_min"], sc["max_steps"], seed=seed0, kernel="counting",
                   timeout=600.0)
    # the counting kernel traverses the binary trees one lane per walk: its
    # visit counts go with that layout's record sizes
    model_info = dict(info, lanes_per_walk=1, node_bytes=48, cone_bytes=32)
    bytes_step, flops_step = work_per_step(r["counts"], r["total_steps"], 2, model_info)
    _log(f"work model: {r['total_steps']} steps counted, {bytes_step:.0f} B and {flops_step:.0f} flop per step")

    # The job: every grid point x 256 walks (36 million walks, ~1.1e11 walk
    # steps), device-resident, run as a resumable solve.  A bench step is
    # one launch of it: every resident lane runs up to `iters` walk steps,
    # drawing new walks as its walks end and carrying unfinished ones over.
    pts_dev = torch.from_numpy(grid_pts).cuda()
    n_all = len(grid_pts)
    clocks = ClockSampler(local)
    clocks.start()
    _barrier(world)
    torch.cuda.synchronize()
    job, total_steps, dev_s, per_launch_ms = _resumable_launches(wost, torch, S, pts_dev, sc, stream, flush,
                                                                 args.iters, args.warmup, args.steps, seed0,
                                                                 block=args.block)
    torch.cuda.synchronize()
    _barrier(world)
    clk = clocks.stop()
    _, _, wd, pr = wost.wost_poll(job, n_all)
    wost.wost_solve_destroy(job)

    t_max = _max_over_ranks(dev_s, world, "cuda")
    steps_all = _sum_over_ranks(float(total_steps), world, "cuda")
    value = steps_all / t_max
    _log(f"timed {args.steps} launches: {value:.3e} steps/s ({1e3 * dev_s / args.steps:.0f} ms per launch)")

    # end to end through the C ABI with host buffers: a whole solve of every
    # e2e_batches-th grid point (host points in, host estimates out, the
    # copies and the tail of the longest walks inside the timed region)
    _barrier(world)
    e2e_steps = 0
    e2e_h2d = e2e_d2h = 0
    e2e_err2 = e2e_ref2 = 0.0
    e2e_walks = 0
    t0 = time.perf_counter()
    for i in range(args.e2e_steps):
        pts_h = np.ascontiguousarray(grid_pts[i:: args.e2e_batches])
        h = wost.wost_solve(S.handle, pts_h, walks, sc["epsilon"], sc["r_min"], sc["max_steps"],
                            seed=seed0 + 500 + i, kernel="resumable", block_size=args.block)
        wost.wost_wait(h, 900.0)
        mean, se, wdone, pe = wost.wost_poll(h, len(pts_h))
        wost.wost_solve_destroy(h)
        e2e_steps += pe["total_steps"]
        e2e_walks += int(wdone.sum())
        e2e_h2d += pts_h.nbytes
        e2e_d2h += len(pts_h) * 8 * 4 + 4 * 8 + 16  # sum, sumsq, walks, steps + counters
        u = scenes.exact_u("sin2x_cos3y", (), pts_h)
        e2e_err2 += float(np.sum((mean - u) ** 2))
        e2e_ref2 += float(np.sum(u**2))
    e2e_t = _max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_val = _sum_over_ranks(float(e2e_steps), world, "cuda") / e2e_t
    steps_per_walk = e2e_steps / max(1, e2e_walks)
    e2e_rel = float(np.sqrt(e2e_err2 / e2e_ref2))
    _log(f"e2e {e2e_val:.3e} steps/s, rel RMS {e2e_rel:.3f}")

    peaks, peak_src = _measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clk.get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1470.0)
    fp32 = 2 * 128 * sms * mhz * 1e6 / 1e12  # TFLOP/s: FMA = 2 flops, 128 FP32 lanes per SM
    fp32_src = f"2 x 128 x {sms} SMs x {mhz:.0f} MHz (median SM clock of the run)"
    l2_gbs = measure_read_gbs(torch, wost, stream, 48 << 20, 40)
    hbm_gbs = measure_read_gbs(torch, wost, stream, 4 << 30, 2, reps=3)
    _log(f"read probe: L2 {l2_gbs:.0f} GB/s, HBM {hbm_gbs:.0f} GB/s")
    roof = roofline_block("k_walk_resume<2>", bytes_step, flops_step, total_steps, dev_s, args.steps, peaks,
                          peak_src, l2_gbs, hbm_gbs, fp32, fp32_src,
                          profiled_traffic("k_walk_resume<2>", kernel_source_hash()),
                          {k: v / r["total_steps"] for k, v in r["counts"].items()})
    line_extra = {}
    if rank == 0 and world == 1 and not args.headline_only:
        for name, fn in (("flower", lambda: sub_flower(wost, torch, stream)),
                         ("cube_torus_3d", lambda: sub_cube_torus(wost, torch, args, stream, flush, peaks, peak_src,
                                                                  l2_gbs, hbm_gbs, fp32, fp32_src)),
                         ("keyhole", lambda: sub_keyhole(wost, torch, stream)),
                         ("batch", lambda: sub_batch(wost, torch, args)),
                         ("serve", lambda: sub_serve(wost, torch, args)),
                         ("serve_knee", lambda: sub_serve_knee(wost, torch, args))):
            _log(f"workload {name}")
            try:
                line_extra[name] = fn()
            except Exception as ex:  # a failed extra workload must not hide the headline line
                line_extra[name] = {"error": f"{type(ex).__name__}: {ex}"}
            _log(f"workload {name} done")
    if rank == 0:
        _log("oracle CPU baseline")
        base = cpu_baseline(sc, walks=args.cpu_walks) if (world == 1 and not args.no_cpu) else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "autotune": None if tune is None else {
                "chosen": {"lanes_per_walk": tune["lanes_per_walk"], "block": tune["block_size"]},
                "tried_steps_per_s": {f"{k[0]}x{k[1]}": v for k, v in tune["tried"].items()}},
            "config": _config_block(sc, {"kernel": "resumable",
                                         "block": args.block or (tune["block_size"] if tune else 128),
                                         "lanes_per_walk": info["lanes_per_walk"],
                                         "parallelism": f"replicas x{world}",
                                         "step": f"one launch of the whole-grid job ({n_all} points x {walks} walks):"
                                                 f" every resident lane runs up to {args.iters} walk steps, drawing"
                                                 f" new walks and carrying unfinished ones to the next launch",
                                         "iters_per_launch": args.iters}),
            "points_per_s": value / (steps_per_walk * walks),
            "mean_steps_per_walk": steps_per_walk,
            "launch_ms": per_launch_ms,
            "job_progress": {"walks_done": int(pr["walks_done"]), "steps_run": int(pr["steps_run"]),
                             "launches": int(pr["launches"])},
            "e2e": {"value": e2e_val, "unit": UNIT,
                    "h2d_bytes_per_step": int(e2e_h2d / max(args.e2e_steps, 1)),
                    "d2h_bytes_per_step": int(e2e_d2h / max(args.e2e_steps, 1)),
                    "what": f"complete resumable solves of every {args.e2e_batches}th grid point x {walks} walks from"
                            f" host memory (wost_solve + wost_wait + wost_poll), per solve",
                    "rel_rms_error_vs_exact": e2e_rel,
                    "rel_rms_points": int(sum(len(grid_pts[i:: args.e2e_batches]) for i in range(args.e2e_steps)))},
            "error_condition": error_condition(value, steps_per_walk, walks, e2e_rel),
            "gpu_launches": args.steps,
            "clocks": clk,
            "roofline": roof,
            "cpu_baseline": base,
            "scene": {k: info[k] for k in ("n_dirichlet", "n_neumann", "n_silhouette", "nodes_dirichlet",
                                           "nodes_neumann", "nodes_silhouette", "depth_dirichlet",
                                           "depth_neumann", "depth_silhouette", "device_bytes", "build_seconds",
                                           "lanes_per_walk", "stack_depth")},
        }
        line.update(line_extra)
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_batch(args):
    """The batched workload alone (--mode batch)."""
    import torch

    from paper_2302_11815_gb300 import wost

    wost.load()
    print(json.dumps(dict(mode="batch", **sub_batch(wost, torch, args))), flush=True)
    return 0


def run_serve(args):
    """The serving workload alone (--mode serve)."""
    import torch

    from paper_2302_11815_gb300 import wost

    wost.load()
    print(json.dumps(dict(mode="serve", **sub_serve(wost, torch, args))), flush=True)
    return 0


def run_profile_case(args):
    """The benchmark job for a profiler: the whole-grid resumable solve,
    `--warmup` launches then `--steps` launches of `--iters` walk steps per
    lane (profile e.g. with -k regex:k_walk_resume -s <warmup> -c 1)."""
    import torch

    from paper_2302_11815_gb300 import scenes, wost

    wost.load()
    sc = scenes.config2()
    S = wost.Scene(sc)
    pts = torch.from_numpy(np.ascontiguousarray(sc["points"], np.float32)).cuda()
    h = wost.wost_solve(S.handle, pts, sc["walks"], sc["epsilon"], sc["r_min"], sc["max_steps"], seed=5,
                        kernel="resumable", block_size=args.block)
    out, steps, before = [], [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        wost.wost_solve_advance(h, args.iters)
        torch.cuda.synchronize()
        out.append(time.perf_counter() - t0)
        _, _, _, pr = wost.wost_poll(h, len(pts))
        steps.append(int(pr["steps_run"]) - before)  # walk steps of this launch (divides ncu's bytes)
        before = int(pr["steps_run"])
    wost.wost_solve_destroy(h)
    print(json.dumps({"mode": "profile", "points": len(pts), "launches": int(pr["launches"]),
                      "iters": args.iters, "steps_run": before, "steps_per_launch": steps, "launch_s": out}),
          flush=True)
    S.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="main", choices=["main", "batch", "serve", "profile"])
    ap.add_argument("--batch-scenes", type=int, default=64)
    ap.add_argument("--batch-max-points", type=float, default=2e3)
    ap.add_argument("--batch-max-walks", type=float, default=64)
    ap.add_argument("--batch-max-prims", type=float, default=5e4)
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-max-points", type=float, default=2.56e5)
    ap.add_argument("--serve-total-prims", type=float, default=5e6)
    ap.add_argument("--serve-walk-cap", type=int, default=4096)
    ap.add_argument("--serve-max-wait", type=float, default=5.0)
    ap.add_argument("--serve-drain", type=float, default=30.0)
    ap.add_argument("--knee-rate", type=float, default=0.5, help="requests/s of the second serving run")
    ap.add_argument("--knee-seconds", type=float, default=60.0)
    ap.add_argument("--knee-walk-cap", type=int, default=64)
    ap.add_argument("--knee-drain", type=float, default=30.0)
    ap.add_argument("--iters3", type=int, default=1024, help="walk steps per lane per launch, 3D workload")
    ap.add_argument("--steps3", type=int, default=5, help="timed launches, 3D workload")
    ap.add_argument("--headline-only", action="store_true", help="skip the other workloads")
    ap.add_argument("--round-seconds", type=float, default=0.02)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--iters", type=int, default=4096, help="walk steps per lane per launch")
    ap.add_argument("--e2e-batches", type=int, default=16, help="the e2e solve takes every n-th grid point")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="persistent", choices=["plain", "persistent"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--count-stride", type=int, default=16)
    ap.add_argument("--cpu-walks", type=int, default=48, help="oracle walks per sampled point")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.mode == "batch":
        sys.exit(run_batch(args))
    if args.mode == "serve":
        sys.exit(run_serve(args))
    if args.mode == "profile":
        sys.exit(run_profile_case(args))
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    sys.exit(run_reference(args) if args.impl == "reference" else run_ours(args))


if __name__ == "__main__":
    main()
