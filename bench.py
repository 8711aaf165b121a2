#!/usr/bin/env python
"""Benchmark of the NEB iteration on one or more GB300s.

Workload (default): the many-lights scene, the largest single-GPU
configuration: the large-city geometry (400 x 400 seeded boxes, ~1.95M
triangles, a glass torus of extent diag/1000) with 65,536 sphere lights chosen
through a power alias table and a rough-conductor roof patch, 1920 x 1080
camera paths per iteration, maximum path length 10, merge radius 1e-3 of the
torus extent, 4M-word density octree, split factor 4.  A step is one NEB
iteration (all passes) over the 2,073,600 paths of one image.
--workload large_city: the same city with 16 lights at 1280 x 720.

Prints one JSON line (rank 0).  value = camera paths per second over all GPUs
(Mpaths/s) with the scene resident in HBM; e2e = the same metric through the
C ABI from pinned host buffers (scene upload, BVH build, iterations and an
image read back per step inside the timed region).

--impl reference times the CPU oracle (the plain single-threaded C
implementation used by the parity tests) on a band of the same image.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpaths/s"
WORKLOAD = "many_lights"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--res", default=None, help="WxH override (smaller cases for ncu captures)")
    ap.add_argument("--bvh", type=int, default=0, help="0 PLOC (default), 1 Karras LBVH")
    ap.add_argument("--octree-cap", type=int, default=None, help="octree capacity override (analysis runs)")
    ap.add_argument("--batch", type=int, default=0,
                    help="batched-jobs measurement: N heterogeneous jobs, batched vs sequential per-job launches")
    ap.add_argument("--mem-budget-gb", type=float, default=150.0, help="admission cap of the batched jobs")
    ap.add_argument("--serve", type=int, default=0,
                    help="served progressive rendering: R requests with Poisson arrivals, each to a relative-RMSE "
                         "target, vs sequential per-job launches")
    ap.add_argument("--rate", type=float, default=200.0, help="mean request arrival rate (per second) for --serve")
    ap.add_argument("--ablation", action="store_true",
                    help="density estimators of Sec. 5 (octree, naive, k nearest) on one iteration's NEE vertices")
    ap.add_argument("--lp-photons", type=int, default=0,
                    help="NEB+LP (Sec. 6.1): conventional light photons per iteration in addition to NEB photons")
    ap.add_argument("--merge-mode", type=int, default=0, choices=[0, 1, 2],
                    help="photon merge: 0 dense hits per cell, sparse per hit (default); 1 per hit; 2 per cell")
    ap.add_argument("--autotune", type=int, default=0,
                    help="run the autotuner (this many iterations per candidate) before the warm-up")
    ap.add_argument("--live-octree-cap", type=int, default=1 << 27,
                    help="word pool of the second measurement, large enough that the octree never fills "
                         "(0: skip it)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- replicas: the pass does not shard, so N GPUs run N independent renders
def replica_seed(rank):
    """Each replica renders its own sample stream (Philox key = seed)."""
    return rank


def max_over_ranks(x, dist=None, device="cpu"):
    """The job's time is the slowest rank's (all-reduce MAX; identity on one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rates(d, world, ms_total):
    """Secondary throughputs of the timed steps, whole job (every rank did the
    same work): rays traced (camera + shadow + photon), merge candidates tested
    and accepted, octree inserts and queries (a robust query counts 5)."""
    s = ms_total / 1000.0
    if s <= 0:
        return None
    f = lambda n: world * n / s / 1e6  # noqa: E731
    rays = d.get("camera_rays", 0) + d.get("shadow_rays", 0) + d.get("photon_hits", 0)
    return {"Mrays_per_s": f(rays), "Mmerge_tests_per_s": f(d.get("merge_tests", 0)),
            "Mmerges_per_s": f(d.get("merges", 0)), "Moctree_inserts_per_s": f(d.get("octree_inserts", 0)),
            "Moctree_queries_per_s": f(d.get("octree_queries", 0))}


def job_value(world, paths_per_step, steps, seconds):
    """Whole-job throughput in Mpaths/s: the paths of all replicas over the job time."""
    return world * paths_per_step * steps / seconds / 1e6


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
def load_peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Counters of a stage's kernel from ncu captures of these sources (profiles/
# holds the summaries and the commands): DRAM traffic (dram__bytes_read.sum +
# dram__bytes_write.sum) per launch at the full workload, and from the full
# capture of a smaller image of the same scene the lane efficiency
# (smsp__thread_inst_executed_per_inst_executed / 32) and the issue-active
# fraction (sm__inst_issued ... per active cycle).  Reported only while the
# kernel's sources hash to the value recorded with the capture, else null.
TRAFFIC_SOURCES = ("paper_1909_00573_gb300/csrc/neb_trace.cu", "paper_1909_00573_gb300/csrc/neb_device.cuh",
                   "paper_1909_00573_gb300/csrc/neb_types.h")
NCU_COUNTERS = {  # (workload, stage): counters of the stage's kernel, captured from these sources
    ("many_lights", "trace_camera"): {
        "bound": "issue",              # instruction issue on dependent chains and divergence, not DRAM
        "bytes_per_launch": 161644518,  # mean DRAM read + write of the 10 camera launches of an iteration
        "lane_efficiency": 12.06 / 32,  # smsp__thread_inst_executed_per_inst_executed, 960 x 540 capture
        "issue_active": 0.688,          # smsp__issue_active, 960 x 540 capture
        "sources_sha256": "44e3203109cfef4c8680dfca0c9edc99f29c05d7d751e6f138eed3cedede8818",
        "profile": "profiles/k_trace_closest_many_lights.md"},
    ("large_city", "trace_camera"): {
        "bound": "issue",
        "bytes_per_launch": 73705164,   # mean DRAM read + write of the 10 camera launches of an iteration
        "lane_efficiency": 10.79 / 32,  # smsp__thread_inst_executed_per_inst_executed, 640 x 360 capture
        "issue_active": 0.618,          # smsp__issue_active, 640 x 360 capture
        "sources_sha256": "44e3203109cfef4c8680dfca0c9edc99f29c05d7d751e6f138eed3cedede8818",
        "profile": "profiles/k_trace_closest_large_city.md"},
}


def sources_sha256():
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_counters(workload, stage):
    """The stored ncu counters of (workload, stage), or None when the sources changed since."""
    e = NCU_COUNTERS.get((workload, stage))
    if not e or e["sources_sha256"] != sources_sha256():
        return None
    return e


def stage_bytes(stage, d, P, iters):
    """Algorithmic bytes of one stage over the profiled iterations, with and
    without BVH traversal.  Per-unit figures: 128 B per visit of a 4-wide BVH
    node and 48 B per triangle test (traversal); 32 B ray read + 8 B hit
    written per traced ray; 64 B per ray record read or written; 112 B per
    NEE record; 48 B per random-hit event; 16 B per merge candidate tested,
    48 B + 24 B of FP64 atomics per accepted merge."""
    trav = {"trace_camera": 0, "shadow": 1, "trace_photon": 2}
    if stage == "trace_camera":
        rec = 40 * d["camera_rays"]
    elif stage == "trace_photon":
        rec = 40 * d["photon_hits"]
    elif stage == "shadow":
        rec = 32 * d["shadow_rays"] + 4 * d["photons"]           # ray record read, lit-list entries (about one per photon)
    elif stage == "extend":
        return (72 * d["camera_rays"] + 64 * max(d["camera_rays"] - P * iters, 0) + 112 * d["nee_vertices"] +
                48 * d["random_hits"]), None
    elif stage == "photon":
        return 72 * d["photon_hits"] + 64 * d["photon_hits"] + 16 * d["merge_tests"] + 72 * d["merges"], None
    else:
        return None, None
    k = trav[stage]
    tr = 128 * d["stage_node_visits"][k] + 48 * d["stage_prim_tests"][k]
    return rec + tr, rec


def stats_delta(a, b):
    out = {}
    for k, v in b.items():
        if isinstance(v, list):
            out[k] = [x - y for x, y in zip(v, a[k])]
        elif isinstance(v, int):
            out[k] = v - a.get(k, 0)
    return out


def cpu_baseline_sample(scene, rc, rows, n_iter=1):
    from oracle import oracle as O
    W, H = rc.width, rc.height
    r0 = max(0, H // 2 - rows // 2)
    res = O.render(scene, rc, n_iter=n_iter, pixel_range=(r0 * W, (r0 + rows) * W), want_split=False)
    t = float(sum(res["iter_seconds"]))
    paths = rows * W * n_iter
    return paths, t, f"{rows} rows x {W} px (rows {r0}..{r0 + rows - 1}) of the {W}x{H} image, " \
                     f"{n_iter} iteration(s), single thread"


# ----------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1909_00573_gb300 import scenes
    O.build()
    scene, rc = scenes.workload(args.workload)
    steps, warm = max(args.steps, 1), max(args.warmup, 0)
    # size one step so the whole run takes ~90 s of oracle time (~5k paths/s)
    t_step = 90.0 / (steps + warm)
    rows = max(1, int(t_step * 5000 / rc.width))
    W = rc.width
    r0 = max(0, rc.height // 2 - rows // 2)
    res = O.render(scene, rc, n_iter=steps + warm, pixel_range=(r0 * W, (r0 + rows) * W), want_split=False)
    it = res["iter_seconds"][warm:]
    paths = rows * W
    sec = float(sum(it))
    value = paths * len(it) / sec / 1e6
    sample = f"{rows} rows x {W} px (rows {r0}..{r0 + rows - 1}) of the {W}x{rc.height} image per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1000 * sec / len(it), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(rc, scene),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(rc, scene):
    return {"workload": f"{scene.name}: {scene.n_tri} triangles, {scene.n_sph} sphere lights, "
                        f"{rc.width}x{rc.height}, 1 spp per iteration, D={rc.max_depth}, "
                        f"r={rc.merge_radius:.3g}, octree {rc.octree_capacity} nodes, split {rc.split_factor}",
            "paths_per_step": rc.width * rc.height, "max_depth": rc.max_depth,
            "octree_mode": "concurrent" if rc.octree_mode == 0 else "sequential",
            "strategies": "e+E+P" + ("+LP" if rc.strategy_mask & 8 else ""),
            "lp_photons": int(getattr(rc, "lp_photons", 0)) if rc.strategy_mask & 8 else 0,
            "l2": "inputs larger than L2 (scene + BVH + per-iteration records > 129 MB)"}


def admission_waves(sizes, budget):
    """Jobs in order into waves whose summed device bytes fit the budget: a
    job that does not fit the current wave starts the next one; a job larger
    than the budget alone is rejected.  Returns ([[job index, ...], ...],
    number rejected)."""
    waves, wave, resident, rejected = [], [], 0, 0
    for i, b in enumerate(sizes):
        if b > budget:
            rejected += 1
            continue
        if wave and resident + b > budget:
            waves.append(wave)
            wave, resident = [], 0
        wave.append(i)
        resident += b
    if wave:
        waves.append(wave)
    return waves, rejected


def run_batch(args):
    """Batched jobs: a seeded mix of heterogeneous jobs (rooms and cities of
    ~1.3k to ~500k triangles, 128^2 to 1024^2 pixels, 1 to 64 lights).  Jobs
    are admitted in order while their predicted device memory fits the
    budget; a job that does not fit starts the next wave, so every job runs
    (a wave's jobs are set up, iterated and closed before the next wave).
    Times args.steps iterations of every job of every wave (a) as plain
    per-job launches, one job after the other, and (b) batched with
    neb_iterate_batch.  Both schedules give every job the same image per
    iteration, so the ratio of the times is also the ratio of the times to
    any equal RMSE."""
    # more hardware work queues for the many job streams (read at CUDA init)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    from paper_1909_00573_gb300 import build as B
    B.build()
    from paper_1909_00573_gb300 import neb, scenes
    jobs = scenes.batch_jobs(args.batch, seed=rank, iterations=args.steps)
    for _, rc in jobs:
        rc.merge_mode = args.merge_mode
    budget = args.mem_budget_gb * 1e9
    sizes = [neb.job_device_bytes(neb.make_config(rc), s.n_tri, s.n_sph, len(s.mats), s.n_emitters)
             for s, rc in jobs]
    plan, rejected = admission_waves(sizes, budget)
    waves = [([jobs[i] for i in w], sum(sizes[i] for i in w)) for w in plan]
    admitted = [j for w, _ in waves for j in w]
    paths = sum(rc.width * rc.height for _, rc in admitted)
    t_seq = t_batch = setup_s = 0.0
    launches, status = 0, 0
    clocks = ClockSampler(local)
    clocks.start()
    for wjobs, _ in waves:
        ctxs = []
        t0 = time.perf_counter()
        for s, rc in wjobs:
            ctx = neb.Context(neb.make_config(rc))   # each job on its own streams
            ctx.scene_upload(s)
            ctx.build_bvh()
            ctxs.append(ctx)
        torch.cuda.synchronize()
        setup_s += time.perf_counter() - t0
        neb.iterate_batch(ctxs, max(args.warmup, 1))
        torch.cuda.synchronize()
        l0 = sum(c.stats(check=False)["kernel_launches"] for c in ctxs)
        t0 = time.perf_counter()
        for c in ctxs:                                # plain per-job launches
            c.iterate(args.steps)
            torch.cuda.synchronize()
        t_seq += time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        neb.iterate_batch(ctxs, args.steps)           # batched
        torch.cuda.synchronize()
        t_batch += time.perf_counter() - t0
        launches += sum(c.stats(check=False)["kernel_launches"] for c in ctxs) - l0
        for c in ctxs:
            status |= c.stats(check=False)["status"]
            c.close()
        torch.cuda.synchronize()
    clk = clocks.stop()
    value = paths * args.steps / t_batch / 1e6
    seq = paths * args.steps / t_seq / 1e6
    tris = [s.n_tri + s.n_sph for s, _ in admitted]
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 1), "ms_per_step": 1000 * t_batch / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch of {len(admitted)} heterogeneous jobs (rooms and cities, "
                                   f"{min(tris)}..{max(tris)} primitives, 128^2..1024^2 px, 1..64 lights), "
                                   "one iteration of every job per step",
                       "jobs": len(admitted), "rejected_by_admission": rejected, "paths_per_step": paths,
                       "waves": len(waves), "resident_gb_per_wave": [round(r / 1e9, 2) for _, r in waves],
                       "mem_budget_gb": args.mem_budget_gb, "setup_s": setup_s,
                       "l2": "inputs larger than L2 (many scenes and per-iteration records)"},
            "sequential_per_job": {"value": seq, "unit": METRIC, "ms_per_step": 1000 * t_seq / args.steps},
            "speedup_vs_sequential": t_seq / t_batch,
            "time_to_equal_rmse_ratio": t_seq / t_batch,
            "timing": "host clock around device synchronisation (many streams), summed over the waves",
            "gpu_launches": int(launches), "clocks": clk, "status": int(status)}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_serve(args):
    """Served progressive rendering: args.serve requests drawn from the
    batched-jobs mix, Poisson arrivals at args.rate per second, each asking
    for a relative RMSE that a pilot run (16 iterations of the same job at
    128 x 128, outside the timed region) predicts it reaches after 16 to 256
    iterations (log-uniform); a job retires when its two-half error estimate
    (checked every 4 iterations) reaches the target, or at 256 iterations.
    Admission capped at --mem-budget-gb.  The same requests are served by
    continuous batching and by sequential per-job launches in arrival order."""
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_1909_00573_gb300 import build as B
    B.build()
    from paper_1909_00573_gb300 import scenes, serve
    budget = args.mem_budget_gb * 1e9
    t_p = time.perf_counter()
    jobs = scenes.batch_jobs(args.serve, seed=rank)
    for _, rc in jobs:
        rc.merge_mode = args.merge_mode
    reqs = serve.poisson_requests(jobs, args.rate, seed=rank, pilot=serve.pilot_rmse)
    pilot_s = time.perf_counter() - t_p
    out = {}
    clocks = ClockSampler(local)
    clocks.start()
    for mode in ("served", "sequential"):
        t0 = time.perf_counter()
        if mode == "served":
            res, rounds, rejected = serve.run_served(reqs, budget, max_jobs=64)
        else:
            res, rejected = serve.run_sequential(reqs), []
        wall = time.perf_counter() - t0
        out[mode] = serve.summary(res, wall)
        out[mode]["rejected"] = len(rejected)
        if mode == "served":
            out[mode]["rounds"] = len(rounds)
            out[mode]["max_resident"] = max(n for _, _, n in rounds)
            out[mode]["mean_resident"] = float(np.mean([n for _, _, n in rounds]))
    clk = clocks.stop()
    sv, sq = out["served"], out["sequential"]
    targets = [r.target_rmse for r in reqs]
    line = {"metric": METRIC, "value": sv["mpaths_per_s"], "unit": METRIC, "n_gpus": 1, "steps": sv["rounds"],
            "warmup": 0, "ms_per_step": sv["iteration_latency_ms"]["p50"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"served progressive rendering: {args.serve} requests from the batched-jobs mix, "
                                   f"Poisson arrivals at {args.rate:g}/s, each to a relative-RMSE target "
                                   f"(two-half estimate; 16..256 iterations by its pilot), admission cap "
                                   f"{args.mem_budget_gb:g} GB, at most 64 resident jobs",
                       "target_rmse": {"min": float(min(targets)), "median": float(np.median(targets)),
                                       "max": float(max(targets))},
                       "pilot_s": pilot_s},
            "served": sv, "sequential_per_job": sq,
            "throughput_ratio": sv["mpaths_per_s"] / sq["mpaths_per_s"],
            "time_to_target_mean_ratio": sq["time_to_target_s"]["mean"] / sv["time_to_target_s"]["mean"],
            "timing": "host clock around device synchronisation", "clocks": clk}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_ablation(args):
    """The density estimators of Sec. 5 on the NEE vertices of one iteration
    of the workload (after one warm-up iteration): the octree (concurrent
    insert + robust query, as the pass uses it), the naive estimator (radius 4
    merge radii) and the k-nearest estimator (k = 4, the paper's smallest),
    each timed on the device (structure build + one query per vertex)."""
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_1909_00573_gb300 import build as B
    B.build()
    from paper_1909_00573_gb300 import neb, scenes
    scene, rc = scenes.workload(args.workload)
    ctx = neb.Context(neb.make_config(rc))
    ctx.scene_upload(scene)
    ctx.build_bvh()
    ctx.iterate(2)
    pos, nrm = ctx.read_nee_vertices()
    ctx.close()
    v = scene.tri.reshape(-1, 3)
    lo = v.min(0)
    hi = v.max(0)
    if len(scene.sph):
        lo = np.minimum(lo, (scene.sph[:, :3] - scene.sph[:, 3:]).min(0))
        hi = np.maximum(hi, (scene.sph[:, :3] + scene.sph[:, 3:]).max(0))
    radius, k = 4.0 * rc.merge_radius, 4
    neb.density_estimators(pos[:4096], nrm[:4096], lo, hi, 1 << 16, rc.split_factor, radius, k)   # warm-up
    rho, ms = neb.density_estimators(pos, nrm, lo, hi, rc.octree_capacity, rc.split_factor, radius, k)
    n = len(pos)
    pos_ok = [(r > 0).mean() for r in rho]
    spread = {}
    for name, a, b in (("naive_vs_octree", rho[1], rho[0]), ("knn_vs_octree", rho[2], rho[0])):
        ok = (a > 0) & (b > 0)
        q = np.log10(a[ok] / b[ok])
        spread[name] = {"median_log10_ratio": float(np.median(q)), "iqr_log10_ratio": float(np.subtract(*np.percentile(q, [75, 25])))}
    line = {"metric": "M density estimates/s", "value": n / (ms[0] / 1e3) / 1e6, "unit": "M estimates/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": float(ms[0]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 normalisation)", "data": "synthetic",
            "config": {"workload": f"density estimators of Sec. 5 on the {n} NEE vertices of one iteration of "
                                   f"{args.workload} ({rc.width}x{rc.height}, D={rc.max_depth})",
                       "naive_radius": radius, "k": k, "octree_capacity": rc.octree_capacity,
                       "split_factor": rc.split_factor},
            "ms": {"octree": float(ms[0]), "naive": float(ms[1]), "knn": float(ms[2])},
            "speedup_of_octree": {"vs_knn": float(ms[2] / ms[0]), "vs_naive": float(ms[1] / ms[0])},
            "fraction_positive": {"octree": float(pos_ok[0]), "naive": float(pos_ok[1]), "knn": float(pos_ok[2])},
            "agreement": spread}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ablation:
        return run_ablation(args)
    if args.batch > 0:
        return run_batch(args)
    if args.serve > 0:
        return run_serve(args)
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1909_00573_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if dist:
        dist.barrier()
    from paper_1909_00573_gb300 import neb, scenes

    scene, rc = scenes.workload(args.workload)
    if args.res:
        rc.width, rc.height = (int(x) for x in args.res.lower().split("x"))
    if args.octree_cap:
        rc.octree_capacity = args.octree_cap
    if args.lp_photons > 0:
        rc.strategy_mask |= 8
        rc.lp_photons = args.lp_photons
    rc.seed = replica_seed(rank)        # replicas render independent sample streams
    rc.merge_mode = args.merge_mode
    P = rc.width * rc.height
    # a dedicated (non-default) stream: the library's kernels and the timing
    # events must be ordered on the same stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    ctx = neb.Context(neb.make_config(rc, bvh_builder=args.bvh), stream.cuda_stream)
    ctx.scene_upload(scene)
    torch.cuda.synchronize()
    t_b0 = time.perf_counter()
    ctx.build_bvh()
    bvh_build_ms = (time.perf_counter() - t_b0) * 1000.0
    bvh_cost = ctx.bvh_cost()
    if args.autotune > 0:
        ctx.autotune(args.autotune)
    tuning = ctx.tuning().as_dict()
    ctx.iterate(args.warmup)
    torch.cuda.synchronize()
    s0 = ctx.stats(check=False)
    t_wall0 = time.perf_counter()

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()          # ncu --profile-from-start off captures exactly the timed steps
    ev0.record(stream)
    ctx.iterate(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    wall_ms = (time.perf_counter() - t_wall0) * 1000.0
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    assert ms > 0.5 * wall_ms / 1.0 - 50.0, (ms, wall_ms)   # device time tracks the host clock
    clk = clocks.stop()
    s1 = ctx.stats(check=False)
    d = stats_delta(s0, s1)
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_value(world, P, args.steps, ms / 1000.0)

    # ---- per-stage times (CUDA events on the context stream), roofline of the dominant kernel
    ctx.set_profiling(True)
    p0 = ctx.stats(check=False)
    ctx.iterate(args.profile_steps)
    torch.cuda.synchronize()
    p1 = ctx.stats(check=False)
    stages = ctx.stage_times()
    ctx.set_profiling(False)
    pd = stats_delta(p0, p1)
    peak, peak_kind = load_peaks()
    dom = max(stages, key=lambda k: stages[k][0])
    dom_ms, dom_launches = stages[dom]
    byt, byt_nt = stage_bytes(dom, pd, P, args.profile_steps)
    roof = None
    if byt is not None and dom_ms > 0:
        per_launch = byt / dom_launches
        avg_ms = dom_ms / dom_launches
        achieved = per_launch / (avg_ms / 1000.0) / 1e9
        cnt = measured_counters(args.workload, dom)
        traffic = cnt["bytes_per_launch"] if cnt else None
        roof = {"bound": cnt["bound"] if cnt else "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "peak_kind": peak_kind, "bytes_per_launch": per_launch, "avg_launch_ms": avg_ms,
                "achieved_without_traversal": (None if byt_nt is None else
                                               (byt_nt / dom_launches) / (avg_ms / 1000.0) / 1e9),
                "dram_frac": (None if traffic is None else traffic / (avg_ms / 1000.0) / 1e9 / peak),
                "lane_efficiency": cnt["lane_efficiency"] if cnt else None,
                "issue_active": cnt["issue_active"] if cnt else None,
                "headroom": (cnt["lane_efficiency"] * cnt["issue_active"]
                             if cnt and cnt["lane_efficiency"] is not None and cnt["issue_active"] is not None
                             else None),
                "counters_source": cnt["profile"] if cnt else None}
    total_stage_ms = sum(v[0] for v in stages.values())
    ctx.close()

    # ---- the octree from a fresh start, in contexts created after every
    # kernel has been loaded: (a) the workload's word pool, iterations timed
    # one by one up to the warm-up count, and the iteration at which the pool
    # fills (from then on no cell splits, inserts count in their leaf: the
    # regime of the timed steps above); (b) a pool the tree does not fill
    # before the end of the timed steps, whose timed steps run the splitting
    # inserts (compare-and-swap counts)
    def fresh_run(capacity, timed_steps):
        rcx = scenes.workload(args.workload)[1]
        rcx.width, rcx.height, rcx.seed = rc.width, rc.height, rc.seed
        rcx.strategy_mask, rcx.lp_photons, rcx.merge_mode = rc.strategy_mask, rc.lp_photons, rc.merge_mode
        rcx.octree_capacity = capacity
        cx = neb.Context(neb.make_config(rcx, bvh_builder=args.bvh), stream.cuda_stream)
        cx.scene_upload(scene)
        cx.build_bvh()
        per_it, full_at = [], None
        for i in range(max(args.warmup, 1)):
            w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w0.record(stream)
            cx.iterate(1)
            w1.record(stream)
            torch.cuda.synchronize()
            per_it.append(w0.elapsed_time(w1))
            if full_at is None and cx.stats(check=False)["status"] & neb.STATUS_OCTREE_FULL:
                full_at = i + 1
        out = {"capacity_words": capacity, "ms_per_iteration_from_the_first": per_it,
               "full_at_iteration": full_at}
        if timed_steps > 0:
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0.record(stream)
            cx.iterate(timed_steps)
            l1.record(stream)
            torch.cuda.synchronize()
            ms_t = l0.elapsed_time(l1)
            out.update({"timed_steps_ms_per_step": ms_t / timed_steps,
                        "timed_steps_value": job_value(1, P, timed_steps, ms_t / 1000.0)})
        st = cx.stats(check=False)
        if full_at is None and st["status"] & neb.STATUS_OCTREE_FULL:
            out["full_during_timed_steps"] = True
        out.update({"words_used": st["octree_nodes"], "depth": st["octree_depth"]})
        cx.close()
        return out

    octree = {"timed_regime": "frozen (pool full: inserts count in their leaf, no splits)"
              if (s0["status"] & neb.STATUS_OCTREE_FULL) else "live (cells still split)",
              "fill": fresh_run(rc.octree_capacity, 0)}
    if args.live_octree_cap > 0:
        octree["live"] = fresh_run(args.live_octree_cap, args.steps)

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hs = scenes.Scene(pin(scene.tri), pin(scene.tri_mat), pin(scene.sph), pin(scene.sph_mat),
                          pin(scene.mats), pin(scene.cam), scene.name)
        img = torch.empty((rc.height, rc.width, 3), dtype=torch.float32).pin_memory()
        h2d = hs.tri.nbytes + hs.tri_mat.nbytes + hs.sph.nbytes + hs.sph_mat.nbytes + hs.mats.nbytes + hs.cam.nbytes
        ctx2 = neb.Context(neb.make_config(rc, bvh_builder=args.bvh), stream.cuda_stream)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2.scene_upload(hs)
        t_up = time.perf_counter()
        ctx2.build_bvh()
        t_bvh = time.perf_counter()
        ctx2.iterate_read(args.steps, img.data_ptr())   # every iteration's image copied to pinned host memory
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e, dist, "cuda")
        ctx2.close()
        e2e = {"value": job_value(world, P, args.steps, t_e2e), "unit": METRIC,
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(img.numel() * 4),
               "upload_ms": 1000 * (t_up - t0), "bvh_ms": 1000 * (t_bvh - t_up),
               "note": "scene upload + BVH build once per job (h2d amortised over the steps); after every "
                       "iteration its image is resolved and copied to pinned host memory (neb_iterate_read, "
                       "asynchronous: the copies overlap the next iteration)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        paths, sec, sample = cpu_baseline_sample(scene, rc, rows=64)
        cpu = {"value": paths / sec / 1e6, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(rc, scene), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(d.get("kernel_launches", 0)), "clocks": clk,
                "stages_ms_per_step": {k: v[0] / args.profile_steps for k, v in stages.items()},
                "stage_sum_ms_per_step": total_stage_ms / args.profile_steps,
                "rates": rates(d, world, ms),
                "counters_per_step": {k: (v / args.steps if not isinstance(v, list) else [x / args.steps for x in v])
                                      for k, v in d.items() if k not in ("iterations",)},
                "status": s1["status"], "octree": octree, "bvh_build_ms": bvh_build_ms,
                "bvh_sah": {"node_visits": bvh_cost[0], "prim_tests": bvh_cost[1]},
                "bvh": "PLOC" if args.bvh == 0 else "LBVH", "tuning": tuning,
                "tuning_source": "autotuned" if args.autotune > 0 else "defaults"}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
