"""Served progressive rendering on one GPU (continuous batching).

Requests arrive over time; each asks for a progressive NEB render of its own
scene and resolution until the relative RMSE of its image falls to a stated
target.  The error is estimated from the job's own samples: the library sums
the contributions of even and odd iterations apart, and the spread of the two
half-means gives the variance of the image (neb_error_estimate).  A job is
checked every `check_every` iterations from `min_iters` on and retired when
its estimate is at or below its target, or at `max_iters`.

The server runs in rounds.  Waiting requests are admitted in arrival order
while their predicted device memory (neb_job_device_bytes) fits the budget
and a slot is free; a setup thread then creates the job's context, uploads
its scene and builds its BVH on the job's own stream while the resident jobs
keep iterating, and the job joins the first round that starts after its setup
is done.  In a round every resident job advances one iteration, all of them
overlapping on the GPU (neb_iterate_batch), and the round ends when those
jobs' streams have drained (setups in flight are not waited for).  Every
job's BVH, octree, photon grid and FP64 sums stay on the device between its
iterations; retired jobs are resolved to host memory and their device memory
released.

A job's image depends only on its own scene, settings and seed: it is the same
whatever else is resident (neb_iterate_batch runs each job exactly as
neb_iterate would).  The comparison schedule, `run_sequential`, serves the same
requests one at a time in arrival order with the same retirement rule.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import time

import numpy as np

from . import neb


@dataclasses.dataclass
class Request:
    """A render job: scene, RenderConfig, arrival time in seconds and the
    relative RMSE it asks for (None: run rc.iterations iterations)."""
    scene: object
    rc: object
    arrival: float
    rid: int = 0
    target_rmse: float | None = None


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    started: float
    finished: float
    iterations: int
    image: np.ndarray | None
    iter_latencies: list
    paths: int = 0
    rmse: float | None = None
    reached: bool = True

    @property
    def time_to_target(self):
        return self.finished - self.arrival


class _Job:
    def __init__(self, req: Request, keep_image: bool):
        self.req = req
        self.ctx = neb.Context(neb.make_config(req.rc))    # on its own stream
        self.ctx.scene_upload(req.scene)
        self.ctx.build_bvh()
        self.ctx.synchronize()
        self.done = 0
        self.latencies = []
        self.keep_image = keep_image
        self.rmse = None


def job_bytes(req: Request) -> int:
    s = req.scene
    return neb.job_device_bytes(neb.make_config(req.rc), s.n_tri, s.n_sph, len(s.mats), s.n_emitters)


def _should_retire(job: _Job, min_iters: int, max_iters: int, check_every: int) -> bool:
    """The retirement rule: a fixed iteration count, or the error estimate
    at or below the target (checked every check_every iterations from
    min_iters on), or max_iters."""
    req = job.req
    if req.target_rmse is None:
        return job.done >= req.rc.iterations
    if job.done >= max_iters:
        job.rmse = job.ctx.error_estimate()
        return True
    if job.done >= min_iters and (job.done - min_iters) % check_every == 0:
        job.rmse = job.ctx.error_estimate()
        return job.rmse <= req.target_rmse
    return False


def _finish(job: _Job, now: float, admitted: float, started: float) -> Result:
    img = job.ctx.resolve() if job.keep_image else None
    job.ctx.close()
    rc = job.req.rc
    reached = job.req.target_rmse is None or (job.rmse is not None and job.rmse <= job.req.target_rmse)
    return Result(job.req.rid, job.req.arrival, admitted, started, now, job.done, img, job.latencies,
                  rc.width * rc.height * job.done, job.rmse, reached)


def run_served(requests, budget_bytes: float, max_jobs: int = 64, keep_images: bool = False,
               min_iters: int = 16, max_iters: int = 256, check_every: int = 4):
    """Continuous batching.  Returns (results, rounds, rejected): the finished
    jobs, (start, duration, resident jobs) of every round, and the ids of
    requests larger than the whole budget.  Arrival times are seconds after
    the call starts."""
    pending = sorted(requests, key=lambda r: r.arrival)
    rejected = []
    resident: list[tuple[_Job, float, float, int]] = []   # job, admission time, first round, predicted bytes
    preparing: list[tuple[cf.Future, float, int]] = []     # setup, admission time, predicted bytes
    used = 0
    results, rounds = [], []
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=1) as setup:
        while pending or resident or preparing:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now and len(resident) + len(preparing) < max_jobs:
                b = job_bytes(pending[0])
                if b > budget_bytes:
                    rejected.append(pending.pop(0).rid)                # never fits
                    continue
                if used + b > budget_bytes:
                    break                                              # wait for memory to free up
                req = pending.pop(0)
                preparing.append((setup.submit(_Job, req, keep_images), now, b))
                used += b
            still = []
            for fut, adm, b in preparing:                              # setups done join this round
                if fut.done():
                    resident.append((fut.result(), adm, time.perf_counter() - t0, b))
                else:
                    still.append((fut, adm, b))
            preparing = still
            if not resident:
                if preparing:                                          # idle until a setup is done
                    cf.wait([f for f, _, _ in preparing], timeout=0.05, return_when=cf.FIRST_COMPLETED)
                elif pending:
                    time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.05)))
                continue
            r_start = time.perf_counter()
            neb.iterate_batch([j.ctx for j, _, _, _ in resident], 1)
            for j, _, _, _ in resident:
                j.ctx.synchronize()
            r_end = time.perf_counter()
            lat = r_end - r_start
            rounds.append((r_start - t0, lat, len(resident)))
            keep = []
            for job, adm, started, b in resident:
                job.done += 1
                job.latencies.append(lat)
                if _should_retire(job, min_iters, max_iters, check_every):
                    results.append(_finish(job, time.perf_counter() - t0, adm, started))
                    used -= b
                else:
                    keep.append((job, adm, started, b))
            resident = keep
    return results, rounds, rejected


def run_sequential(requests, keep_images: bool = False, min_iters: int = 16, max_iters: int = 256,
                   check_every: int = 4):
    """The comparison schedule: one job at a time in arrival order, each run
    to its target with the same retirement rule, its iterations timed one by
    one."""
    results = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        adm = time.perf_counter() - t0
        job = _Job(req, keep_images)
        started = time.perf_counter() - t0
        while True:
            a = time.perf_counter()
            job.ctx.iterate(1)
            job.ctx.synchronize()
            job.latencies.append(time.perf_counter() - a)
            job.done += 1
            if _should_retire(job, min_iters, max_iters, check_every):
                break
        results.append(_finish(job, time.perf_counter() - t0, adm, started))
    return results


def poisson_requests(jobs, rate_per_s: float, seed: int = 0, min_iters: int = 16, max_iters: int = 256,
                     pilot=None):
    """Requests for [(scene, rc)] with exponential inter-arrival times of mean
    1/rate.  Each request draws n log-uniform in [min_iters, max_iters]; with
    a pilot (a function (scene, rc) -> relative RMSE of one iteration) it asks
    for the relative RMSE pilot / sqrt(n), which the job reaches after about n
    iterations; without one it asks for n iterations."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i, (s, rc) in enumerate(jobs):
        t += rng.exponential(1.0 / rate_per_s)
        n = min_iters * (max_iters / min_iters) ** rng.uniform()
        rc.iterations = int(round(n))
        target = None if pilot is None else float(pilot(s, rc)) / float(np.sqrt(n))
        out.append(Request(s, rc, t, i, target))
    return out


def pilot_rmse(scene, rc, iterations: int = 16, side: int = 128) -> float:
    """Relative RMSE of one iteration of a job, estimated from `iterations`
    iterations of the same scene and settings at side x side pixels (the
    per-pixel noise depends on the samples per pixel, not on the resolution)."""
    import copy
    small = copy.copy(rc)
    small.width = small.height = side
    small.octree_capacity = max(1 << 16, min(rc.octree_capacity, 4 * side * side))
    ctx = neb.Context(neb.make_config(small))
    ctx.scene_upload(scene)
    ctx.build_bvh()
    ctx.iterate(iterations)
    e = ctx.error_estimate()
    ctx.close()
    return e * float(np.sqrt(iterations))


def summary(results, wall_s: float):
    """Per-iteration latency percentiles (every iteration of every job),
    time-to-target statistics and aggregate throughput of a schedule."""
    lat = np.array([x for r in results for x in r.iter_latencies])
    ttt = np.array([r.time_to_target for r in results])
    wait = np.array([r.started - r.arrival for r in results])
    its = np.array([r.iterations for r in results])
    paths = sum(r.paths for r in results)
    return {"jobs": len(results),
            "iteration_latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                     "p99": 1e3 * float(np.percentile(lat, 99))},
            "time_to_target_s": {"mean": float(ttt.mean()), "p50": float(np.percentile(ttt, 50)),
                                 "p99": float(np.percentile(ttt, 99))},
            "wait_before_first_iteration_s": {"mean": float(wait.mean()), "p99": float(np.percentile(wait, 99))},
            "iterations": {"mean": float(its.mean()), "min": int(its.min()), "max": int(its.max())},
            "reached_target": float(np.mean([r.reached for r in results])),
            "wall_s": wall_s, "paths": paths, "mpaths_per_s": paths / wall_s / 1e6}
