"""Served progressive rendering on one GPU (continuous batching).

Requests arrive over time; each asks for a progressive NEB render of its own
scene and resolution to a target iteration count (the RMSE of the consistent
estimator falls with the iteration count, so a relative-RMSE target is stated
as the iterations that reach it).  The server runs in rounds.  Before a round
it admits waiting requests in arrival order while their predicted device
memory (neb_job_device_bytes) fits the budget and a slot is free, uploading
the scene and building its BVH; in the round every resident job advances one
iteration, all of them overlapping on the GPU (neb_iterate_batch); after the
round, jobs that reached their target are resolved to host memory and their
device memory is released.  Every job's BVH, octree, photon grid and FP64
accumulation stay on the device between its iterations.

A job's image depends only on its own scene, settings and seed: it is the same
whatever else is resident (neb_iterate_batch runs each job exactly as
neb_iterate would).  The comparison schedule, `run_sequential`, serves the same
requests one at a time in arrival order.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import neb


@dataclasses.dataclass
class Request:
    """A render job: scene, RenderConfig (iterations = target), arrival time in seconds."""
    scene: object
    rc: object
    arrival: float
    rid: int = 0


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    iterations: int
    image: np.ndarray | None
    iter_latencies: list
    paths: int = 0

    @property
    def time_to_target(self):
        return self.finished - self.arrival


class _Job:
    def __init__(self, req: Request, keep_image: bool, stream=None):
        self.req = req
        self.ctx = neb.Context(neb.make_config(req.rc), stream)
        self.ctx.scene_upload(req.scene)
        self.ctx.build_bvh()
        self.done = 0
        self.latencies = []
        self.keep_image = keep_image


def job_bytes(req: Request) -> int:
    s = req.scene
    return neb.job_device_bytes(neb.make_config(req.rc), s.n_tri, s.n_sph, len(s.mats), s.n_emitters)


def _sync():
    import torch
    torch.cuda.synchronize()


def _finish(job: _Job, now: float, admitted: float) -> Result:
    img = job.ctx.resolve() if job.keep_image else None
    job.ctx.close()
    rc = job.req.rc
    return Result(job.req.rid, job.req.arrival, admitted, now, job.done, img, job.latencies,
                  rc.width * rc.height * job.done)


def run_served(requests, budget_bytes: float, max_jobs: int = 64, keep_images: bool = False):
    """Continuous batching.  Returns (results, rounds, rejected): the finished
    jobs, (start, duration, resident jobs) of every round, and the ids of
    requests larger than the whole budget.  Arrival times are seconds after
    the call starts."""
    pending = sorted(requests, key=lambda r: r.arrival)
    rejected = []
    resident: list[tuple[_Job, float, int]] = []   # job, admission time, predicted bytes
    used = 0
    results, rounds = [], []
    t0 = time.perf_counter()
    while pending or resident:
        now = time.perf_counter() - t0
        if not resident and pending and pending[0].arrival > now:
            time.sleep(pending[0].arrival - now)                      # idle until the next arrival
        r_start = time.perf_counter()
        now = r_start - t0
        while pending and pending[0].arrival <= now and len(resident) < max_jobs:
            b = job_bytes(pending[0])
            if b > budget_bytes:
                rejected.append(pending.pop(0).rid)                    # never fits
                continue
            if used + b > budget_bytes:
                break                                                  # wait for memory to free up
            req = pending.pop(0)
            resident.append((_Job(req, keep_images), now, b))
            used += b
        if not resident:
            continue
        neb.iterate_batch([j.ctx for j, _, _ in resident], 1)
        _sync()
        r_end = time.perf_counter()
        lat = r_end - r_start
        rounds.append((r_start - t0, lat, len(resident)))
        keep = []
        for job, adm, b in resident:
            job.done += 1
            job.latencies.append(lat)
            if job.done >= job.req.rc.iterations:
                results.append(_finish(job, r_end - t0, adm))
                used -= b
            else:
                keep.append((job, adm, b))
        resident = keep
    return results, rounds, rejected


def run_sequential(requests, keep_images: bool = False):
    """The comparison schedule: one job at a time in arrival order, each run to
    its target with its iterations timed one by one."""
    results = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        adm = time.perf_counter() - t0
        job = _Job(req, keep_images)
        for _ in range(req.rc.iterations):
            a = time.perf_counter()
            job.ctx.iterate(1)
            _sync()
            job.latencies.append(time.perf_counter() - a)
            job.done += 1
        results.append(_finish(job, time.perf_counter() - t0, adm))
    return results


def poisson_requests(jobs, rate_per_s: float, seed: int = 0, min_iters: int = 16, max_iters: int = 256):
    """Requests for [(scene, rc)] with exponential inter-arrival times of mean
    1/rate and targets log-uniform in [min_iters, max_iters] iterations."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i, (s, rc) in enumerate(jobs):
        t += rng.exponential(1.0 / rate_per_s)
        rc.iterations = int(round(min_iters * (max_iters / min_iters) ** rng.uniform()))
        out.append(Request(s, rc, t, i))
    return out


def summary(results, wall_s: float):
    """Per-iteration latency percentiles (every iteration of every job),
    time-to-target statistics and aggregate throughput of a schedule."""
    lat = np.array([x for r in results for x in r.iter_latencies])
    ttt = np.array([r.time_to_target for r in results])
    paths = sum(r.paths for r in results)
    return {"jobs": len(results),
            "iteration_latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                     "p99": 1e3 * float(np.percentile(lat, 99))},
            "time_to_target_s": {"mean": float(ttt.mean()), "p50": float(np.percentile(ttt, 50)),
                                 "p99": float(np.percentile(ttt, 99))},
            "wall_s": wall_s, "paths": paths, "mpaths_per_s": paths / wall_s / 1e6}
