"""Host logic of the multi-GPU path (replicas only: each GPU renders its own
sample stream, no data-path collective) with two gloo ranks on the CPU:
per-rank seeds, the max-over-ranks job time and the whole-job throughput."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.replica_seed(rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        t = bench.max_over_ranks(times[rank], dist, "cpu")
        v = bench.job_value(world, 921600, 8, t)
        q.put((rank, seeds, t, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    times = [0.25, 0.40]
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(2):
        rank, seeds, t, v = q.get(timeout=120)
        out[rank] = (seeds, t, v)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(2):
        seeds, t, v = out[rank]
        assert seeds == [0, 1]                      # independent sample streams
        assert t == pytest.approx(0.40)             # every rank sees the slowest rank's time
        assert v == pytest.approx(2 * 921600 * 8 / 0.40 / 1e6)


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.job_value(1, 100, 10, 2.0) == pytest.approx(100 * 10 / 2.0 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the oracle arm is timed once: ranks other than 0 exit 0
    without work and print nothing."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 2, "warmup": 1, "gpus": 2, "workload": "large_city"})()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_secondary_rates_and_traffic_lookup(monkeypatch):
    """Rates are whole-job counts per second; stored ncu counters are used
    only for their workload and stage, and only while the traversal sources
    hash to those they were captured from."""
    import bench
    d = {"camera_rays": 4e6, "shadow_rays": 3e6, "photon_hits": 1e6, "merge_tests": 2e6, "merges": 5e4,
         "octree_inserts": 3e6, "octree_queries": 1e5}
    r = bench.rates(d, 2, 1000.0)                      # two ranks, one second
    assert r["Mrays_per_s"] == 16.0 and r["Mmerges_per_s"] == 0.1 and r["Moctree_inserts_per_s"] == 6.0
    assert bench.rates(d, 1, 0.0) is None
    key = ("many_lights", "trace_camera")
    entry = {"bound": "issue", "bytes_per_launch": 1.0e8, "lane_efficiency": 0.4, "issue_active": 0.6,
             "profile": "profiles/x.md", "sources_sha256": bench.sources_sha256()}
    monkeypatch.setitem(bench.NCU_COUNTERS, key, entry)
    assert bench.measured_counters("many_lights", "trace_camera") == entry
    assert bench.measured_counters("tiny_room", "trace_camera") is None
    assert bench.measured_counters("many_lights", "shadow") is None
    monkeypatch.setitem(bench.NCU_COUNTERS, key, dict(entry, sources_sha256="0" * 64))
    assert bench.measured_counters("many_lights", "trace_camera") is None


def test_batch_admission_waves():
    """The batched-jobs benchmark runs every job: jobs go in order into waves
    whose summed device bytes fit the budget, a job that does not fit starts
    the next wave, and only a job larger than the budget alone is rejected."""
    import bench
    waves, rejected = bench.admission_waves([40, 50, 20, 70, 10, 120, 30], 100)
    assert rejected == 1                                   # the 120-byte job
    assert waves == [[0, 1], [2, 3, 4], [6]]
    assert all(sum([40, 50, 20, 70, 10, 120, 30][i] for i in w) <= 100 for w in waves)
    assert bench.admission_waves([], 100) == ([], 0)
    assert bench.admission_waves([100, 100], 100) == ([[0], [1]], 0)   # a wave may be exactly full
