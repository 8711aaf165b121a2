"""Batched jobs (neb_iterate_batch) and admission (neb_job_device_bytes) on
the GPU: every job's result is the same alone and in the batch, and the
device-memory estimate matches what a job allocates."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def neb():
    from paper_1909_00573_gb300 import build
    build.build()
    from paper_1909_00573_gb300 import neb as N
    return N


def _jobs():
    from paper_1909_00573_gb300 import scenes
    room = scenes.tiny_room()
    out = [(room, scenes.RenderConfig(96, 80, 8, 0.01, 1 << 16, 8, 3, seed=11, octree_mode=1))]
    for i, (g, nl, side) in enumerate([(12, 3, 128), (20, 9, 144)]):
        s = scenes.large_city(seed=i + 3, grid=g, n_lights=nl)
        out.append((s, scenes.RenderConfig(side, side, 10, 2e-3, 1 << 18, 4, 3, seed=20 + i, octree_mode=1)))
    return out


def _start(neb, s, rc, merge_mode=0):
    ctx = neb.Context(neb.make_config(rc, merge_mode=merge_mode))
    ctx.scene_upload(s)
    ctx.build_bvh()
    return ctx


def _close(a, b, merge_mode):
    # per-cell merge (modes 0 and 2): FP32 partial sums per view vertex and
    # tile, in an order that varies from run to run; per-hit merge (mode 1):
    # FP64 order only
    rtol, atol = (1e-12, 1e-12) if merge_mode == 1 else (1e-5, 1e-7)
    np.testing.assert_allclose(a, b, rtol=rtol, atol=atol * float(np.abs(b).max()))


@pytest.mark.parametrize("merge_mode", [1, 2])
def test_batch_results_equal_alone(neb, merge_mode):
    """Three heterogeneous jobs (a room and two cities of different sizes,
    resolutions, light counts and seeds), deterministic octree: each job's
    densities are bit-identical and its FP64 sums equal up to the order of the
    additions whether it runs alone or round-robin with the others."""
    jobs = _jobs()
    alone = []
    for s, rc in jobs:
        ctx = _start(neb, s, rc, merge_mode)
        ctx.iterate(rc.iterations)
        alone.append((ctx.read_nee_rho(), ctx.read_accum(), ctx.stats()))
        ctx.close()
    ctxs = [_start(neb, s, rc, merge_mode) for s, rc in jobs]
    neb.iterate_batch(ctxs, jobs[0][1].iterations)
    for ctx, (rho, acc, st) in zip(ctxs, alone):
        r2, a2, st2 = ctx.read_nee_rho(), ctx.read_accum(), ctx.stats()
        assert np.array_equal(rho, r2)
        _close(a2, acc, merge_mode)
        keys = ["iterations", "camera_rays", "nee_vertices", "shadow_rays", "photons", "merges", "octree_inserts",
                "octree_nodes", "merge_hits_staged"]
        for key in keys + (["merge_tests"] if merge_mode == 1 else []):
            assert st2[key] == st[key], key
        assert acc.sum() > 0
        ctx.close()


def test_job_device_bytes_matches_allocation(neb):
    """neb_job_device_bytes predicts the device memory a job holds after
    neb_create, neb_scene_upload and neb_build_bvh."""
    torch = pytest.importorskip("torch")
    from paper_1909_00573_gb300 import scenes
    s, rc = scenes.workload("large_city")
    rc.width, rc.height = 640, 360
    cfg = neb.make_config(rc)
    expect = neb.job_device_bytes(cfg, s.n_tri, s.n_sph, len(s.mats), s.n_emitters)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx = neb.Context(cfg)
    ctx.scene_upload(s)
    ctx.build_bvh()
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    ctx.close()
    assert abs(used - expect) <= 0.05 * expect + (64 << 20), (used, expect)


def test_tuning_changes_no_result(neb):
    """Launch settings (grouping resolutions, shading grid) leave every result
    unchanged (deterministic octree: densities identical, FP64 sums equal up to
    the order of the additions); invalid settings are rejected; the
    autotuner returns valid settings after running real iterations."""
    from paper_1909_00573_gb300 import scenes
    s, rc = scenes.workload("tiny_room")
    rc.octree_mode = 1
    out = []
    for t in (None, neb.Tuning(0, 4, 1, 1, 3)):
        ctx = _start(neb, s, rc)
        if t is not None:
            ctx.set_tuning(t)
            assert ctx.tuning().as_dict() == t.as_dict()
        ctx.iterate(3)
        out.append((ctx.read_nee_rho(), ctx.read_accum()))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0])
    _close(out[1][1], out[0][1], 0)
    ctx = _start(neb, s, rc)
    for bad in (neb.Tuning(5, 0, 2, 2, 8), neb.Tuning(2, 3, 2, 2, 8), neb.Tuning(1, 3, 2, 2, 0)):
        with pytest.raises(neb.NebError):
            ctx.set_tuning(bad)
    t = ctx.autotune(1)
    assert ctx.stats()["iterations"] == 5 + 4 + 3          # one iteration per candidate
    assert ctx.tuning().as_dict() == t.as_dict()
    assert 3 * (t.cam_origin_bits + t.cam_dir_bits) <= 12 and 1 <= t.shade_blocks_per_sm <= 32
    ctx.close()


def test_photon_regrouping_changes_no_result(neb):
    """Photon rays regrouped before each walk (a launch setting, on where the
    photon queue holds at least 2^20 rays): the same photons, hits and merges
    as without, and the FP64 sums equal up to the order of the additions
    (every hit merged on its own).  A 400 x 400 room: 1.12 M photon slots."""
    from paper_1909_00573_gb300 import scenes
    s = scenes.tiny_room()
    rc = scenes.RenderConfig(400, 400, 8, 0.01, 1 << 20, 8, 2, seed=5, octree_mode=1)
    out = []
    for grouping in (1, 0):
        ctx = _start(neb, s, rc, merge_mode=1)
        t = ctx.tuning()
        assert t.photon_grouping == 1                     # on by default
        t.photon_grouping = grouping
        ctx.set_tuning(t)
        ctx.iterate(rc.iterations)
        out.append((ctx.read_nee_rho(), ctx.read_accum(), ctx.stats()))
        ctx.close()
    (r1, a1, st1), (r0, a0, st0) = out
    assert np.array_equal(r1, r0)
    for key in ("photons", "photon_hits", "merges", "merge_tests", "camera_rays"):
        assert st1[key] == st0[key], key
    assert st1["kernel_launches"] > st0["kernel_launches"]   # the regrouping launches ran
    _close(a1, a0, 1)
    assert a0.sum() > 0

