"""Served progressive rendering (continuous batching): a job's image is the
same alone and in the mix, whenever it is admitted."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1909_00573_gb300 import build
    build.build()
    from paper_1909_00573_gb300 import neb, scenes, serve
    return neb, scenes, serve


def test_served_images_equal_solo_runs(mods):
    neb, scenes, serve = mods
    room = scenes.tiny_room()
    city = scenes.large_city(seed=5, grid=10, n_lights=3)
    specs = [(room, 64, 48, 4, 0.0), (city, 96, 96, 6, 0.0), (room, 80, 64, 3, 0.05), (city, 64, 64, 5, 0.08)]
    reqs = []
    for i, (s, w, h, iters, t) in enumerate(specs):
        r = 0.01 if s is room else 2e-3
        rc = scenes.RenderConfig(w, h, 8, r, 1 << 16, 4, iters, seed=100 + i, octree_mode=1)
        reqs.append(serve.Request(s, rc, t, i))
    results, rounds, rejected = serve.run_served(reqs, budget_bytes=8e9, max_jobs=3, keep_images=True)
    assert not rejected and len(results) == len(reqs)
    assert max(n for _, _, n in rounds) <= 3
    assert len({r.admitted for r in results}) > 1          # admitted at different rounds
    for res in results:
        req = reqs[res.rid]
        ctx = neb.Context(neb.make_config(req.rc))
        ctx.scene_upload(req.scene)
        ctx.build_bvh()
        ctx.iterate(req.rc.iterations)
        solo = ctx.resolve()
        ctx.close()
        assert res.iterations == req.rc.iterations
        np.testing.assert_allclose(res.image, solo, rtol=1e-5, atol=1e-7 * float(np.abs(solo).max()))
        assert solo.sum() > 0
    s = serve.summary(results, max(r.finished for r in results))
    assert s["jobs"] == 4 and s["iteration_latency_ms"]["p99"] >= s["iteration_latency_ms"]["p50"] > 0
