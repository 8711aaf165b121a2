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


def test_error_estimate_matches_the_true_error_on_the_plane(mods):
    """Random hits and NEE (unbiased) on the diffuse plane under a sphere
    light, whose pixel values are known in closed form: the two-half
    estimate of the relative RMSE agrees with the true relative RMSE of the
    image, and falls as 1 / sqrt(iterations)."""
    neb, scenes, serve = mods
    from test_oracle_closed_forms import _plane_expectation
    a, R, h, L = 0.6, 0.1, 1.0, 5.0
    s = scenes.plane_under_sphere(a, R, h, L)
    W = H = 48
    expect = 3.0 * _plane_expectation(s, W, H, a, R, h, L)
    est = {}
    for n in (8, 32):
        rc = scenes.RenderConfig(W, H, 3, 0.01, 1 << 16, 4, n, seed=7, strategy_mask=3)
        ctx = neb.render(s, rc, n_iter=n)
        img = ctx.resolve().reshape(H, W, 3).sum(-1)
        est[n] = ctx.error_estimate()
        ctx.close()
        true = float(np.sqrt(np.sum((img - expect) ** 2) / np.sum(expect ** 2)))
        assert 0.75 < est[n] / true < 1.33, (n, est[n], true)
    assert 1.6 < est[8] / est[32] < 2.5, est
    ctx = neb.render(s, scenes.RenderConfig(W, H, 3, 0.01, 1 << 16, 4, 1, seed=7, strategy_mask=3), n_iter=1)
    with pytest.raises(neb.NebError):
        ctx.error_estimate()                       # one iteration: no second half yet
    ctx.close()


def test_served_jobs_retire_at_their_rmse_target(mods):
    """Requests that ask for a relative RMSE: each job stops at the first
    check (every 4 iterations from 16) where its estimate meets the target,
    or at the cap, and its image equals a solo run of as many iterations."""
    neb, scenes, serve = mods
    room = scenes.tiny_room()
    city = scenes.large_city(seed=5, grid=10, n_lights=3)
    specs = [(room, 48, 48, 0.0, 0.6), (city, 64, 64, 0.0, 1.2), (room, 64, 48, 0.02, 3.0)]
    reqs = []
    for i, (s, w, h, t, f) in enumerate(specs):
        r = 0.01 if s is room else 2e-3
        rc = scenes.RenderConfig(w, h, 8, r, 1 << 16, 4, 0, seed=200 + i, octree_mode=1)
        target = f * serve.pilot_rmse(s, rc, side=48) / np.sqrt(32.0)
        reqs.append(serve.Request(s, rc, t, i, target))
    results, rounds, rejected = serve.run_served(reqs, budget_bytes=8e9, max_jobs=2, keep_images=True,
                                                 min_iters=16, max_iters=64, check_every=4)
    assert not rejected and len(results) == len(reqs)
    for res in results:
        req = reqs[res.rid]
        assert 16 <= res.iterations <= 64 and (res.iterations - 16) % 4 == 0
        assert res.reached == (res.rmse <= req.target_rmse)
        assert res.reached or res.iterations == 64
        ctx = neb.render(req.scene, req.rc, n_iter=res.iterations)
        solo = ctx.resolve()
        # the same samples; per-cell merge sums round differently from run to run
        assert ctx.error_estimate() == pytest.approx(res.rmse, rel=1e-5)
        ctx.close()
        np.testing.assert_allclose(res.image, solo, rtol=1e-5, atol=1e-7 * float(np.abs(solo).max()))
    its = sorted(r.iterations for r in results)
    assert its[0] < its[-1]                      # the targets ask for different amounts of work
