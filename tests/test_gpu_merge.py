"""The per-cell photon merge (merge mode 2: every hit staged; mode 0, the
default: hits with many view vertices around them staged, the others merged
per hit) against the per-hit merge (mode 1) on the GPU.

All modes find the pairs (photon hit, view vertex) within r with the same
FP32 distance test and compute each pair's term the same way, so with the
deterministic octree they give the same number of merges and the same
per-strategy sums up to the FP32 rounding of the per-cell partial sums
(Sec. 3.2).  The cases cover the paths through the per-cell merge: one cell
per bucket, cells that share a bucket of the photon table (a small staging
list has a small table), buckets of more than one tile (a large radius), a
staging list too small for the iteration (the rest merges per hit), light
photons (Sec. 6.1, their own channel and first-hit weights), and the
default mode on a dense image (most hits staged) and a sparse one (few)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def neb():
    from paper_1909_00573_gb300 import build
    build.build()
    from paper_1909_00573_gb300 import neb as N
    return N


# name: (width, height, merge radius, staging capacity (0: default), light photons, mode against mode 1)
CASES = {
    "cell_per_bucket": (64, 64, 0.01, 0, 0, 2),
    "shared_buckets": (48, 48, 0.01, 30000, 0, 2),
    "tiles_per_bucket": (128, 128, 0.05, 0, 0, 2),
    "list_full": (64, 64, 0.01, 2000, 0, 2),
    "light_photons": (64, 64, 0.01, 0, 4096, 2),
    "default_dense": (256, 256, 0.01, 0, 0, 0),
    "default_sparse": (64, 64, 0.01, 0, 0, 0),
}


def _run(neb, name, merge_mode):
    from paper_1909_00573_gb300 import scenes
    w, h, r, cap, lp, _ = CASES[name]
    s = scenes.tiny_room()
    rc = scenes.RenderConfig(w, h, 8, r, 1 << 16, 8, 3, seed=3, octree_mode=1)
    if lp:
        rc.strategy_mask |= 8
        rc.lp_photons = lp
    ctx = neb.Context(neb.make_config(rc, keep_split=True, merge_mode=merge_mode, merge_hits=cap))
    ctx.scene_upload(s)
    ctx.build_bvh()
    ctx.iterate(rc.iterations)
    out = (ctx.read_split(), ctx.read_accum(), ctx.stats(), ctx.read_nee_rho())
    ctx.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_per_cell_merge_equals_per_hit_merge(neb, name):
    mode = CASES[name][5]
    sp0, a0, st0, r0 = _run(neb, name, mode)
    sp1, a1, st1, r1 = _run(neb, name, 1)
    assert np.array_equal(r0, r1)
    for key in ("photons", "photon_hits", "merges", "nee_vertices"):
        assert st0[key] == st1[key], key
    assert st0["merges"] > 0 and st1["merge_hits_staged"] == 0
    staged = st0["merge_hits_staged"]
    cap = CASES[name][3]
    if cap:
        assert 0 < staged <= 3 * cap                       # at most cap staged per iteration
    if name == "list_full":
        assert staged == 3 * cap                           # the rest merged per hit
    elif name.startswith("default"):
        assert staged < st0["photon_hits"]
    else:
        assert staged > 3 * 2000
    # per strategy: random hits and NEE do not merge; the merge channels
    # (2: NEB photons, 3: light photons) agree to the FP32 partial sums
    for k in range(4):
        ref = sp1[k]
        np.testing.assert_allclose(sp0[k], ref, rtol=2e-5, atol=1e-7 * max(float(np.abs(ref).max()), 1e-30))
    assert float(np.abs(sp1[2]).sum()) > 0
    if CASES[name][4]:
        assert float(np.abs(sp1[3]).sum()) > 0
    np.testing.assert_allclose(a0, a1, rtol=2e-5, atol=1e-7 * float(np.abs(a1).max()))


def test_default_mode_stages_the_dense_hits(neb):
    """Merge mode 0 stages a hit when more than 16 view vertices lie in its
    grid cells: with 16 times the pixels of the same room most hits are
    staged, a larger share than at the smaller size."""
    frac = {}
    for name in ("default_sparse", "default_dense"):
        st = _run(neb, name, 0)[2]
        frac[name] = st["merge_hits_staged"] / st["photon_hits"]
    assert frac["default_dense"] > 0.5 and frac["default_dense"] > frac["default_sparse"], frac
