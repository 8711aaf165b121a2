"""Pins of the oracle's building blocks against things other than itself:
published known-answer vectors, exact geometry computed a different way,
brute force, textbook formulas and hand-worked examples."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10 (random numbers, keyed by (iteration, pixel, bounce, dim))
# --------------------------------------------------------------------------
def load_kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle):
    for ctr, key, out in load_kat():
        assert oracle.philox4x32_10(ctr, key).tolist() == out


# --------------------------------------------------------------------------
# plane/box intersection area (Eq. area, Sec. 5.3 and Appendix A)
# --------------------------------------------------------------------------
def exact_area(bmin, bmax, p, n):
    """Area of {x in box : n.x = n.p} by clipping: plane/edge crossings,
    ordered by angle around their centroid, then the 3D shoelace formula."""
    bmin = np.asarray(bmin, np.float64)
    bmax = np.asarray(bmax, np.float64)
    n = np.asarray(n, np.float64)
    n = n / np.linalg.norm(n)
    h = float(n @ np.asarray(p, np.float64))
    corners = np.array([[bmax[0] if i & 1 else bmin[0], bmax[1] if i & 2 else bmin[1],
                         bmax[2] if i & 4 else bmin[2]] for i in range(8)])
    pts = []
    for i in range(8):
        for bit in (1, 2, 4):
            j = i | bit
            if j == i:
                continue
            a, b = corners[i], corners[j]
            da, db = a @ n - h, b @ n - h
            if da == 0.0:
                pts.append(a)
            if db == 0.0:
                pts.append(b)
            if da * db < 0:
                t = da / (da - db)
                pts.append(a + t * (b - a))
    if len(pts) < 3:
        return 0.0
    P = np.unique(np.round(np.array(pts), 14), axis=0)
    if len(P) < 3:
        return 0.0
    c = P.mean(0)
    u = np.cross(n, [1.0, 0, 0]) if abs(n[0]) < 0.9 else np.cross(n, [0, 1.0, 0])
    u /= np.linalg.norm(u)
    w = np.cross(n, u)
    ang = np.arctan2((P - c) @ w, (P - c) @ u)
    P = P[np.argsort(ang)]
    s = np.zeros(3)
    for i in range(len(P)):
        s += np.cross(P[i], P[(i + 1) % len(P)])
    return 0.5 * abs(s @ n)


def test_area_closed_forms(oracle):
    unit = ([0, 0, 0], [1, 1, 1])
    # axis-aligned planes cut a face-sized rectangle
    assert oracle.intersection_area(*unit, [0.3, 0.4, 0.5], [0, 0, 1]) == pytest.approx(1.0, rel=1e-12)
    assert oracle.intersection_area([0, 0, 0], [2, 3, 5], [1, 1, 1], [1, 0, 0]) == pytest.approx(15.0, rel=1e-12)
    # plane x + y = 1 (one zero component) cuts a sqrt(2) x 1 rectangle
    n = np.array([1, 1, 0]) / math.sqrt(2)
    assert oracle.intersection_area(*unit, [0.5, 0.5, 0.5], n) == pytest.approx(math.sqrt(2), rel=1e-6)
    # plane through the cube centre with normal (1,1,1)/sqrt(3): regular hexagon of side sqrt(2)/2
    n = np.ones(3) / math.sqrt(3)
    hexagon = 3 * math.sqrt(3) / 2 * 0.5
    assert oracle.intersection_area(*unit, [0.5, 0.5, 0.5], n) == pytest.approx(hexagon, rel=1e-6)
    # corner triangle: plane x+y+z = 0.5 cuts a triangle with legs 0.5
    tri = math.sqrt(3) / 4 * (0.5 * math.sqrt(2)) ** 2
    assert oracle.intersection_area(*unit, [0.5, 0, 0], n) == pytest.approx(tri, rel=1e-6)
    # plane beyond the box: the alternating sum of eight squares cancels to 0
    # (in FP32 it would leave a few 1e-6, the precision issue Sec. 5.3 notes)
    assert oracle.intersection_area(*unit, [2.0, 2.0, 2.0], n) == pytest.approx(0.0, abs=1e-12)


def test_area_matches_polygon_clipping(oracle):
    rng = np.random.default_rng(1)
    errs = []
    for _ in range(3000):
        bmin = rng.uniform(-2, 2, 3).astype(np.float32)
        bmax = (bmin + rng.uniform(0.1, 2.0, 3)).astype(np.float32)
        p = (bmin + rng.uniform(0, 1, 3) * (bmax - bmin)).astype(np.float32)
        while True:
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            if np.all(np.abs(n) > 0.05):
                break
        n = n.astype(np.float32)
        a = oracle.intersection_area(bmin, bmax, p, n)
        e = exact_area(bmin, bmax, p, n)
        scale = max(e, 1e-3 * float(np.prod(bmax - bmin)) ** (2 / 3))
        errs.append(abs(a - e) / scale)
    # FP64 evaluation; what remains is the FP32 normal's length, 1 +- 2e-7
    assert max(errs) < 1e-6, max(errs)


def test_area_is_unchanged_by_mirroring_the_axes(oracle):
    """Mirroring an axis (box, point and normal together) leaves the
    intersection unchanged; in Eq. area it flips the parity sign of every
    corner and the sign of the product of the normal's components at once."""
    rng = np.random.default_rng(8)
    for _ in range(500):
        lo = rng.uniform(-1, 1, 3)
        hi = lo + rng.uniform(0.1, 1.0, 3)
        p = lo + rng.uniform(0, 1, 3) * (hi - lo)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        a0 = oracle.intersection_area(lo.astype(np.float32), hi.astype(np.float32), p.astype(np.float32),
                                      n.astype(np.float32))
        f = np.where(rng.uniform(size=3) < 0.5, -1.0, 1.0)
        lo2, hi2 = np.minimum(lo * f, hi * f), np.maximum(lo * f, hi * f)
        a1 = oracle.intersection_area(lo2.astype(np.float32), hi2.astype(np.float32), (p * f).astype(np.float32),
                                      (n * f).astype(np.float32))
        assert a1 == pytest.approx(a0, rel=1e-9, abs=1e-12)


def test_area_near_the_implementation_thresholds_is_bounded(oracle):
    """The paper's implementation switches to the 1D / 2D formulas when a component is within
    1e-3 of 1 or below 1e-4; the error there stays small (documented reading)."""
    rng = np.random.default_rng(2)
    for _ in range(500):
        bmin = np.zeros(3, np.float32)
        bmax = rng.uniform(0.5, 1.5, 3).astype(np.float32)
        p = (rng.uniform(0.2, 0.8, 3) * bmax).astype(np.float32)
        eps = rng.uniform(0, 2e-3)
        n = np.array([math.sqrt(max(0.0, 1 - eps * eps)), eps * 0.6, eps * 0.8], np.float64)
        n = rng.permutation(n).astype(np.float32)
        a = oracle.intersection_area(bmin, bmax, p, n)
        e = exact_area(bmin, bmax, p, n)
        assert abs(a - e) <= 5e-3 * e + 1e-6


# --------------------------------------------------------------------------
# density octree (Sec. 5, Appendix B)
# --------------------------------------------------------------------------
def test_octree_capacity_rounding_and_root(oracle):
    o = oracle.Octree([0, 0, 0], [1, 1, 1], 10, 4)
    nodes, alloc, depth = o.dump()
    assert len(nodes) == 17          # 1 + round_up(10, 8)
    assert alloc == 1 and depth == 0 and nodes[0] == 0


def test_octree_split_hand_worked(oracle):
    """split factor 8, iteration 1: threshold 8, children start at ceil(8/4 * 1) = 2."""
    o = oracle.Octree([0, 0, 0], [1, 1, 1], 64, 8)
    o.set_iteration(1)
    nodes, alloc, depth = o.dump()
    assert alloc == 1 and np.all(nodes[1:] == 2)
    p = [0.2, 0.2, 0.2]                      # lower octant 0 at every level
    o.insert([p] * 7)
    nodes, alloc, depth = o.dump()
    assert nodes[0] == 7 and alloc == 1
    o.insert([p])                            # 8th vertex reaches the threshold: split
    nodes, alloc, depth = o.dump()
    assert nodes[0] == -1 and alloc == 9 and depth == 1
    assert np.all(nodes[1:9] == 2)           # children untouched by the splitting insert
    o.insert([p])                            # descends into child 0 (octant of p)
    nodes, alloc, depth = o.dump()
    assert nodes[1] == 3 and np.all(nodes[2:9] == 2)
    q = [0.8, 0.2, 0.8]                      # octant x=1, y=0, z=1 -> index 1 + 4 = 5
    o.insert([q])
    nodes, _, _ = o.dump()
    assert nodes[1 + 5] == 3
    # iteration 2: threshold 16, unused nodes re-armed to ceil(8/4*2) = 4
    o.set_iteration(2)
    nodes, alloc, _ = o.dump()
    assert alloc == 9 and np.all(nodes[9:] == 4) and nodes[1] == 3


def test_octree_allocation_overflow(oracle):
    o = oracle.Octree([0, 0, 0], [1, 1, 1], 8, 4)   # capacity 9: one split only
    o.set_iteration(1)
    o.insert([[0.1, 0.1, 0.1]] * 4)                  # root split
    nodes, alloc, depth = o.dump()
    assert nodes[0] == -1 and alloc == 9 and depth == 1
    o.insert([[0.1, 0.1, 0.1]] * 3)                  # child 0: 1 + 3 = 4 -> split wanted, overflow
    nodes, alloc, depth = o.dump()
    assert nodes[1] == 4 and alloc == 10 and depth == 1
    # a vertex is counted before a split is tried, so the full leaf keeps
    # counting; no further allocation is attempted
    o.insert([[0.1, 0.1, 0.1]] * 5)
    nodes2, alloc2, _ = o.dump()
    assert nodes2[1] == 9 and np.array_equal(nodes[2:], nodes2[2:]) and alloc2 == 10


def test_octree_out_of_box_is_dropped(oracle):
    o = oracle.Octree([0, 0, 0], [1, 1, 1], 64, 4)
    o.set_iteration(1)
    o.insert([[1.5, 0.5, 0.5], [-0.5, 0.5, 0.5]])
    nodes, alloc, _ = o.dump()
    assert nodes[0] == 0
    assert o.density([[1.5, 0.5, 0.5]], [[0, 1, 0]], robust=False)[0] == 0.0


def _descend(nodes, mn, size, q):
    """Brute-force walk of the node array using only the encoding of Sec. 5.5:
    a negative value is the negated index of the first of eight children."""
    lo = np.zeros(3)
    hi = np.ones(3)
    nq = (np.asarray(q, np.float64) - mn) / size
    idx = 0
    while nodes[idx] < 0:
        base = -int(nodes[idx])
        mid = 0.5 * (lo + hi)
        bits = (nq >= mid).astype(int)
        idx = base + bits[0] + 2 * bits[1] + 4 * bits[2]
        lo = np.where(bits, mid, lo)
        hi = np.where(bits, hi, mid)
    return int(nodes[idx]), mn + lo * size, mn + hi * size, hi[0] - lo[0]


def test_octree_density_matches_descent_and_exact_area(oracle):
    rng = np.random.default_rng(3)
    smin = np.array([0, 0, 0], np.float32)
    smax = np.array([1, 1, 1], np.float32)
    o = oracle.Octree(smin, smax, 1 << 14, 4)
    o.set_iteration(1)
    # points on a tilted plane through the box
    n = np.array([0.3, 0.8, 0.52])
    n /= np.linalg.norm(n)
    pts = []
    while len(pts) < 4000:
        x = rng.uniform(0, 1, 3)
        x = x - ((x - 0.5) @ n) * n
        if np.all((x > 0) & (x < 1)):
            pts.append(x)
    pts = np.array(pts, np.float32)
    o.insert(pts)
    nodes, alloc, depth = o.dump()
    # the octree box: the scene box grown by 0.2 % about its centre (Appendix B)
    size = ((smax - smin) * np.float32(1.002)).astype(np.float32)
    mn = (smin - size * np.float32(0.001 / 1.002)).astype(np.float32)
    scale = float(np.sqrt(np.sum(size.astype(np.float64) ** 2)))
    q = pts[:400]
    rho = o.density(q, np.tile(n.astype(np.float32), (len(q), 1)), robust=False)
    checked = 0
    for i in range(len(q)):
        c, lo, hi, frac = _descend(nodes, mn.astype(np.float64), size.astype(np.float64), q[i])
        res = round(1.0 / frac)
        # skip points within float noise of a cell face
        nq = (q[i].astype(np.float64) - mn) / size * res
        if np.min(np.abs(nq - np.round(nq))) < 1e-4:
            continue
        area = exact_area(lo, hi, q[i], n)
        diag = scale / res
        expect = 0.0 if c <= 0 else c / max(0.01 * diag * diag, area)
        assert rho[i] == pytest.approx(expect, rel=1e-5), (i, c, area)
        checked += 1
    assert checked > 300


def test_octree_density_of_uniform_plane(oracle):
    """N vertices spread uniformly over a unit square give rho ~ N per unit area."""
    rng = np.random.default_rng(4)
    o = oracle.Octree([0, 0, 0], [1, 1, 1], 1 << 16, 4)
    N = 20000
    o.set_iteration(1)
    pts = np.stack([rng.uniform(0, 1, N), np.full(N, 0.37), rng.uniform(0, 1, N)], 1).astype(np.float32)
    o.insert(pts)
    q = np.stack([rng.uniform(0.05, 0.95, 2000), np.full(2000, 0.37), rng.uniform(0.05, 0.95, 2000)], 1)
    rho = o.density(q, np.tile([0, 1, 0], (2000, 1)), robust=True)
    # the estimate is biased by the child initialisation guess (Sec. 5.2) and
    # the leaf counts are small; the mean must still land close to N
    assert 0.7 * N < float(np.mean(rho)) < 1.3 * N


def _uniform_level3_tree(counts):
    """Flat layout (Sec. 5.5) of a tree split uniformly down to level 3
    (8 x 8 x 8 leaves), built by hand: words 1-8 the children of the root,
    9-72 level 2, 73-584 level 3.  counts maps leaf cell (x, y, z) to its
    count (0 elsewhere).  Returns the words and the word of every leaf."""
    words = np.zeros(585, np.int32)
    leaf_word = {}
    words[0] = -1
    for o1 in range(8):
        w1 = 1 + o1
        words[w1] = -(9 + 8 * o1)
        for o2 in range(8):
            w2 = 9 + 8 * o1 + o2
            words[w2] = -(73 + 8 * (8 * o1 + o2))
            for o3 in range(8):
                w3 = 73 + 8 * (8 * o1 + o2) + o3
                cell = tuple(((o1 >> a) & 1) * 4 + ((o2 >> a) & 1) * 2 + ((o3 >> a) & 1) for a in range(3))
                leaf_word[cell] = w3
                words[w3] = counts.get(cell, 0)
    return words, leaf_word


@pytest.mark.parametrize("case", ["odd", "even", "tie", "centre_empty", "none"])
def test_octree_robust_median_hand_worked(oracle, case):
    """Robust density at the centre of leaf (3, 3, 3) of a hand-built level-3
    tree over the unit box (octree box 1.002 wide), normal +z: the tangents
    are +-x and +-y, the step 1.1 level-3 diagonals (1.9 cell widths), so the
    four displaced queries land in leaves (5,3,3), (1,3,3), (3,5,3), (3,1,3).
    Every leaf has the same area (the face, 1D case), so each density is its
    count over that area.  The result is the median of the positive ones,
    the upper of the middle two for an even number; with the centre cell
    empty the step is 1.1e-3 and all five queries stay in that cell."""
    c0, px, mx, py, my = {"odd": (10, 4, 7, 9, 3), "even": (10, 4, 9, 3, 0), "tie": (6, 6, 2, 0, 8),
                          "centre_empty": (0, 5, 5, 5, 5), "none": (0, 0, 0, 0, 0)}[case]
    counts = {(3, 3, 3): c0, (5, 3, 3): px, (1, 3, 3): mx, (3, 5, 3): py, (3, 1, 3): my}
    words, _ = _uniform_level3_tree(counts)
    o = oracle.Octree([0, 0, 0], [1, 1, 1], 584, 4)
    o.set_iteration(1)
    o.load(words, 585, 3)
    edge = 1.002 / 8
    p = np.float32(-0.001) + np.float32(3.5 * edge)
    rho = o.density([[p, p, p]], [[0, 0, 1]], robust=True)[0]
    positive = sorted(c for c in (c0, px, mx, py, my) if c > 0)
    expect_count = {"odd": 7, "even": 9, "tie": 6, "centre_empty": 0, "none": 0}[case]
    if positive and case != "centre_empty":
        assert positive[len(positive) // 2] == expect_count
    assert rho == pytest.approx(expect_count / (edge * edge), rel=1e-5)
    # the single query reads the centre cell alone, with the 0.01 floor
    assert o.density([[p, p, p]], [[0, 0, 1]], robust=False)[0] == pytest.approx(c0 / (edge * edge), rel=1e-5)


def test_octree_load_dump_round_trip_and_malformed_layouts(oracle):
    rng = np.random.default_rng(17)
    counts = {tuple(rng.integers(0, 8, 3)): int(rng.integers(1, 50)) for _ in range(40)}
    words, _ = _uniform_level3_tree(counts)
    o = oracle.Octree([0, 0, 0], [1, 1, 1], 584, 4)
    o.set_iteration(1)
    o.load(words, 585, 3)
    nodes, used, depth = o.dump()
    assert np.array_equal(nodes, words) and used == 585 and depth == 3
    bad = words.copy()
    bad[0] = -580                       # children would run past the array
    with pytest.raises(ValueError):
        o.load(bad, 585, 3)
    bad = words.copy()
    bad[1] = -1                         # a cycle back to the root's children
    with pytest.raises(ValueError):
        o.load(bad, 585, 3)


@pytest.mark.parametrize("n", [[0, 0, 1], [0, 0, -1], [0, 0, -0.9999999], [1, 0, 0], [0, -1, 0],
                               [0.6, 0.0, -0.8], [-0.48, 0.6, -0.64]])
def test_duff_basis_is_orthonormal_and_right_handed(oracle, n):
    """The tangents of the robust density query: t, b, n orthonormal with
    t x b = n, also at and near n_z = -1 where the published construction
    switches sign."""
    n = np.asarray(n, np.float64)
    n /= np.linalg.norm(n)
    t, b = oracle.onb(n.astype(np.float32))
    t = t.astype(np.float64)
    b = b.astype(np.float64)
    assert np.linalg.norm(t) == pytest.approx(1.0, abs=1e-6)
    assert np.linalg.norm(b) == pytest.approx(1.0, abs=1e-6)
    assert abs(t @ b) < 1e-6 and abs(t @ n) < 1e-6 and abs(b @ n) < 1e-6
    assert np.allclose(np.cross(t, b), n, atol=2e-6)


def test_duff_basis_random_normals(oracle):
    rng = np.random.default_rng(9)
    for _ in range(2000):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        t, b = oracle.onb(n.astype(np.float32))
        assert np.allclose(np.cross(t.astype(np.float64), b.astype(np.float64)), n, atol=3e-6)
        assert abs(float(t @ b)) < 2e-6


# --------------------------------------------------------------------------
# light selection: Vose's alias table over the light powers
# --------------------------------------------------------------------------
@pytest.mark.parametrize("power", [[1.0, 2.0, 4.0, 8.0, 100.0], [3.0], [1.0, 1.0, 1.0], [1e-3, 1.0, 1e3]])
def test_alias_selection_frequencies_match_power(oracle, power):
    """The renderer picks light i with probability power_i / sum: psel equals
    it, and the frequencies of 2^21 choices made the renderer's way pass a
    chi-square test against it (each bin's standardised deviation too)."""
    w = np.asarray(power, np.float64)
    n = 1 << 21
    psel, counts = oracle.light_selection(w, n, seed=3)
    assert np.allclose(psel, w / w.sum(), rtol=1e-12)
    assert counts.sum() == n
    expect = n * psel
    z = (counts - expect) / np.sqrt(np.maximum(expect * (1 - psel), 1e-12))
    assert np.all(np.abs(z) < 5), z
    if len(w) > 1:
        chi2 = float(np.sum((counts - expect) ** 2 / expect))
        assert chi2 < len(w) - 1 + 6 * math.sqrt(2 * (len(w) - 1)), chi2


def test_alias_selection_many_lights(oracle):
    """1000 lights with powers log-uniform over two decades (the many-lights
    workload's distribution): chi-square per degree of freedom near 1."""
    rng = np.random.default_rng(10)
    w = 10 ** rng.uniform(2, 4, 1000)
    n = 1 << 22
    psel, counts = oracle.light_selection(w, n, seed=4)
    expect = n * psel
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    dof = len(w) - 1
    assert abs(chi2 / dof - 1.0) < 6 * math.sqrt(2.0 / dof), chi2 / dof


# --------------------------------------------------------------------------
# BVH closest hit versus brute force and versus an independent FP64 test
# --------------------------------------------------------------------------
def _random_rays(rng, n, lo, hi):
    o = rng.uniform(lo, hi, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.concatenate([o, d], 1).astype(np.float32)


def test_bvh_equals_brute_force(oracle):
    from paper_1909_00573_gb300 import scenes
    s = scenes.tiny_room()
    rng = np.random.default_rng(5)
    rays = _random_rays(rng, 4000, 0.02, 0.98)
    p1, t1 = oracle.trace(s, rays, brute=False)
    p2, t2 = oracle.trace(s, rays, brute=True)
    assert np.array_equal(p1, p2)
    assert np.array_equal(t1[p1 >= 0], t2[p2 >= 0])
    assert np.mean(p1 >= 0) > 0.75          # the room is open at z = 0


def test_bvh_equals_brute_force_axis_aligned_rays(oracle):
    """Rays parallel to box planes (direction components +0 and -0) from
    origins on those planes: a slab whose distance is 0 * inf = NaN must not
    reject the box, whatever the sign of the zero."""
    from paper_1909_00573_gb300 import scenes
    rng = np.random.default_rng(13)
    tri = np.concatenate([scenes.box_faces((2.0 * i, 0.0, 2.0 * j), (2.0 * i + 1.0, 2.0, 2.0 * j + 1.0))
                          for i in range(4) for j in range(4)], 0).astype(np.float32)
    s = scenes.Scene(tri, np.zeros(len(tri)), np.zeros((0, 4)), np.zeros(0),
                     scenes.material(0, (0.5,) * 3)[None], np.zeros(10))
    n = 6000
    o = rng.integers(-2, 17, (n, 3)) * 0.5
    o[:, 1] = rng.integers(0, 5, n) * 0.5
    d = np.concatenate([np.eye(3), -np.eye(3)])[rng.integers(0, 6, n)]   # -np.eye holds -0.0
    rays = np.concatenate([o, d], 1).astype(np.float32)
    assert np.signbit(rays[:, 3:][rays[:, 3:] == 0]).any()
    p1, t1 = oracle.trace(s, rays, brute=False)
    p2, t2 = oracle.trace(s, rays, brute=True)
    assert np.mean(p2 >= 0) > 0.2
    assert np.array_equal(p1, p2)
    assert np.array_equal(t1[p1 >= 0], t2[p2 >= 0])


def _mt_double(o, d, tri):
    """Moeller-Trumbore in FP64 over all triangles: (prim, t)."""
    v0, v1, v2 = tri[:, 0].astype(np.float64), tri[:, 1].astype(np.float64), tri[:, 2].astype(np.float64)
    e1, e2 = v1 - v0, v2 - v0
    pv = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    ok = np.abs(det) > 1e-14
    inv = np.where(ok, 1.0 / np.where(ok, det, 1), 0)
    tv = o - v0
    u = np.einsum("ij,ij->i", tv, pv) * inv
    qv = np.cross(tv, e1)
    v = (qv @ d) * inv
    t = np.einsum("ij,ij->i", e2, qv) * inv
    hit = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 1e-9)
    if not hit.any():
        return -1, np.inf
    t = np.where(hit, t, np.inf)
    i = int(np.argmin(t))
    return i, float(t[i])


def test_watertight_triangle_test_vs_fp64(oracle):
    from paper_1909_00573_gb300 import scenes
    rng = np.random.default_rng(6)
    tri = rng.uniform(-1, 1, (60, 3, 3)).astype(np.float32)
    s = scenes.Scene(tri, np.zeros(60), np.zeros((0, 4)), np.zeros(0), scenes.material(0, (0.5,) * 3)[None],
                     np.zeros(10))
    rays = _random_rays(rng, 1500, -0.5, 0.5)
    prim, t = oracle.trace(s, rays, brute=True)
    agree = 0
    for i in range(len(rays)):
        j, tt = _mt_double(rays[i, :3].astype(np.float64), rays[i, 3:].astype(np.float64), tri)
        if j == prim[i]:
            agree += 1
            if j >= 0:
                assert t[i] == pytest.approx(tt, rel=1e-4, abs=1e-5)
    assert agree >= len(rays) - 3      # edge / near-tie cases only


def test_sphere_intersection(oracle):
    from paper_1909_00573_gb300 import scenes
    s = scenes.Scene(np.zeros((0, 3, 3)), np.zeros(0), np.array([[0, 0, 5, 1.0], [100, 0, 0, 0.05]]),
                     np.array([0, 0]), scenes.material(0, emission=(1, 1, 1))[None], np.zeros(10))
    rays = np.array([[0, 0, 0, 0, 0, 1], [0, 0.5, 0, 0, 0, 1], [0, 0, 5, 1, 0, 0], [0, 0, 0, 1, 0, 0],
                     [0, 0.06, 0, 1, 0, 0]], np.float32)
    prim, t = oracle.trace(s, rays)
    assert prim.tolist() == [0, 0, 0, 1, -1]
    assert t[0] == pytest.approx(4.0, rel=1e-6)
    assert t[1] == pytest.approx(5 - math.sqrt(0.75), rel=1e-6)
    assert t[2] == pytest.approx(1.0, rel=1e-6)     # from the centre: far root
    assert t[3] == pytest.approx(99.95, rel=1e-6)   # distant small sphere (cancellation-free form)


# --------------------------------------------------------------------------
# merge candidate search (range search around photons)
# --------------------------------------------------------------------------
def test_neighbour_search_equals_brute_force(oracle):
    rng = np.random.default_rng(7)
    pts = rng.uniform(0, 1, (3000, 3)).astype(np.float32)
    q = rng.uniform(0, 1, (500, 3)).astype(np.float32)
    r = 0.05
    a = oracle.count_neighbours(pts, q, r, brute=False)
    b = oracle.count_neighbours(pts, q, r, brute=True)
    d2 = ((pts[None, :, :] - q[:, None, :]) ** 2)
    d2 = (d2[..., 0] + d2[..., 1]) + d2[..., 2]          # FP32, same order
    c = (d2 <= np.float32(r) * np.float32(r)).sum(1)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert c.sum() > 0


# --------------------------------------------------------------------------
# BSDFs: textbook Fresnel, Snell, cosine sampling, sampler/pdf consistency
# --------------------------------------------------------------------------
def fresnel_textbook(cos_i, n1, n2):
    sin_t = n1 / n2 * math.sqrt(max(0.0, 1 - cos_i ** 2))
    if sin_t >= 1:
        return 1.0
    cos_t = math.sqrt(1 - sin_t ** 2)
    rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t)
    rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t)
    return 0.5 * (rs * rs + rp * rp)


@pytest.mark.parametrize("theta_deg,entering", [(0, True), (30, True), (56.31, True), (80, True),
                                                 (20, False), (41, False), (45, False)])
def test_dielectric_fresnel_snell_and_scaling(oracle, theta_deg, entering):
    from paper_1909_00573_gb300 import scenes
    glass = scenes.material(scenes.MAT_DIELECTRIC, ior=1.5)
    th = math.radians(theta_deg)
    n = np.array([0, 0, 1.0], np.float32)
    wo = np.array([math.sin(th), 0, math.cos(th) if entering else -math.cos(th)], np.float32)
    n1, n2 = (1.0, 1.5) if entering else (1.5, 1.0)
    F = fresnel_textbook(math.cos(th), n1, n2)
    # bisection on the lobe random number locates the reflect/refract switch
    lo, hi = 0.0, 1.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        ok, wi, w, pdf, f = oracle.bsdf_sample(glass, n, wo, [mid, 0.5, 0.5])
        reflected = (wi[2] > 0) == (wo[2] > 0)
        lo, hi = (mid, hi) if reflected else (lo, mid)
    assert lo == pytest.approx(F, abs=2e-6)
    ok, wi, w, pdf, f = oracle.bsdf_sample(glass, n, wo, [0.0, 0.5, 0.5])   # reflection
    assert np.allclose(wi, [-wo[0], -wo[1], wo[2]], atol=1e-6) and np.allclose(w, 1)
    if F < 1:
        ok, wi, w, pdf, f = oracle.bsdf_sample(glass, n, wo, [0.999999, 0.5, 0.5], camera=True)
        sin_t = math.hypot(wi[0], wi[1])
        assert n1 * math.sin(th) == pytest.approx(n2 * sin_t, abs=1e-5)       # Snell
        assert (wi[2] > 0) != (wo[2] > 0)
        assert w[0] == pytest.approx((n1 / n2) ** 2, rel=1e-6)                 # radiance scaling
        ok, wi, w, pdf, f = oracle.bsdf_sample(glass, n, wo, [0.999999, 0.5, 0.5], camera=False)
        assert w[0] == pytest.approx(1.0)


def test_lambert_sampling_is_cosine_weighted(oracle):
    from paper_1909_00573_gb300 import scenes
    m = scenes.material(0, (0.6, 0.5, 0.4))
    rng = np.random.default_rng(8)
    n = np.array([0.0, 0.6, 0.8], np.float32)
    wo = np.array([0.0, 0.0, 1.0], np.float32)
    cos = []
    for u in rng.uniform(0, 1, (4000, 3)):
        ok, wi, w, pdf, f = oracle.bsdf_sample(m, n, wo, u)
        c = float(wi @ n)
        assert ok and c > 0 and np.allclose(w, [0.6, 0.5, 0.4], rtol=1e-6)
        assert pdf == pytest.approx(c / math.pi, rel=1e-5) and f[0] == pytest.approx(0.6 / math.pi)
        cos.append(c)
    assert np.mean(cos) == pytest.approx(2 / 3, abs=0.015)                  # E[cos] under cos/pi
    assert np.mean(np.square(cos)) == pytest.approx(0.5, abs=0.015)         # E[cos^2] = 1/2


def test_ggx_sampler_matches_its_pdf_and_brdf(oracle):
    """E[f cos / pdf] over the sampler equals the quadrature of f cos over the
    hemisphere, and f is reciprocal."""
    from paper_1909_00573_gb300 import scenes
    m = scenes.material(scenes.MAT_GGX, (0.9, 0.9, 0.9), alpha=0.3)
    n = np.array([0, 0, 1.0], np.float32)
    th = math.radians(35)
    wo = np.array([math.sin(th), 0, math.cos(th)], np.float32)
    rng = np.random.default_rng(9)
    acc = []
    for u in rng.uniform(0, 1, (20000, 3)):
        ok, wi, w, pdf, f = oracle.bsdf_sample(m, n, wo, u)
        acc.append(w[0] if ok else 0.0)
    mc = float(np.mean(acc))
    # midpoint quadrature in (cos theta, phi)
    N = 200
    tot = 0.0
    for i in range(N):
        ct = (i + 0.5) / N
        st = math.sqrt(1 - ct * ct)
        for j in range(2 * N):
            ph = (j + 0.5) / (2 * N) * 2 * math.pi
            wi = np.array([st * math.cos(ph), st * math.sin(ph), ct], np.float32)
            f, _ = oracle.bsdf_eval(m, n, wo, wi)
            tot += f[0] * ct
    quad = tot * (1.0 / N) * (2 * math.pi / (2 * N))
    assert mc == pytest.approx(quad, rel=0.03)
    wi = np.array([-0.3, 0.2, 0.93], np.float32)
    wi /= np.linalg.norm(wi)
    f1, p1 = oracle.bsdf_eval(m, n, wo, wi)
    f2, p2 = oracle.bsdf_eval(m, n, wi, wo)
    assert f1[0] == pytest.approx(f2[0], rel=1e-5) and p1 == pytest.approx(p2, rel=1e-5)


# --------------------------------------------------------------------------
# MIS weights (Eq. rhpdf, Eq. neepdf, Eq. photonpdf, Eq. misw): hand-worked
# --------------------------------------------------------------------------
def test_mis_length_two_hand_worked(oracle):
    # camera (0,1,0) -> floor point (0,0,0), normal +y -> light point (0,2,0)
    # facing down, NEE area pdf p_l = 0.25.
    # p_e = p_{0->1} p_{1->2} = 1 * (cos/pi = 1/pi) * cos_y / d^2 = 1/(4 pi)
    # p_E = p_l * p_{0->1} = 0.25
    verts = [[0, 1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 1, 0, 0]]
    light = [0, 2, 0, 0, -1, 0, 0.25]
    w = oracle.mis_weights(verts, light, 0.01, 50.0)
    pe, pE = 1 / (4 * math.pi), 0.25
    assert w[0] == pytest.approx(pe / (pe + pE), rel=1e-6)
    assert w[1] == pytest.approx(pE / (pe + pE), rel=1e-6)
    assert w.sum() == pytest.approx(1.0)


def test_mis_length_three_hand_worked(oracle):
    """Path x0=(0,1,0) camera, x1=(0,0,0) floor (n=+y), x2=(0,1,1) wall (n=-z),
    light x3=(0,1,0) facing +z, p_l=0.5, rho=100, r=0.05.
      F2 = p_{1->2} = (cos_1/pi)(cos_2)/d^2 = (1/sqrt2/pi)(1/sqrt2)/2 = 1/(4 pi)
      F3 = p_{2->3} = (1/pi)(1)/1 = 1/pi
      R1 = p_{2->1} = (1/sqrt2/pi)(1/sqrt2)/2 = 1/(4 pi)
      p_e = F2 F3 = 1/(4 pi^2);  p_E = p_l F2 = 1/(8 pi)
      n_P p_P1 = p_l rho pi r^2 R1 = 0.5*100*pi*0.0025/(4 pi) = 1/32"""
    verts = [[0, 1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 1, 0, 0], [0, 1, 1, 0, 0, -1, 0]]
    light = [0, 1, 0, 0, 0, 1, 0.5]
    pe, pE, pP = 1 / (4 * math.pi ** 2), 1 / (8 * math.pi), 1 / 32
    s = pe + pE + pP
    w = oracle.mis_weights(verts, light, 0.05, 100.0)
    assert w.tolist() == pytest.approx([pe / s, pE / s, pP / s], rel=1e-5)
    # strategy mask: without photons the same path is weighted between e and E only
    w = oracle.mis_weights(verts, light, 0.05, 100.0, mask=3)
    assert w.tolist() == pytest.approx([pe / (pe + pE), pE / (pe + pE), 0.0], rel=1e-5)
    # rho = 0 (no density) removes the photon strategy
    w = oracle.mis_weights(verts, light, 0.05, 0.0)
    assert w[2] == 0.0


def test_mis_delta_vertices(oracle):
    verts = [[0, 1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 1, 0, 0], [0, 1, 1, 0, 0, -1, 1]]
    light = [0, 1, 0, 0, 0, 1, 0.5]
    w = oracle.mis_weights(verts, light, 0.05, 100.0)
    assert w[1] == 0.0                      # no NEE at a delta vertex
    # pdf at the delta vertex x2 is 1: F3 = 1 * 1 / 1, R1 = 1 * (1/sqrt2) / 2
    pe = 1 / (4 * math.pi) * 1.0
    pP = 0.5 * 100 * math.pi * 0.0025 * (1 / (2 * math.sqrt(2)))
    assert w[0] == pytest.approx(pe / (pe + pP), rel=1e-5)
    verts[1][6] = 1                         # merge vertex on glass: no merge strategy
    verts[2][6] = 0
    w = oracle.mis_weights(verts, light, 0.05, 100.0)
    assert w[2] == 0.0 and w[0] + w[1] == pytest.approx(1.0)


def test_mis_with_light_photons_hand_worked(oracle):
    """Eq. stdphotonpdf with n_LP light photons: p_LP,k = p_l^LP pi r^2
    prod_{i=k}^{l-1} p_{i+1->i} prod_{i<k} p_{i->i+1}, where the light emits
    cosine-weighted, p_{l->l-1} = (cos_y / pi) |cos_{l-1}| / d^2.
    Length 2 (x1 floor at the origin, light (0,2,0) facing down): R1 = 1/(4 pi),
      n_LP p_LP1 = 1000 pi 1e-4 0.125 / (4 pi) = 3.125e-3.
    Length 3 (the path of the length-three test, light facing +z):
      R1 = 1/(4 pi), R2 = 1/pi, F2 = 1/(4 pi):
      n_LP p_LP1 = 500 pi 0.0025 0.25 R1 R2 = n_LP p_LP2 = 500 pi 0.0025 0.25 R2 F2."""
    verts = [[0, 1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 1, 0, 0]]
    light = [0, 2, 0, 0, -1, 0, 0.25, 0.125]
    w = oracle.mis_weights_lp(verts, light, 0.01, 50.0, 1000.0)
    pe, pE, pLP = 1 / (4 * math.pi), 0.25, 1000 * math.pi * 1e-4 * 0.125 / (4 * math.pi)
    S = pe + pE + pLP
    assert w.tolist() == pytest.approx([pe / S, pE / S, pLP / S], rel=1e-5)
    verts = [[0, 1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 1, 0, 0], [0, 1, 1, 0, 0, -1, 0]]
    light = [0, 1, 0, 0, 0, 1, 0.5, 0.25]
    pe, pE, pP = 1 / (4 * math.pi ** 2), 1 / (8 * math.pi), 1 / 32
    lp = 500 * math.pi * 0.0025 * 0.25 * (1 / (4 * math.pi)) * (1 / math.pi)
    S = pe + pE + pP + 2 * lp
    w = oracle.mis_weights_lp(verts, light, 0.05, 100.0, 500.0)
    assert w.tolist() == pytest.approx([pe / S, pE / S, pP / S, lp / S, lp / S], rel=1e-5)
    assert w.sum() == pytest.approx(1.0)
    # no light photons: the weights of the plain combination, LP weights 0
    w0 = oracle.mis_weights_lp(verts, light, 0.05, 100.0, 0.0)
    assert w0[:3].tolist() == pytest.approx(oracle.mis_weights(verts, light[:7], 0.05, 100.0).tolist(), rel=1e-9)
    assert w0[3:].tolist() == [0.0, 0.0]
    # a delta vertex cannot be a merge vertex: LP weight there is 0
    verts[2][6] = 1
    w = oracle.mis_weights_lp(verts, light, 0.05, 100.0, 500.0)
    assert w[4] == 0.0 and w[1] == 0.0 and w.sum() == pytest.approx(1.0)


def test_density_estimators_closed_forms(oracle):
    """The naive and k-nearest estimators of Sec. 5 on a unit square lattice
    in the plane z = 0: within radius 1.5 an interior point sees itself and 8
    neighbours (9 / (pi 2.25)); its 5th nearest other point is at sqrt(2)
    ((5 - 1) / (pi 2)); its 4th at distance 1 ((4 - 1) / pi)."""
    g = np.stack(np.meshgrid(np.arange(9.0), np.arange(9.0), indexing="ij"), -1).reshape(-1, 2)
    pts = np.concatenate([g, np.zeros((len(g), 1))], 1).astype(np.float32)
    interior = np.all((g >= 1) & (g <= 7), axis=1)
    naive = oracle.density_naive(pts, 1.5)
    assert np.allclose(naive[interior], 9.0 / (np.pi * 2.25), rtol=1e-6)
    corner = np.all(g == 0, axis=1)
    assert np.allclose(naive[corner], 4.0 / (np.pi * 2.25), rtol=1e-6)
    assert np.allclose(oracle.density_knn(pts, 5)[interior], 4.0 / (np.pi * 2.0), rtol=1e-6)
    assert np.allclose(oracle.density_knn(pts, 4)[interior], 3.0 / np.pi, rtol=1e-6)
    assert np.all(oracle.density_knn(pts[:3], 4) == 0.0)          # fewer than k other points


def test_knn_estimator_unbiased_on_uniform_points(oracle):
    """(k - 1) / (pi d_k^2) is unbiased for a Poisson process of intensity
    lambda (Loftsgaarden and Quesenberry 1965): 4000 uniform points in a unit
    square (lambda = 4000), mean over points away from the border."""
    rng = np.random.default_rng(12)
    xy = rng.uniform(0, 1, (4000, 2))
    pts = np.concatenate([xy, np.zeros((4000, 1))], 1).astype(np.float32)
    inner = np.all((xy > 0.1) & (xy < 0.9), axis=1)
    for k in (4, 8):
        est = oracle.density_knn(pts, k)[inner]
        assert abs(est.mean() / 4000.0 - 1.0) < 0.05, (k, est.mean())
    # the naive estimator counts the point itself: E = lambda + 1 / (pi h^2)
    h = 0.02
    est = oracle.density_naive(pts, h)[inner]
    assert abs(est.mean() / (4000.0 + 1.0 / (np.pi * h * h)) - 1.0) < 0.03
