"""The allocation-free neighbour count (neb_count_neighbours_noalloc).

It serves callers that must not allocate device memory (their memory is held
by their own pool, or cudaMalloc's implicit synchronisation is not acceptable
in their loop).  Its results must equal the allocating entry point's on the
same inputs, also on back-to-back calls that reuse the shared scratch array.
This file is collected last on purpose; it must pass both alone in a fresh
process and after the other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_1909_00573_gb300 import build
    build.build()
    from paper_1909_00573_gb300 import neb
    rng = np.random.default_rng(71)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    for call, (n, m, r) in enumerate([(50000, 4000, 0.02), (neb.NOALLOC_MAX_POINTS, 3000, 0.005)]):
        pts = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
        q = np.concatenate([rng.uniform(-1, 1, (m - 500, 3)), pts[:500]]).astype(np.float32)
        ref = neb.count_neighbours(pts, q, r)                       # allocating entry point
        d_pts = torch.from_numpy(pts).to(dev)
        d_q = torch.from_numpy(q).to(dev)
        d_out = torch.full((m,), -7, dtype=torch.int32, device=dev)
        neb.count_neighbours_noalloc(d_pts.data_ptr(), n, d_q.data_ptr(), m, r, d_out.data_ptr(),
                                     stream.cuda_stream)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy()
        assert np.array_equal(got, ref), call          # integer counts: exact
        assert ref.sum() > 0
    # sizes beyond the fixed scratch are rejected before any device work
    with pytest.raises(neb.NebError):
        neb.count_neighbours_noalloc(d_pts.data_ptr(), neb.NOALLOC_MAX_POINTS + 1, d_q.data_ptr(), 10, 0.01,
                                     d_out.data_ptr(), stream.cuda_stream)


def test_noalloc_far_coordinates_and_stream_of_another_device():
    """Coordinates near 5e6 with r = 1e-3 (grid cells beyond 2^30 per axis,
    held at the boundary cell) give the allocating entry point's counts; a
    stream that does not belong to the current device is refused."""
    torch = pytest.importorskip("torch")
    from paper_1909_00573_gb300 import build
    build.build()
    from paper_1909_00573_gb300 import neb
    rng = np.random.default_rng(72)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    lattice = (5.0e6 + 0.5 * rng.integers(0, 40, (300, 3))).astype(np.float32)
    pts = np.repeat(lattice, rng.integers(1, 5, len(lattice)), axis=0)
    q = lattice.copy()
    ref = neb.count_neighbours(pts, q, 1e-3)
    d_pts = torch.from_numpy(pts).to(dev)
    d_q = torch.from_numpy(q).to(dev)
    for _ in range(2):
        d_out = torch.full((len(q),), -7, dtype=torch.int32, device=dev)
        neb.count_neighbours_noalloc(d_pts.data_ptr(), len(pts), d_q.data_ptr(), len(q), 1e-3, d_out.data_ptr(),
                                     stream.cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(d_out.cpu().numpy(), ref)
    if torch.cuda.device_count() > 1:
        other = torch.cuda.Stream(device=torch.device("cuda", 1))
        with pytest.raises(neb.NebError):
            neb.count_neighbours_noalloc(d_pts.data_ptr(), len(pts), d_q.data_ptr(), len(q), 1e-3,
                                         d_out.data_ptr(), other.cuda_stream)
