"""CPU-side checks of the C ABI: the library builds, loads and exports every
function that include/neb.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "neb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(neb_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libneb():
    from paper_1909_00573_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_function(libneb):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(libneb, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1909_00573_gb300 import neb
    assert sorted(neb.EXPORTS) == declared_functions()


def test_argument_errors_without_gpu(libneb):
    """Invalid arguments are rejected before any device call."""
    from paper_1909_00573_gb300 import neb
    L = neb.lib()
    h = ctypes.c_void_p()
    cfg = neb.Config(0, 8, 4, 0.01, 64, 4, 0, 0, 0, 7, 0, 0)       # width 0
    assert L.neb_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    cfg = neb.Config(8, 8, 99, 0.01, 64, 4, 0, 0, 0, 7, 0, 0)      # depth above 64
    assert L.neb_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    cfg = neb.Config(8, 8, 4, 0.01, 64, 4, 0, 0, 0, 17, 0, 0)      # unknown strategy bit
    assert L.neb_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    cfg = neb.Config(8, 8, 4, 0.01, 64, 4, 0, 0, 0, 15, 0, 0, 0, -1)  # negative light-photon count
    assert L.neb_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    cfg = neb.Config(8, 8, 4, 0.01, 64, 4, 0, 0, 0, 7, 0, 0, 0, 0, 2)  # density_all not 0 or 1
    assert L.neb_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    cfg = neb.Config(8, 8, 4, 0.01, 64, 4, 0, 0, 0, 7, 0, 5)       # unknown BVH builder
    assert L.neb_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    assert L.neb_iterate(None, 1) == -1
    assert L.neb_iterate_read(None, 1, None) == -1
    assert L.neb_bvh_cost(None, None) == -1
    assert L.neb_philox(None, -1, None, None) == -1


def test_batch_and_admission_arguments_without_gpu(libneb):
    """neb_iterate_batch rejects bad arguments before any device call, an empty
    batch is a no-op, and neb_job_device_bytes is a pure host computation."""
    from paper_1909_00573_gb300 import neb, scenes
    L = neb.lib()
    assert L.neb_iterate_batch(None, -1, 1) == neb.ERR_ARG
    assert L.neb_iterate_batch(None, 2, 1) == neb.ERR_ARG
    assert L.neb_iterate_batch(None, 0, 3) == neb.NEB_OK
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.neb_iterate_batch(arr, 2, 1) == neb.ERR_ARG
    s, rc = scenes.workload("large_city")
    cfg = neb.make_config(rc)
    b = neb.job_device_bytes(cfg, s.n_tri, s.n_sph, len(s.mats), s.n_emitters)
    # two NEE slots of 112 B per vertex dominate: 2 x 921,600 x 9 x 112 B
    assert 2 * 921600 * 9 * 112 < b < 7e9
    # the staging list of the per-cell merge: 2 x 921,600 x 9 hits of 48 B, a
    # 4-B order and an 8-B tile each, and two 4-B arrays per photon bucket
    inline = neb.job_device_bytes(neb.make_config(rc, merge_mode=1), s.n_tri, s.n_sph, len(s.mats),
                                  s.n_emitters)
    assert b - inline == 2 * 921600 * 9 * 60 + 2 * 4 * ((1 << 22) + 1)
    split = neb.job_device_bytes(neb.make_config(rc, keep_split=True), s.n_tri, s.n_sph, len(s.mats),
                                 s.n_emitters)
    assert split - b == 921600 * 12 * 8                         # the FP64 per-strategy split (4 strategies)
    rc2 = scenes.RenderConfig(2 * rc.width, rc.height, rc.max_depth, rc.merge_radius, rc.octree_capacity,
                              rc.split_factor, 1)
    assert neb.job_device_bytes(neb.make_config(rc2), s.n_tri, s.n_sph, len(s.mats), s.n_emitters) > b
    with pytest.raises(neb.NebError):
        neb.job_device_bytes(cfg, 0, 0, len(s.mats), 0)        # empty scene
    with pytest.raises(neb.NebError):
        neb.job_device_bytes(cfg, 10, 0, 1, 11)                 # more lights than primitives


def test_product_path_does_not_import_the_oracle():
    """The package never reaches into oracle/ (the oracle is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1909_00573_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert not re.search(r"(from\s+oracle|import\s+oracle|liboracle|neb_oracle)", txt), f
