"""ctypes front end of the CPU oracle (neb_oracle.c).

Test infrastructure only: imported by the tests, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product path never imports
this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIB_DIR, "liboracle.so")
SRC = os.path.join(HERE, "neb_oracle.c")

ST_NAMES = ["camera_rays", "nee_vertices", "shadow_rays", "photons", "photon_hits",
            "merges", "random_hits", "octree_nodes", "octree_depth"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-ffp-contract=off: FP32 parts round identically on every host)."""
    os.makedirs(LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                            os.path.getmtime(os.path.join(HERE, "neb_oracle.h")))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
           "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


class _Scene(C.Structure):
    _fields_ = [("tri", C.c_void_p), ("tri_mat", C.c_void_p), ("nt", C.c_int),
                ("sph", C.c_void_p), ("sph_mat", C.c_void_p), ("ns", C.c_int),
                ("mats", C.c_void_p), ("nm", C.c_int), ("cam", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("max_depth", C.c_int),
                ("merge_radius", C.c_float), ("octree_capacity", C.c_int), ("split_factor", C.c_int),
                ("seed", C.c_uint64), ("density_mode", C.c_int), ("strategy_mask", C.c_uint32),
                ("first_iteration", C.c_int), ("pixel_begin", C.c_int), ("pixel_end", C.c_int),
                ("iter_seconds", C.c_void_p), ("lp_photons", C.c_int), ("iter_images", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        L.orc_render.argtypes = [C.POINTER(_Scene), C.POINTER(_Config), C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
        L.orc_render.restype = C.c_int
        L.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_intersection_area.argtypes = [C.c_void_p] * 4
        L.orc_intersection_area.restype = C.c_double
        L.orc_octree_new.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int]
        L.orc_octree_new.restype = C.c_void_p
        L.orc_octree_free.argtypes = [C.c_void_p]
        L.orc_octree_set_iteration.argtypes = [C.c_void_p, C.c_int]
        L.orc_octree_increment.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_octree_density.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.orc_octree_density.restype = C.c_float
        L.orc_octree_dump.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.orc_octree_dump.restype = C.c_int
        L.orc_octree_load.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int]
        L.orc_octree_load.restype = C.c_int
        L.orc_onb.argtypes = [C.c_void_p] * 3
        L.orc_light_selection.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_uint64, C.c_void_p, C.c_void_p]
        L.orc_light_selection.restype = C.c_int
        L.orc_trace.argtypes = [C.POINTER(_Scene), C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        L.orc_count_neighbours.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_float, C.c_int,
                                           C.c_void_p]
        L.orc_density_naive.argtypes = [C.c_void_p, C.c_int, C.c_float, C.c_void_p]
        L.orc_density_knn.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.orc_mis_weights.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_float, C.c_double, C.c_uint32,
                                      C.c_void_p]
        L.orc_mis_weights.restype = C.c_int
        L.orc_mis_weights_lp.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_float, C.c_double, C.c_uint32,
                                         C.c_double, C.c_void_p]
        L.orc_mis_weights_lp.restype = C.c_int
        L.orc_bsdf_probe.argtypes = [C.c_void_p] * 4 + [C.c_int] + [C.c_void_p] * 4
        L.orc_bsdf_probe.restype = C.c_int
        L.orc_bsdf_eval_probe.argtypes = [C.c_void_p] * 6
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _scene_struct(scene):
    keep = [np.ascontiguousarray(scene.tri, np.float32), np.ascontiguousarray(scene.tri_mat, np.uint32),
            np.ascontiguousarray(scene.sph, np.float32), np.ascontiguousarray(scene.sph_mat, np.uint32),
            np.ascontiguousarray(scene.mats, np.float32), np.ascontiguousarray(scene.cam, np.float32)]
    s = _Scene(_ptr(keep[0]), _ptr(keep[1]), len(keep[1]), _ptr(keep[2]), _ptr(keep[3]), len(keep[3]),
               _ptr(keep[4]), len(keep[4]), _ptr(keep[5]))
    return s, keep


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def intersection_area(bmin, bmax, pos, normal):
    a = [np.ascontiguousarray(x, np.float32) for x in (bmin, bmax, pos, normal)]
    return float(lib().orc_intersection_area(*[_ptr(x) for x in a]))


class Octree:
    """Density octree of Sec. 5, counted sequentially (deterministic insertion order)."""

    def __init__(self, scene_min, scene_max, capacity, split_factor):
        self._mn = np.ascontiguousarray(scene_min, np.float32)
        self._mx = np.ascontiguousarray(scene_max, np.float32)
        self.h = lib().orc_octree_new(_ptr(self._mn), _ptr(self._mx), int(capacity), int(split_factor))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_octree_free(self.h)
            self.h = None

    def set_iteration(self, it):
        lib().orc_octree_set_iteration(self.h, int(it))

    def insert(self, positions):
        P = np.ascontiguousarray(positions, np.float32).reshape(-1, 3)
        for p in P:
            lib().orc_octree_increment(self.h, _ptr(np.ascontiguousarray(p)))

    def density(self, positions, normals, robust=True):
        P = np.ascontiguousarray(positions, np.float32).reshape(-1, 3)
        N = np.ascontiguousarray(normals, np.float32).reshape(-1, 3)
        out = np.zeros(len(P), np.float32)
        for i in range(len(P)):
            out[i] = lib().orc_octree_density(self.h, _ptr(np.ascontiguousarray(P[i])),
                                              _ptr(np.ascontiguousarray(N[i])), int(robust))
        return out

    def dump(self):
        meta = np.zeros(3, np.int32)
        cap = lib().orc_octree_dump(self.h, None, 0, _ptr(meta))
        nodes = np.zeros(cap, np.int32)
        lib().orc_octree_dump(self.h, _ptr(nodes), cap, _ptr(meta))
        return nodes, int(meta[0]), int(meta[1])

    def load(self, words, words_used, depth):
        """Replace the tree by the one in the flat layout of Sec. 5.5."""
        w = np.ascontiguousarray(words, np.int32)
        rc = lib().orc_octree_load(self.h, _ptr(w), len(w), int(words_used), int(depth))
        if rc != 0:
            raise ValueError("malformed octree layout")


def onb(normal):
    """(t, b) of the Duff et al. basis of a unit normal."""
    n = np.ascontiguousarray(normal, np.float32)
    t = np.zeros(3, np.float32)
    b = np.zeros(3, np.float32)
    lib().orc_onb(_ptr(n), _ptr(t), _ptr(b))
    return t, b


def light_selection(power, n_samples, seed=0):
    """(psel, counts): selection probabilities of the alias table built from
    `power` and how often the renderer's selection picked each light."""
    w = np.ascontiguousarray(power, np.float64)
    psel = np.zeros(len(w), np.float64)
    counts = np.zeros(len(w), np.int64)
    rc = lib().orc_light_selection(_ptr(w), len(w), int(n_samples), C.c_uint64(seed), _ptr(psel), _ptr(counts))
    assert rc == 0
    return psel, counts


def trace(scene, rays, brute=False):
    s, keep = _scene_struct(scene)
    R = np.ascontiguousarray(rays, np.float32).reshape(-1, 6)
    prim = np.zeros(len(R), np.int32)
    t = np.zeros(len(R), np.float32)
    lib().orc_trace(C.byref(s), _ptr(R), len(R), int(brute), _ptr(prim), _ptr(t))
    return prim, t


def count_neighbours(points, queries, r, brute=False):
    P = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    Q = np.ascontiguousarray(queries, np.float32).reshape(-1, 3)
    out = np.zeros(len(Q), np.int32)
    lib().orc_count_neighbours(_ptr(P), len(P), _ptr(Q), len(Q), C.c_float(r), int(brute), _ptr(out))
    return out


def density_naive(points, radius):
    """Naive estimator (Sec. 5) at every point, brute force."""
    P = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    out = np.zeros(len(P), np.float32)
    lib().orc_density_naive(_ptr(P), len(P), C.c_float(radius), _ptr(out))
    return out


def density_knn(points, k):
    """k-nearest-neighbour estimator (Sec. 5) at every point, brute force."""
    P = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    out = np.zeros(len(P), np.float32)
    lib().orc_density_knn(_ptr(P), len(P), int(k), _ptr(out))
    return out


def mis_weights(verts, light, merge_radius, rho, mask=7):
    V = np.ascontiguousarray(verts, np.float32).reshape(-1, 7)
    Lt = np.ascontiguousarray(light, np.float32).reshape(7)
    w = np.zeros(len(V) + 1, np.float64)
    rc = lib().orc_mis_weights(_ptr(V), len(V), _ptr(Lt), C.c_float(merge_radius), C.c_double(rho),
                               C.c_uint32(mask), _ptr(w))
    assert rc == 0
    return w[:len(V)]   # w_e, w_E, w_P1 .. w_P(l-2)


def mis_weights_lp(verts, light, merge_radius, rho, n_lp, mask=15):
    """light = pos, normal, p_l, p_l^LP.  Returns w_e, w_E, w_P1 .. w_P(l-2),
    w_LP1 .. w_LP(l-1) with l = len(verts)."""
    V = np.ascontiguousarray(verts, np.float32).reshape(-1, 7)
    Lt = np.ascontiguousarray(light, np.float32).reshape(8)
    w = np.zeros(2 * len(V) + 1, np.float64)
    rc = lib().orc_mis_weights_lp(_ptr(V), len(V), _ptr(Lt), C.c_float(merge_radius), C.c_double(rho),
                                  C.c_uint32(mask), C.c_double(n_lp), _ptr(w))
    assert rc == 0
    return w[:2 * len(V) - 1]


def render(scene, cfg, n_iter=None, first_iteration=1, pixel_range=None, want_split=True, want_rho=False,
           want_iterations=False):
    """Run the oracle.  Returns dict with accum [H,W,3] (sum over iterations),
    split [4,H,W,3] of the last iteration (random hits, NEE, NEB photon merges,
    light-photon merges), rho [H*W, D-1], stats and, with want_iterations,
    iterations [n_iter,H,W,3] (each iteration's own image)."""
    n_iter = cfg.iterations if n_iter is None else n_iter
    s, keep = _scene_struct(scene)
    pb, pe = (0, 0) if pixel_range is None else pixel_range
    iter_sec = np.zeros(max(int(n_iter), 1), np.float64)
    P = cfg.width * cfg.height
    iters = np.zeros((max(int(n_iter), 1), P, 3), np.float64) if want_iterations else None
    c = _Config(cfg.width, cfg.height, cfg.max_depth, cfg.merge_radius, cfg.octree_capacity, cfg.split_factor,
                cfg.seed, cfg.density_mode, cfg.strategy_mask, first_iteration, pb, pe, _ptr(iter_sec),
                getattr(cfg, "lp_photons", 0), _ptr(iters))
    accum = np.zeros((P, 3), np.float64)
    split = np.zeros((4, P, 3), np.float64) if want_split else None
    rho = np.zeros((P, max(cfg.max_depth - 1, 1)), np.float32) if want_rho else None
    stats = np.zeros(len(ST_NAMES), np.int64)
    rc = lib().orc_render(C.byref(s), C.byref(c), int(n_iter), _ptr(accum), _ptr(split), _ptr(rho), _ptr(stats))
    if rc != 0:
        raise RuntimeError(f"orc_render failed: {rc}")
    out = {"accum": accum.reshape(cfg.height, cfg.width, 3),
           "stats": dict(zip(ST_NAMES, stats.tolist())),
           "iter_seconds": iter_sec[:n_iter]}
    if want_split:
        out["split"] = split.reshape(4, cfg.height, cfg.width, 3)
    if want_rho:
        out["rho"] = rho
    if want_iterations:
        out["iterations"] = iters[:n_iter].reshape(n_iter, cfg.height, cfg.width, 3)
    return out


def bsdf_sample(mrow, n, wo, u, camera=True):
    """(ok, wi, weight, pdf, f) of one BSDF sample."""
    a = [np.ascontiguousarray(x, np.float32) for x in (mrow, n, wo, u)]
    wi = np.zeros(3, np.float32)
    w = np.zeros(3, np.float64)
    pdf = np.zeros(1, np.float64)
    f = np.zeros(3, np.float64)
    ok = lib().orc_bsdf_probe(*[_ptr(x) for x in a], int(camera), _ptr(wi), _ptr(w), _ptr(pdf), _ptr(f))
    return bool(ok), wi, w, float(pdf[0]), f


def bsdf_eval(mrow, n, wo, wi):
    a = [np.ascontiguousarray(x, np.float32) for x in (mrow, n, wo, wi)]
    f = np.zeros(3, np.float64)
    pdf = np.zeros(1, np.float64)
    lib().orc_bsdf_eval_probe(*[_ptr(x) for x in a], _ptr(f), _ptr(pdf))
    return f, float(pdf[0])
