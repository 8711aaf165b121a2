"""Thin ctypes binding of libneb.so (C ABI in include/neb.h).

Argument marshalling only: every step of the NEB iteration runs in the CUDA
kernels of the library.  There is no CPU fallback; if the library cannot be
loaded the import of :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libneb.so")

NEB_OK = 0
ERRORS = {-1: "NEB_ERR_ARG", -2: "NEB_ERR_OOM", -3: "NEB_ERR_CUDA", -4: "NEB_ERR_DEVICE_TIMEOUT",
          -5: "NEB_ERR_QUEUE_OVERFLOW", -6: "NEB_ERR_NO_DEVICE"}
STATUS_SPIN_TIMEOUT, STATUS_QUEUE_OVERFLOW, STATUS_STACK_OVERFLOW, STATUS_OCTREE_FULL = 1, 2, 4, 8
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_QUEUE_OVERFLOW, ERR_NO_DEVICE = -1, -2, -3, -4, -5, -6

# every function declared in include/neb.h
EXPORTS = ["neb_create", "neb_destroy", "neb_last_error", "neb_scene_upload", "neb_build_bvh", "neb_iterate",
           "neb_resolve", "neb_read_accum", "neb_read_split", "neb_read_nee_rho", "neb_get_stats",
           "neb_set_profiling", "neb_get_stage_times", "neb_trace_closest", "neb_philox", "neb_plane_box_area",
           "neb_octree_create", "neb_octree_destroy", "neb_octree_set_iteration", "neb_octree_insert",
           "neb_octree_density", "neb_octree_read", "neb_octree_load", "neb_count_neighbours",
           "neb_count_neighbours_noalloc", "neb_iterate_batch", "neb_job_device_bytes", "neb_get_tuning",
           "neb_set_tuning", "neb_autotune", "neb_density_estimators", "neb_read_nee_vertices",
           "neb_iterate_read", "neb_bvh_cost", "neb_error_estimate", "neb_synchronize"]
NOALLOC_MAX_POINTS = 1 << 18


class NebError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("max_depth", C.c_int), ("merge_radius", C.c_float),
                ("octree_capacity", C.c_int), ("split_factor", C.c_int), ("seed", C.c_uint64),
                ("octree_mode", C.c_int), ("density_mode", C.c_int), ("strategy_mask", C.c_uint32),
                ("keep_split", C.c_int), ("bvh_builder", C.c_int), ("photon_records", C.c_int),
                ("lp_photons", C.c_int), ("density_all", C.c_int), ("merge_mode", C.c_int),
                ("merge_hits", C.c_int)]


class Tuning(C.Structure):
    _fields_ = [("cam_origin_bits", C.c_int), ("cam_dir_bits", C.c_int), ("shadow_origin_bits", C.c_int),
                ("shadow_light_bits", C.c_int), ("shade_blocks_per_sm", C.c_int), ("photon_grouping", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("camera_rays", C.c_int64), ("nee_vertices", C.c_int64),
                ("shadow_rays", C.c_int64), ("photons", C.c_int64), ("photon_hits", C.c_int64),
                ("merge_tests", C.c_int64), ("merges", C.c_int64), ("random_hits", C.c_int64),
                ("octree_inserts", C.c_int64), ("octree_queries", C.c_int64), ("bvh_node_visits", C.c_int64),
                ("prim_tests", C.c_int64), ("kernel_launches", C.c_int64),
                ("stage_node_visits", C.c_int64 * 3), ("stage_prim_tests", C.c_int64 * 3),
                ("octree_nodes", C.c_int32), ("octree_depth", C.c_int32),
                ("status", C.c_uint32), ("pad", C.c_int32), ("merge_hits_staged", C.c_int64)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            if k == "pad":
                continue
            v = getattr(self, k)
            d[k] = list(v) if k.startswith("stage_") else v
        return d


_lib = None
vp = C.c_void_p


def lib():
    """Loads libneb.so (built by paper_1909_00573_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libneb.so not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        sig = {
            "neb_create": ([C.POINTER(Config), vp, C.POINTER(vp)], C.c_int),
            "neb_destroy": ([vp], None),
            "neb_last_error": ([vp], C.c_char_p),
            "neb_scene_upload": ([vp, vp, vp, C.c_int, vp, vp, C.c_int, vp, C.c_int, vp], C.c_int),
            "neb_build_bvh": ([vp], C.c_int),
            "neb_iterate": ([vp, C.c_int], C.c_int),
            "neb_iterate_read": ([vp, C.c_int, vp], C.c_int),
            "neb_bvh_cost": ([vp, vp], C.c_int),
            "neb_resolve": ([vp, vp, C.c_int], C.c_int),
            "neb_read_accum": ([vp, vp], C.c_int),
            "neb_error_estimate": ([vp, vp], C.c_int),
            "neb_synchronize": ([vp], C.c_int),
            "neb_read_split": ([vp, vp], C.c_int),
            "neb_read_nee_rho": ([vp, vp], C.c_int),
            "neb_get_stats": ([vp, C.POINTER(Stats)], C.c_int),
            "neb_set_profiling": ([vp, C.c_int], C.c_int),
            "neb_get_stage_times": ([vp, vp, vp, vp, C.c_int], C.c_int),
            "neb_trace_closest": ([vp, vp, C.c_int, vp, vp], C.c_int),
            "neb_philox": ([vp, C.c_int, vp, vp], C.c_int),
            "neb_plane_box_area": ([vp, vp, vp, C.c_int, vp], C.c_int),
            "neb_octree_create": ([vp, vp, C.c_int, C.c_int, vp, C.POINTER(vp)], C.c_int),
            "neb_octree_destroy": ([vp], None),
            "neb_octree_set_iteration": ([vp, C.c_int], C.c_int),
            "neb_octree_insert": ([vp, vp, C.c_int, C.c_int], C.c_int),
            "neb_octree_density": ([vp, vp, vp, C.c_int, C.c_int, vp], C.c_int),
            "neb_octree_read": ([vp, vp, C.c_int, vp], C.c_int),
            "neb_octree_load": ([vp, vp, C.c_int, C.c_int, C.c_int], C.c_int),
            "neb_iterate_batch": ([vp, C.c_int, C.c_int], C.c_int),
            "neb_get_tuning": ([vp, vp], C.c_int),
            "neb_set_tuning": ([vp, vp], C.c_int),
            "neb_autotune": ([vp, C.c_int, vp], C.c_int),
            "neb_density_estimators": ([vp, vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_float, C.c_int, vp, vp],
                                       C.c_int),
            "neb_read_nee_vertices": ([vp, vp, vp, C.c_int, vp], C.c_int),
            "neb_job_device_bytes": ([vp, C.c_int, C.c_int, C.c_int, C.c_int, vp], C.c_int),
            "neb_count_neighbours": ([vp, C.c_int, vp, C.c_int, C.c_float, vp], C.c_int),
            "neb_count_neighbours_noalloc": ([vp, C.c_int, vp, C.c_int, C.c_float, vp, vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(vp)


def _check(rc, ctx=None):
    if rc != NEB_OK:
        msg = lib().neb_last_error(ctx).decode() if ctx else ""
        raise NebError(rc, msg)


def make_config(rc, keep_split=False, octree_mode=None, density_mode=None, strategy_mask=None, bvh_builder=0,
                photon_records=0, merge_mode=None, merge_hits=0):
    """neb_config from a scenes.RenderConfig."""
    return Config(rc.width, rc.height, rc.max_depth, rc.merge_radius, rc.octree_capacity, rc.split_factor,
                  rc.seed, rc.octree_mode if octree_mode is None else octree_mode,
                  rc.density_mode if density_mode is None else density_mode,
                  rc.strategy_mask if strategy_mask is None else strategy_mask, int(keep_split), int(bvh_builder),
                  int(photon_records), int(getattr(rc, "lp_photons", 0)), int(getattr(rc, "density_all", 0)),
                  int(getattr(rc, "merge_mode", 0) if merge_mode is None else merge_mode), int(merge_hits))


class Context:
    """One NEB render context (neb_ctx) bound to a CUDA stream."""

    def __init__(self, cfg: Config, stream: int | None = None):
        self.cfg = cfg
        h = vp()
        _check(lib().neb_create(C.byref(cfg), vp(stream) if stream else None, C.byref(h)))
        self.h = h
        self.P = cfg.width * cfg.height

    def close(self):
        if getattr(self, "h", None):
            lib().neb_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, rc):
        _check(rc, self.h)

    def scene_upload(self, scene):
        keep = [np.ascontiguousarray(scene.tri, np.float32), np.ascontiguousarray(scene.tri_mat, np.uint32),
                np.ascontiguousarray(scene.sph, np.float32), np.ascontiguousarray(scene.sph_mat, np.uint32),
                np.ascontiguousarray(scene.mats, np.float32), np.ascontiguousarray(scene.cam, np.float32)]
        self._c(lib().neb_scene_upload(self.h, _p(keep[0]), _p(keep[1]), len(keep[1]), _p(keep[2]), _p(keep[3]),
                                       len(keep[3]), _p(keep[4]), len(keep[4]), _p(keep[5])))

    def build_bvh(self):
        self._c(lib().neb_build_bvh(self.h))

    def iterate(self, n=1):
        self._c(lib().neb_iterate(self.h, int(n)))

    def bvh_cost(self):
        """(expected node visits, expected primitive tests) of the built tree by the surface area heuristic."""
        out = np.zeros(2, np.float64)
        self._c(lib().neb_bvh_cost(self.h, _p(out)))
        return float(out[0]), float(out[1])

    def iterate_read(self, n, rgb_host_ptr):
        """n iterations, the running image copied to host memory at rgb_host_ptr
        ([H][W][3] float32, preferably pinned) after each; asynchronous: read
        the buffer only after synchronising the context stream."""
        self._c(lib().neb_iterate_read(self.h, int(n), vp(rgb_host_ptr)))

    def read_nee_vertices(self):
        n = C.c_int(0)
        self._c(lib().neb_read_nee_vertices(self.h, None, None, 0, C.byref(n)))
        pos = np.zeros((n.value, 3), np.float32)
        nrm = np.zeros((n.value, 3), np.float32)
        self._c(lib().neb_read_nee_vertices(self.h, _p(pos), _p(nrm), n.value, C.byref(n)))
        return pos, nrm

    def tuning(self):
        t = Tuning()
        self._c(lib().neb_get_tuning(self.h, C.byref(t)))
        return t

    def set_tuning(self, t):
        self._c(lib().neb_set_tuning(self.h, C.byref(t)))

    def autotune(self, iterations_per_candidate=2):
        t = Tuning()
        self._c(lib().neb_autotune(self.h, int(iterations_per_candidate), C.byref(t)))
        return t

    def resolve(self, out_device_ptr: int | None = None):
        if out_device_ptr is not None:
            self._c(lib().neb_resolve(self.h, vp(out_device_ptr), 1))
            return None
        out = np.zeros((self.cfg.height, self.cfg.width, 3), np.float32)
        self._c(lib().neb_resolve(self.h, _p(out), 0))
        return out

    def read_accum(self):
        out = np.zeros((self.cfg.height, self.cfg.width, 3), np.float64)
        self._c(lib().neb_read_accum(self.h, _p(out)))
        return out

    def synchronize(self):
        """Wait for this context's enqueued work only."""
        self._c(lib().neb_synchronize(self.h))

    def error_estimate(self):
        """Relative RMSE of the current image from its even and odd iterations (needs two or more)."""
        out = np.zeros(1, np.float64)
        self._c(lib().neb_error_estimate(self.h, _p(out)))
        return float(out[0])

    def read_split(self):
        out = np.zeros((4, self.cfg.height, self.cfg.width, 3), np.float64)
        self._c(lib().neb_read_split(self.h, _p(out)))
        return out

    def read_nee_rho(self):
        out = np.zeros((self.P, max(self.cfg.max_depth - 1, 1)), np.float32)
        self._c(lib().neb_read_nee_rho(self.h, _p(out)))
        return out

    def stats(self, check=True):
        s = Stats()
        rc = lib().neb_get_stats(self.h, C.byref(s))
        if check:
            self._c(rc)
        return s.as_dict()

    def set_profiling(self, on=True):
        self._c(lib().neb_set_profiling(self.h, int(on)))

    def stage_times(self):
        ms = np.zeros(32, np.float64)
        n_l = np.zeros(32, np.int64)
        names = C.create_string_buffer(32 * 32)
        n = lib().neb_get_stage_times(self.h, _p(ms), _p(n_l), names, 32)
        raw = names.raw
        return {raw[32 * i:32 * i + 32].split(b"\0")[0].decode(): (float(ms[i]), int(n_l[i])) for i in range(n)}

    def trace_closest(self, rays):
        R = np.ascontiguousarray(rays, np.float32).reshape(-1, 6)
        prim = np.zeros(len(R), np.int32)
        t = np.zeros(len(R), np.float32)
        self._c(lib().neb_trace_closest(self.h, _p(R), len(R), _p(prim), _p(t)))
        return prim, t


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32).reshape(2)
    out = np.zeros_like(c)
    _check(lib().neb_philox(_p(c), len(c), _p(k), _p(out)))
    return out


def plane_box_area(boxes, pos, nrm):
    b = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
    p = np.ascontiguousarray(pos, np.float32).reshape(-1, 3)
    n = np.ascontiguousarray(nrm, np.float32).reshape(-1, 3)
    out = np.zeros(len(b), np.float64)
    _check(lib().neb_plane_box_area(_p(b), _p(p), _p(n), len(b), _p(out)))
    return out


def count_neighbours(points, queries, r):
    P = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    Q = np.ascontiguousarray(queries, np.float32).reshape(-1, 3)
    out = np.zeros(len(Q), np.int32)
    _check(lib().neb_count_neighbours(_p(P), len(P), _p(Q), len(Q), C.c_float(r), _p(out)))
    return out


def count_neighbours_noalloc(d_points: int, n: int, d_queries: int, m: int, r: float, d_out: int,
                             stream: int = 0):
    """Allocation-free neighbour count on caller-owned device buffers (raw
    device pointers); enqueues on `stream` and returns without synchronising."""
    _check(lib().neb_count_neighbours_noalloc(vp(d_points), int(n), vp(d_queries), int(m), C.c_float(r),
                                              vp(d_out), vp(stream) if stream else None))


class Octree:
    """Stand-alone device density octree (neb_octree_*)."""

    def __init__(self, scene_min, scene_max, capacity, split_factor, stream=None):
        self._mn = np.ascontiguousarray(scene_min, np.float32)
        self._mx = np.ascontiguousarray(scene_max, np.float32)
        h = vp()
        _check(lib().neb_octree_create(_p(self._mn), _p(self._mx), int(capacity), int(split_factor),
                                       vp(stream) if stream else None, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().neb_octree_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_iteration(self, it):
        _check(lib().neb_octree_set_iteration(self.h, int(it)))

    def insert(self, positions, mode=0):
        P = np.ascontiguousarray(positions, np.float32).reshape(-1, 3)
        rc = lib().neb_octree_insert(self.h, _p(P), len(P), int(mode))
        _check(rc)

    def density(self, positions, normals, robust=True):
        P = np.ascontiguousarray(positions, np.float32).reshape(-1, 3)
        N = np.ascontiguousarray(normals, np.float32).reshape(-1, 3)
        out = np.zeros(len(P), np.float32)
        _check(lib().neb_octree_density(self.h, _p(P), _p(N), len(P), int(robust), _p(out)))
        return out

    def read(self):
        meta = np.zeros(4, np.int32)
        _check(lib().neb_octree_read(self.h, None, 0, _p(meta)))
        nodes = np.zeros(int(meta[2]), np.int32)
        _check(lib().neb_octree_read(self.h, _p(nodes), len(nodes), _p(meta)))
        return nodes, int(meta[0]), int(meta[1]), int(meta[3])

    def load(self, nodes, alloc, depth):
        N = np.ascontiguousarray(nodes, np.int32)
        _check(lib().neb_octree_load(self.h, _p(N), len(N), int(alloc), int(depth)))


def density_estimators(pos, nrm, scene_min, scene_max, octree_capacity, split_factor, radius, k):
    """neb_density_estimators: rho[3][n] (octree, naive, k nearest) and the
    device milliseconds of each (structure build plus queries)."""
    P = np.ascontiguousarray(pos, np.float32).reshape(-1, 3)
    N = np.ascontiguousarray(nrm, np.float32).reshape(-1, 3)
    lo = np.ascontiguousarray(scene_min, np.float32)
    hi = np.ascontiguousarray(scene_max, np.float32)
    rho = np.zeros((3, len(P)), np.float32)
    ms = np.zeros(3, np.float64)
    _check(lib().neb_density_estimators(_p(P), _p(N), len(P), _p(lo), _p(hi), int(octree_capacity),
                                        int(split_factor), float(radius), int(k), _p(rho), _p(ms)))
    return rho, ms


def iterate_batch(contexts, n_iterations):
    """Batched jobs (neb_iterate_batch): n_iterations iterations of every
    context, enqueued round-robin so the jobs overlap on the GPU."""
    arr = (vp * max(len(contexts), 1))(*[c.h for c in contexts])
    rc = lib().neb_iterate_batch(arr, len(contexts), int(n_iterations))
    _check(rc, contexts[0].h if (rc != NEB_OK and contexts) else None)


def job_device_bytes(cfg: "Config", n_tri, n_sph, n_mat, n_lights):
    """Device bytes a job keeps resident (neb_job_device_bytes)."""
    out = C.c_uint64(0)
    _check(lib().neb_job_device_bytes(C.byref(cfg), int(n_tri), int(n_sph), int(n_mat), int(n_lights),
                                      C.byref(out)))
    return int(out.value)


def render(scene, rc, n_iter=None, keep_split=True, stream=None, **over):
    """Convenience: upload, build the BVH and run n_iter iterations; returns the context."""
    ctx = Context(make_config(rc, keep_split=keep_split, **over), stream)
    ctx.scene_upload(scene)
    ctx.build_bvh()
    ctx.iterate(rc.iterations if n_iter is None else n_iter)
    return ctx
