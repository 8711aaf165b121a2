"""Seeded synthetic scenes for the Next Event Backtracking pass.

This module only produces input data: triangle soups, analytic spheres,
materials and a pinhole camera.  It holds none of the method's arithmetic and
is the one module shared by the CPU oracle and the CUDA library (both receive
the same plain arrays).  Scene randomness uses SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) so the
same seed gives the same scene on every machine.

Array conventions (all little-endian, C-contiguous):

* ``tri``      float32 [nt, 3, 3]  vertex positions v0, v1, v2 of each triangle.
                The geometric normal is normalize(cross(v1 - v0, v2 - v0)); an
                emissive triangle emits only on that side.
* ``tri_mat``  uint32  [nt]        material index per triangle.
* ``sph``      float32 [ns, 4]     centre xyz and radius of analytic spheres
                (spheres are pure emitters: black, emitting outward).
* ``sph_mat``  uint32  [ns]        material index per sphere.
* ``mats``     float32 [nm, 12]    type, albedo rgb, emission rgb, ior, alpha,
                pad x3.  type 0 = Lambertian (two-sided), 1 = smooth dielectric,
                2 = GGX rough conductor (albedo is the Schlick F0).
* ``cam``      float32 [10]        eye xyz, target xyz, up xyz, vertical FOV in
                degrees.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MAT_DIFFUSE = 0
MAT_DIELECTRIC = 1
MAT_GGX = 2


def material(mtype, albedo=(0.0, 0.0, 0.0), emission=(0.0, 0.0, 0.0), ior=1.0, alpha=0.0):
    m = np.zeros(12, np.float32)
    m[0] = mtype
    m[1:4] = albedo
    m[4:7] = emission
    m[7] = ior
    m[8] = alpha
    return m


@dataclasses.dataclass
class Scene:
    tri: np.ndarray
    tri_mat: np.ndarray
    sph: np.ndarray
    sph_mat: np.ndarray
    mats: np.ndarray
    cam: np.ndarray
    name: str = ""

    def __post_init__(self):
        self.tri = np.ascontiguousarray(self.tri, np.float32).reshape(-1, 3, 3)
        self.tri_mat = np.ascontiguousarray(self.tri_mat, np.uint32).reshape(-1)
        self.sph = np.ascontiguousarray(self.sph, np.float32).reshape(-1, 4)
        self.sph_mat = np.ascontiguousarray(self.sph_mat, np.uint32).reshape(-1)
        self.mats = np.ascontiguousarray(self.mats, np.float32).reshape(-1, 12)
        self.cam = np.ascontiguousarray(self.cam, np.float32).reshape(10)
        assert len(self.tri) == len(self.tri_mat)
        assert len(self.sph) == len(self.sph_mat)

    @property
    def n_tri(self):
        return len(self.tri)

    @property
    def n_sph(self):
        return len(self.sph)

    @property
    def n_emitters(self):
        """Primitives whose material emits (the light list of neb_scene_upload)."""
        emits = self.mats[:, 4:7].sum(axis=1) > 0.0
        return int(emits[self.tri_mat].sum() + emits[self.sph_mat].sum())


@dataclasses.dataclass
class RenderConfig:
    """Render settings of one workload (mirrors ``neb_config`` in include/neb.h)."""
    width: int
    height: int
    max_depth: int
    merge_radius: float
    octree_capacity: int
    split_factor: int
    iterations: int
    seed: int = 0
    octree_mode: int = 0        # 0 concurrent, 1 deterministic sequential insert
    density_mode: int = 0       # 0 robust median of five, 1 single query
    strategy_mask: int = 7      # bit 0 random hit (e), bit 1 NEE (E), bit 2 NEB photon merge (P),
                                # bit 3 conventional light-photon merge (LP, Sec. 6.1)
    lp_photons: int = 0         # light photons per iteration (n_LP) when bit 3 is set
    density_all: int = 0        # 1: evaluate rho at every NEE vertex, not only where a result uses it
    merge_mode: int = 0         # photon merge: 0 dense hits per cell, sparse per hit; 1 per hit; 2 per cell


class SplitMix64:
    """SplitMix64 stream; ``uniform`` returns doubles in [0, 1) from the top 53 bits."""

    def __init__(self, seed: int):
        self.state = seed & 0xFFFFFFFFFFFFFFFF

    def next_u64(self, n: int) -> np.ndarray:
        # Vectorised: state_i = seed + (i+1) * gamma, then the finaliser.
        gamma = np.uint64(0x9E3779B97F4A7C15)
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * gamma
            self.state = int((np.uint64(self.state) + np.uint64(n) * gamma))
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------
# geometry helpers (pure mesh construction)
# ----------------------------------------------------------------------------

def quad(p0, p1, p2, p3):
    """Two triangles (p0,p1,p2) and (p0,p2,p3); normal follows the p0->p1->p2 winding."""
    p0, p1, p2, p3 = (np.asarray(p, np.float64) for p in (p0, p1, p2, p3))
    return np.array([[p0, p1, p2], [p0, p2, p3]])


def ground_tiles(x0, z0, x1, z1, n, y=0.0):
    """n x n grid of +y facing quads covering [x0,x1] x [z0,z1] at height y.

    Large surfaces are tiled so that no triangle is far larger than the
    features around it (the FP32 ray/triangle error grows with triangle size)."""
    xs = np.linspace(x0, x1, n + 1)
    zs = np.linspace(z0, z1, n + 1)
    out = []
    for i in range(n):
        for j in range(n):
            out.append(quad((xs[i], y, zs[j]), (xs[i], y, zs[j + 1]), (xs[i + 1], y, zs[j + 1]),
                            (xs[i + 1], y, zs[j])))
    return np.concatenate(out, 0)


def box_faces(lo, hi, inward=False, faces=("x-", "x+", "y-", "y+", "z-", "z+")):
    """Triangles of an axis-aligned box; normals outward unless ``inward``."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    out = {
        "x-": quad((x0, y0, z0), (x0, y0, z1), (x0, y1, z1), (x0, y1, z0)),
        "x+": quad((x1, y0, z0), (x1, y1, z0), (x1, y1, z1), (x1, y0, z1)),
        "y-": quad((x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1)),
        "y+": quad((x0, y1, z0), (x0, y1, z1), (x1, y1, z1), (x1, y1, z0)),
        "z-": quad((x0, y0, z0), (x0, y1, z0), (x1, y1, z0), (x1, y0, z0)),
        "z+": quad((x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)),
    }
    tris = []
    for f in faces:
        t = out[f]
        if inward:
            t = t[:, ::-1, :]
        tris.append(t)
    return np.concatenate(tris, 0)


def icosphere(subdiv: int, centre, radius):
    """Icosphere with 20*4^subdiv triangles, outward winding."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius + np.asarray(centre, np.float64)
    return V[np.array(faces)]


def torus(n_major: int, n_minor: int, centre, R: float, r: float):
    """Torus around the +y axis with 2*n_major*n_minor triangles, outward winding."""
    i = np.arange(n_major)
    j = np.arange(n_minor)
    u = 2 * np.pi * i / n_major
    v = 2 * np.pi * j / n_minor
    U, Vv = np.meshgrid(u, v, indexing="ij")
    X = (R + r * np.cos(Vv)) * np.cos(U)
    Z = (R + r * np.cos(Vv)) * np.sin(U)
    Y = r * np.sin(Vv)
    P = np.stack([X, Y, Z], -1) + np.asarray(centre, np.float64)
    tris = []
    for a in range(n_major):
        a1 = (a + 1) % n_major
        for b in range(n_minor):
            b1 = (b + 1) % n_minor
            p00, p10, p01, p11 = P[a, b], P[a1, b], P[a, b1], P[a1, b1]
            tris.append((p00, p01, p11))
            tris.append((p00, p11, p10))
    T = np.array(tris)
    # orient outward: the normal must point away from the tube centre line
    e1 = T[:, 1] - T[:, 0]
    e2 = T[:, 2] - T[:, 0]
    n = np.cross(e1, e2)
    c = T.mean(1) - np.asarray(centre, np.float64)
    ring = c.copy()
    ring[:, 1] = 0
    ring *= (R / np.maximum(np.linalg.norm(ring, axis=1, keepdims=True), 1e-12))
    outward = (c - ring)
    flip = (n * outward).sum(1) < 0
    T[flip] = T[flip][:, ::-1]
    return T


def _camera(eye, target, up, vfov):
    return np.array(list(eye) + list(target) + list(up) + [vfov], np.float32)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def tiny_room(seed: int = 0) -> Scene:
    """Unit box open at z=0 with a glass icosphere and a small ceiling emitter.

    10 wall triangles (grey 0.7, left wall red, right wall green, as seen by the camera), a 0.05 x 0.05
    emitter of radiance 50 facing down from just below the ceiling, and an IOR
    1.5 icosphere (subdivision 3, 1280 triangles, radius 0.15) on the floor.
    """
    mats = np.stack([
        material(MAT_DIFFUSE, (0.7, 0.7, 0.7)),
        material(MAT_DIFFUSE, (0.7, 0.1, 0.1)),
        material(MAT_DIFFUSE, (0.1, 0.7, 0.1)),
        material(MAT_DIELECTRIC, ior=1.5),
        material(MAT_DIFFUSE, (0, 0, 0), emission=(50.0, 50.0, 50.0)),
    ])
    walls = []
    wmat = []
    # the camera looks down +z with +y up, so the x = 1 wall is on the left of the image
    for face, m in (("y-", 0), ("y+", 0), ("z+", 0), ("x+", 1), ("x-", 2)):
        walls.append(box_faces((0, 0, 0), (1, 1, 1), inward=True, faces=(face,)))
        wmat += [m, m]
    h = 0.025
    yl = 0.999
    emitter = quad((0.5 - h, yl, 0.5 - h), (0.5 + h, yl, 0.5 - h),
                   (0.5 + h, yl, 0.5 + h), (0.5 - h, yl, 0.5 + h))  # normal -y
    sphere = icosphere(3, (0.62, 0.15, 0.5), 0.15)
    tri = np.concatenate(walls + [emitter, sphere], 0)
    tri_mat = np.array(wmat + [4, 4] + [3] * len(sphere), np.uint32)
    cam = _camera((0.5, 0.5, -1.2), (0.5, 0.5, 0.5), (0, 1, 0), 45.0)
    return Scene(tri, tri_mat, np.zeros((0, 4)), np.zeros(0), mats, cam, "tiny_room")


def _city(seed: int, grid: int, n_albedo_levels: int = 256):
    rng = SplitMix64(seed)
    n = grid * grid
    heights = 0.5 + 19.5 * rng.uniform(n)
    alb = 0.2 + 0.6 * rng.uniform(n)
    level = np.minimum((alb - 0.2) / 0.6 * n_albedo_levels, n_albedo_levels - 1).astype(np.int64)
    mats = [material(MAT_DIFFUSE, (0.5, 0.5, 0.5))]
    for l in range(n_albedo_levels):
        a = 0.2 + 0.6 * (l + 0.5) / n_albedo_levels
        mats.append(material(MAT_DIFFUSE, (a, a, a)))
    ci, cj = grid // 2, grid // 2
    centre_cell = ci * grid + cj
    heights[centre_cell] = 5.0
    # ground
    g = float(grid)
    ground = ground_tiles(0.0, 0.0, g, g, 50)  # 5,000 triangles, normal +y
    # boxes: 12 triangles each, vectorised
    ii, jj = np.divmod(np.arange(n), grid)
    x0 = ii + 0.1
    x1 = ii + 0.9
    z0 = jj + 0.1
    z1 = jj + 0.9
    y0 = np.zeros(n)
    y1 = heights
    template = box_faces((0, 0, 0), (1, 1, 1))  # 12 tris in unit box, outward
    lo = np.stack([x0, y0, z0], -1)[:, None, None, :]
    ext = np.stack([x1 - x0, y1 - y0, z1 - z0], -1)[:, None, None, :]
    boxes = (lo + template[None] * ext).reshape(-1, 3, 3)
    tri = np.concatenate([ground, boxes], 0)
    tri_mat = np.concatenate([np.zeros(len(ground)), np.repeat(1 + level, 12)]).astype(np.uint32)
    top = float(heights[centre_cell])
    roof_tris = len(ground) + centre_cell * 12 + np.arange(12)
    return rng, tri, tri_mat, mats, (ci + 0.5, top, cj + 0.5), roof_tris


def _torus_and_camera(scene_diag, base):
    extent = scene_diag / 1000.0
    Rmaj = 0.2 / 0.283 * extent / 2.0
    rmin = 0.083 / 0.283 * extent / 2.0
    cx, top, cz = base
    centre = (cx, top + rmin, cz)
    T = torus(200, 50, centre, Rmaj, rmin)
    eye = (cx + 0.8 * extent, top + 1.0 * extent, cz + 1.3 * extent)
    cam = _camera(eye, (cx, top, cz), (0, 1, 0), 40.0)
    return T, centre, cam


def large_city(seed: int = 0, grid: int = 400, n_lights: int = 16) -> Scene:
    """400x400 grid of seeded boxes (~1.92M triangles) with a small glass torus.

    Box heights U[0.5, 20], grey albedo U[0.2, 0.8] (quantised to 256 levels),
    16 spherical lights of radius 0.05 with power log-uniform in [1e2, 1e4] at
    heights U[21, 40]; light 0 hangs 10 units above a glass torus (IOR 1.5,
    20,000 triangles) whose extent is 1/1000 of the scene diagonal and which
    sits on the roof of the centre box (height 5).  The camera looks at the
    torus and the caustic it throws onto the roof.
    """
    rng, tri, tri_mat, mats, base, _ = _city(seed, grid)
    diag = math.sqrt(grid * grid * 2 + 20.0 * 20.0)
    T, centre, cam = _torus_and_camera(diag, base)
    glass = len(mats)
    mats.append(material(MAT_DIELECTRIC, ior=1.5))
    tri = np.concatenate([tri, T], 0)
    tri_mat = np.concatenate([tri_mat, np.full(len(T), glass)]).astype(np.uint32)
    sph, sph_mat = _sphere_lights(rng, mats, n_lights, grid, (0.05, 0.05), centre)
    return Scene(tri, tri_mat, sph, sph_mat, np.stack(mats), cam, "large_city")


def _sphere_lights(rng, mats, n, grid, rrange, torus_centre):
    u = rng.uniform(n * 5).reshape(n, 5)
    pos = np.stack([u[:, 0] * grid, 21.0 + 19.0 * u[:, 1], u[:, 2] * grid], -1)
    pos[0] = (torus_centre[0], torus_centre[1] + 10.0, torus_centre[2])
    rad = rrange[0] + (rrange[1] - rrange[0]) * u[:, 3]
    power = 10.0 ** (2.0 + 2.0 * u[:, 4])
    le = power / (4.0 * math.pi * math.pi * rad * rad)
    base = len(mats)
    for i in range(n):
        mats.append(material(MAT_DIFFUSE, (0, 0, 0), emission=(le[i],) * 3))
    sph = np.concatenate([pos, rad[:, None]], 1)
    return sph, base + np.arange(n)


def many_lights(seed: int = 0, grid: int = 400, n_lights: int = 65536) -> Scene:
    """The large city with 65,536 sphere lights and a GGX (alpha 0.05) roof patch.

    Sphere radii U[0.01, 0.1], power log-uniform in [1e2, 1e4]; the roof of the
    centre box under the torus is a rough conductor with Schlick F0 = 0.9.
    """
    rng, tri, tri_mat, mats, base, roof = _city(seed, grid)
    diag = math.sqrt(grid * grid * 2 + 20.0 * 20.0)
    T, centre, cam = _torus_and_camera(diag, base)
    glass = len(mats)
    mats.append(material(MAT_DIELECTRIC, ior=1.5))
    ggx = len(mats)
    mats.append(material(MAT_GGX, (0.9, 0.9, 0.9), alpha=0.05))
    tri = np.concatenate([tri, T], 0)
    tri_mat = np.concatenate([tri_mat, np.full(len(T), glass)]).astype(np.uint32)
    # the roof quad of the centre box is the "+y" face: triangles 6,7 of its 12
    tri_mat[roof[6:8]] = ggx
    sph, sph_mat = _sphere_lights(rng, mats, n_lights, grid, (0.01, 0.1), centre)
    return Scene(tri, tri_mat, sph, sph_mat, np.stack(mats), cam, "many_lights")


# closed-form test scenes ------------------------------------------------------

def white_furnace(albedo: float = 0.5, le: float = 1.0) -> Scene:
    """Closed unit box, all 12 triangles Lambertian with albedo a and emission Le (inward)."""
    tri = box_faces((0, 0, 0), (1, 1, 1), inward=True)
    mats = np.stack([material(MAT_DIFFUSE, (albedo,) * 3, emission=(le,) * 3)])
    cam = _camera((0.5, 0.5, 0.3), (0.5, 0.5, 1.0), (0, 1, 0), 60.0)
    return Scene(tri, np.zeros(len(tri)), np.zeros((0, 4)), np.zeros(0), mats, cam, "white_furnace")


def plane_under_sphere(albedo=0.6, radius=0.1, height=1.0, le=5.0, half=50.0) -> Scene:
    """Lambertian plane y=0 (half-size ``half``) under one sphere light at (0, height, 0)."""
    tri = ground_tiles(-half, -half, half, half, 20)
    mats = np.stack([material(MAT_DIFFUSE, (albedo,) * 3),
                     material(MAT_DIFFUSE, (0, 0, 0), emission=(le,) * 3)])
    sph = np.array([[0.0, height, 0.0, radius]])
    cam = _camera((0.0, 0.6, -1.0), (0.0, 0.0, 0.3), (0, 1, 0), 50.0)
    return Scene(tri, np.zeros(len(tri)), sph, np.array([1]), mats, cam, "plane_under_sphere")


def glass_in_emitting_box(ior=1.5, radius=0.25, subdiv=3) -> Scene:
    """Closed box of black walls emitting Le = 1 around a glass icosphere."""
    walls = box_faces((0, 0, 0), (1, 1, 1), inward=True)
    ball = icosphere(subdiv, (0.5, 0.5, 0.6), radius)
    mats = np.stack([material(MAT_DIFFUSE, (0, 0, 0), emission=(1.0, 1.0, 1.0)),
                     material(MAT_DIELECTRIC, ior=ior)])
    tri = np.concatenate([walls, ball], 0)
    tri_mat = np.array([0] * len(walls) + [1] * len(ball), np.uint32)
    cam = _camera((0.5, 0.5, 0.05), (0.5, 0.5, 0.6), (0, 1, 0), 60.0)
    return Scene(tri, tri_mat, np.zeros((0, 4)), np.zeros(0), mats, cam, "glass_in_emitting_box")


def batch_jobs(n: int, seed: int = 0, iterations: int = 64):
    """A seeded mix of n heterogeneous render jobs, [(scene, RenderConfig)].

    A quarter are the room of the tiny-room workload (1,292 triangles, a
    two-triangle emitter, D = 8, r = 0.01, split 8), the rest cities of the large-city
    generator with a grid of g x g boxes, g log-uniform in [9, 200] (~26k to
    ~500k triangles with the torus and ground), 1 to 64 sphere lights
    (log-uniform), D = 10, r = 1e-3 of the torus extent, split 4.  Image sides
    are log-uniform in [128, 1024] (multiples of 16, square); octree capacity
    4 nodes per pixel, within [2^16, 2^22].  Job i renders with Philox seed i.
    """
    rng = SplitMix64(0xBA7C4 + 7919 * seed)
    u = rng.uniform(4 * n).reshape(n, 4)
    out = []
    for i in range(n):
        side = int(round(128.0 * 8.0 ** u[i, 1] / 16.0)) * 16
        cap = int(min(1 << 22, max(1 << 16, 4 * side * side)))
        if u[i, 0] < 0.25:
            sc = tiny_room()
            rc = RenderConfig(side, side, 8, 0.01, cap, 8, iterations, seed=i)
        else:
            grid = int(round(9.0 * (200.0 / 9.0) ** u[i, 3]))
            n_lights = int(round(64.0 ** u[i, 2]))
            sc = large_city(seed=i + 1, grid=grid, n_lights=n_lights)
            torus_extent = math.sqrt(grid * grid * 2 + 400.0) / 1000.0
            rc = RenderConfig(side, side, 10, 1e-3 * torus_extent, cap, 4, iterations, seed=i)
        out.append((sc, rc))
    return out


def workload(name: str):
    """(scene, RenderConfig) of a named workload."""
    if name == "tiny_room":
        return tiny_room(), RenderConfig(64, 64, 8, 0.01, 1 << 16, 8, 4)
    if name == "large_city":
        s = large_city()
        torus_extent = math.sqrt(400 * 400 * 2 + 400.0) / 1000.0
        return s, RenderConfig(1280, 720, 10, 1e-3 * torus_extent, 4 << 20, 4, 64)
    if name == "many_lights":
        s = many_lights()
        torus_extent = math.sqrt(400 * 400 * 2 + 400.0) / 1000.0
        return s, RenderConfig(1920, 1080, 10, 1e-3 * torus_extent, 4 << 20, 4, 32)
    raise KeyError(name)
