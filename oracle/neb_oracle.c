/*
 * neb_oracle.c -- plain, single-threaded CPU oracle of the Next Event
 * Backtracking iteration.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product path.
 *
 * What it computes, in the paper's order (Sec. 3 outline, Fig. 2):
 *   pass 1  trace view paths; every vertex at which NEE is attempted is an
 *           NEE vertex, stored and counted in the density octree (Sec. 3.1,
 *           Sec. 5.1); random hits of emitters are stored (Sec. 3.1).
 *   pass 2  (a) density rho at every NEE vertex (Eq. octdensity, the robust
 *           median of five queries); (b) NEE contribution L_E (Sec. 3.2);
 *           (c) photon Phi = dE / rho (Eq. flux) walked from the NEE vertex,
 *           merged at view vertices found by a range search around each
 *           photon hit (Sec. 3.2, uniform kernel 1/(pi r^2)).
 *   pass 3  self emission L_e of the stored random hits (Sec. 3.3).
 * MIS: balance heuristic (Eq. misweight) over the random hit, the NEE and the
 * NEB photon merges of each path (Eq. rhpdf, Eq. neepdf, Eq. photonpdf,
 * Eq. misw), evaluated explicitly from the full vertex list of the path.
 *
 * Readings where the paper is silent (all shared with the CUDA path by
 * definition, not by code):
 *  - every view vertex x_k (1 <= k <= D-1) on a non-black surface is an NEE
 *    vertex and is counted in the octree, whatever the shadow ray says and
 *    also on delta (glass) surfaces; photons leave only where dE > 0, rho > 0.
 *  - a directional pdf at a delta vertex is taken as 1 in both directions:
 *    the true value (lobe probability times a Dirac) is common to every
 *    strategy that can create the path and cancels; NEE at a delta vertex and
 *    merges at delta vertices have pdf 0.
 *  - the camera factor p_{0->1} is 1 (it is common to all strategies).
 *  - merges: 3D ball, accept d^2 <= r^2 in FP32, photon hits j >= 1 on
 *    non-delta surfaces, view vertices 1 <= k <= D-2, k + j + 1 <= D.
 *  - geometric normals only; refraction scales camera throughput by
 *    (eta_i/eta_t)^2 and leaves photon flux unscaled.
 *  - random numbers: Philox4x32-10 keyed by the seed, counter (pixel, stream,
 *    dim/4, iteration); stream = 256*k for view vertex k, 256*k + 1 + s for
 *    the s-th scattering of the photon leaving NEE vertex k.
 */
#define _POSIX_C_SOURCE 199309L
#include "neb_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

static double now_seconds(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

#define PI_D 3.14159265358979323846
#define ORC_LP_STREAM 0x40000000u /* Philox stream of light photon i: + bounce */
#define TWO_PI_F 6.28318530717958647692f
#define INV_PI_F 0.318309886183790671538f

/* ------------------------------------------------------------------------ */
/* small vector helpers (FP32 geometry, FP64 colour)                         */
/* ------------------------------------------------------------------------ */
typedef struct { float x, y, z; } v3;
typedef struct { double r, g, b; } c3;

static v3 mk3(float x, float y, float z) { v3 v; v.x = x; v.y = y; v.z = z; return v; }
static v3 vadd(v3 a, v3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 vsub(v3 a, v3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 vmul(v3 a, float s) { return mk3(a.x * s, a.y * s, a.z * s); }
static v3 vneg(v3 a) { return mk3(-a.x, -a.y, -a.z); }
static float vdot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 vcross(v3 a, v3 b) {
  return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static v3 vnorm(v3 a) { float l = sqrtf(vdot(a, a)); float inv = 1.0f / l; return vmul(a, inv); }
static float vget(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
static v3 vload(const float* p) { return mk3(p[0], p[1], p[2]); }

static c3 ck(double r, double g, double b) { c3 c; c.r = r; c.g = g; c.b = b; return c; }
static c3 cmul(c3 a, c3 b) { return ck(a.r * b.r, a.g * b.g, a.b * b.b); }
static c3 cscale(c3 a, double s) { return ck(a.r * s, a.g * s, a.b * s); }
static double cmax(c3 a) { return fmax(a.r, fmax(a.g, a.b)); }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its      */
/* published definition: 10 rounds of two 32x32->64 multiplies with a Weyl  */
/* key schedule.                                                             */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3v = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3v ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3v = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3v;
}

typedef struct { uint32_t key[2]; uint32_t iter; } rng_t;

static uint32_t rng_raw(const rng_t* g, uint32_t pixel, uint32_t stream, uint32_t dim) {
  uint32_t ctr[4] = {pixel, stream, dim >> 2, g->iter};
  uint32_t out[4];
  orc_philox4x32_10(ctr, g->key, out);
  return out[dim & 3u];
}
static float u01(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }
static float rng_u(const rng_t* g, uint32_t pixel, uint32_t stream, uint32_t dim) {
  return u01(rng_raw(g, pixel, stream, dim));
}

/* ------------------------------------------------------------------------ */
/* orthonormal basis: Duff et al. 2017, "Building an Orthonormal Basis,     */
/* Revisited" (JCGT 6(1)).                                                   */
/* ------------------------------------------------------------------------ */
static void onb(v3 n, v3* t, v3* b) {
  float sign = copysignf(1.0f, n.z);
  float a = -1.0f / (sign + n.z);
  float bb = n.x * n.y * a;
  *t = mk3(1.0f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
  *b = mk3(bb, sign + n.y * n.y * a, -n.y);
}
static v3 from_local(v3 n, float lx, float ly, float lz) {
  v3 t, b;
  onb(n, &t, &b);
  return vadd(vadd(vmul(t, lx), vmul(b, ly)), vmul(n, lz));
}

/* ------------------------------------------------------------------------ */
/* scene, lights, alias table (Vose 1991)                                     */
/* ------------------------------------------------------------------------ */
enum { MT_DIFFUSE = 0, MT_DIELECTRIC = 1, MT_GGX = 2 };

typedef struct {
  int type;
  float albedo[3], emission[3];
  float ior, alpha;
} mat_t;

typedef struct {
  int kind;      /* 0 triangle, 1 sphere */
  int prim;      /* primitive index (triangles first, then spheres) */
  double power, psel;
  float area;
} light_t;

typedef struct {
  int nt, ns, nprim;
  const float* tri;
  const float* sph;
  int* prim_mat;
  mat_t* mats;
  int nm;
  int nl;
  light_t* lights;
  float* alias_prob;
  int* alias_idx;
  int* prim_light;
  float bmin[3], bmax[3];
} scene_t;

static double mean3(const float* e) { return ((double)e[0] + (double)e[1] + (double)e[2]) / 3.0; }

/* Vose's alias table (Vose 1991) for choosing item i with probability
 * w_i / sum w: cell i keeps i with probability prob[i] and otherwise gives
 * alias[i]; cells start at n w_i / sum w, and each cell below 1 is paired with
 * one above 1, which gives up the difference. */
static void alias_build(const double* w, int n, double* psel, float* prob, int* alias) {
  double total = 0.0;
  for (int i = 0; i < n; ++i) total += w[i];
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  int* small = (int*)malloc(sizeof(int) * (size_t)n);
  int* large = (int*)malloc(sizeof(int) * (size_t)n);
  int ns = 0, nl = 0;
  for (int i = 0; i < n; ++i) {
    psel[i] = w[i] / total;
    p[i] = w[i] * (double)n / total;
    alias[i] = i;
    if (p[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  while (ns > 0 && nl > 0) {
    int l = small[--ns];
    int g = large[--nl];
    prob[l] = (float)p[l];
    alias[l] = g;
    p[g] = (p[g] + p[l]) - 1.0;
    if (p[g] < 1.0) small[ns++] = g; else large[nl++] = g;
  }
  while (nl > 0) { int g = large[--nl]; prob[g] = 1.0f; }
  while (ns > 0) { int l = small[--ns]; prob[l] = 1.0f; }
  free(p); free(small); free(large);
}

/* Item chosen by the random word x0 (cell: its top 24 bits scaled to n) and
 * the uniform ua (keep the cell or take its alias). */
static int alias_pick(const float* prob, const int* alias, int n, uint32_t x0, float ua) {
  int i = (int)(((uint64_t)(x0 >> 8) * (uint64_t)n) >> 24);
  return ua < prob[i] ? i : alias[i];
}

static void build_alias(scene_t* s) {
  int n = s->nl;
  s->alias_prob = (float*)calloc(n > 0 ? n : 1, sizeof(float));
  s->alias_idx = (int*)calloc(n > 0 ? n : 1, sizeof(int));
  if (n == 0) return;
  double* w = (double*)calloc((size_t)n, sizeof(double));
  double* psel = (double*)calloc((size_t)n, sizeof(double));
  for (int i = 0; i < n; ++i) w[i] = s->lights[i].power;
  alias_build(w, n, psel, s->alias_prob, s->alias_idx);
  for (int i = 0; i < n; ++i) s->lights[i].psel = psel[i];
  free(w); free(psel);
}

static v3 tri_v(const scene_t* s, int t, int k) { return vload(s->tri + (size_t)t * 9 + k * 3); }

static v3 prim_normal(const scene_t* s, int prim, v3 p) {
  if (prim < s->nt) {
    v3 a = tri_v(s, prim, 0), b = tri_v(s, prim, 1), c = tri_v(s, prim, 2);
    return vnorm(vcross(vsub(b, a), vsub(c, a)));
  }
  const float* sp = s->sph + (size_t)(prim - s->nt) * 4;
  return vnorm(vsub(p, vload(sp)));
}

static int scene_init(scene_t* s, const orc_scene* in) {
  memset(s, 0, sizeof(*s));
  s->nt = in->nt; s->ns = in->ns; s->nprim = in->nt + in->ns;
  s->tri = in->tri; s->sph = in->sph;
  s->nm = in->nm;
  s->mats = (mat_t*)calloc(in->nm > 0 ? in->nm : 1, sizeof(mat_t));
  for (int i = 0; i < in->nm; ++i) {
    const float* m = in->mats + (size_t)i * 12;
    s->mats[i].type = (int)m[0];
    for (int c = 0; c < 3; ++c) { s->mats[i].albedo[c] = m[1 + c]; s->mats[i].emission[c] = m[4 + c]; }
    s->mats[i].ior = m[7];
    s->mats[i].alpha = m[8];
  }
  s->prim_mat = (int*)malloc(sizeof(int) * (s->nprim > 0 ? s->nprim : 1));
  for (int i = 0; i < s->nt; ++i) s->prim_mat[i] = (int)in->tri_mat[i];
  for (int i = 0; i < s->ns; ++i) s->prim_mat[s->nt + i] = (int)in->sph_mat[i];
  s->prim_light = (int*)malloc(sizeof(int) * (s->nprim > 0 ? s->nprim : 1));
  s->lights = (light_t*)calloc(s->nprim > 0 ? s->nprim : 1, sizeof(light_t));
  s->nl = 0;
  for (int i = 0; i < s->nprim; ++i) {
    s->prim_light[i] = -1;
    const mat_t* m = &s->mats[s->prim_mat[i]];
    double le = mean3(m->emission);
    if (le <= 0.0) continue;
    light_t L;
    memset(&L, 0, sizeof(L));
    L.prim = i;
    if (i < s->nt) {
      v3 a = tri_v(s, i, 0), b = tri_v(s, i, 1), c = tri_v(s, i, 2);
      v3 cr = vcross(vsub(b, a), vsub(c, a));
      double area = 0.5 * sqrt((double)cr.x * cr.x + (double)cr.y * cr.y + (double)cr.z * cr.z);
      L.kind = 0;
      L.area = (float)area;
      L.power = PI_D * area * le;
    } else {
      double R = s->sph[(size_t)(i - s->nt) * 4 + 3];
      L.kind = 1;
      L.area = (float)(4.0 * PI_D * R * R);
      L.power = 4.0 * PI_D * PI_D * R * R * le;
    }
    s->prim_light[i] = s->nl;
    s->lights[s->nl++] = L;
  }
  build_alias(s);
  for (int c = 0; c < 3; ++c) { s->bmin[c] = FLT_MAX; s->bmax[c] = -FLT_MAX; }
  for (int i = 0; i < s->nt * 3; ++i)
    for (int c = 0; c < 3; ++c) {
      float v = s->tri[(size_t)i * 3 + c];
      if (v < s->bmin[c]) s->bmin[c] = v;
      if (v > s->bmax[c]) s->bmax[c] = v;
    }
  for (int i = 0; i < s->ns; ++i)
    for (int c = 0; c < 3; ++c) {
      float ce = s->sph[(size_t)i * 4 + c], r = s->sph[(size_t)i * 4 + 3];
      if (ce - r < s->bmin[c]) s->bmin[c] = ce - r;
      if (ce + r > s->bmax[c]) s->bmax[c] = ce + r;
    }
  return 0;
}

static void scene_free(scene_t* s) {
  free(s->mats); free(s->prim_mat); free(s->prim_light); free(s->lights);
  free(s->alias_prob); free(s->alias_idx);
}

/* ------------------------------------------------------------------------ */
/* ray / primitive intersection (FP32, as the renderer traces its rays)      */
/* ------------------------------------------------------------------------ */
/* gamma_n = n u / (1 - n u), u = 2^-24: bound on the relative rounding error
 * of n chained FP32 operations (Pharr, Jakob, Humphreys, PBRT 3rd ed.,
 * Sec. 3.9.1). */
static float gamma_f32(int n) {
  double u = ldexp(1.0, -24);
  return (float)((double)n * u / (1.0 - (double)n * u));
}

typedef struct {
  v3 o, d;
  int k[3];          /* k[2]: axis of the largest |d| component (lowest on ties); k[0], k[1] the others, in winding order */
  float shear[3];    /* d[k0] / d[k2], d[k1] / d[k2], 1 / d[k2] */
} ray_t;

static ray_t make_ray(v3 o, v3 d) {
  ray_t r;
  r.o = o;
  r.d = d;
  const float dd[3] = {d.x, d.y, d.z};
  int z = 0;
  for (int i = 1; i < 3; ++i)
    if (fabsf(dd[i]) > fabsf(dd[z])) z = i;
  r.k[0] = (z + 1) % 3;
  r.k[1] = (z + 2) % 3;
  r.k[2] = z;
  if (dd[z] < 0.0f) { int t = r.k[0]; r.k[0] = r.k[1]; r.k[1] = t; }
  r.shear[0] = dd[r.k[0]] / dd[z];
  r.shear[1] = dd[r.k[1]] / dd[z];
  r.shear[2] = 1.0f / dd[z];
  return r;
}

/* Watertight ray/triangle test (Woop, Benthin and Wald, "Watertight
 * Ray/Triangle Intersection", JCGT 2(1), 2013).  The vertices are taken into
 * the frame in which the ray starts at the origin and runs along +z
 * (translation, the ray's axis permutation, shear); the 2D edge functions of
 * the sheared triangle tell by their signs whether the ray passes inside (all
 * >= 0 or all <= 0).  An edge shared by two triangles gives the same edge
 * function, of opposite sign, in both, so no ray slips between them; when an
 * edge function rounds to zero in FP32 all three are evaluated again in FP64.
 * Hits closer than the test's own rounding error (the bound deltaT of PBRT
 * 3rd ed., Sec. 3.9.6) are rejected, so a ray does not find the surface it
 * leaves.  Returns 1 with the distance t and the barycentric weights of
 * v0, v1, v2 (bary may be NULL), or 0 for a miss. */
static int tri_hit(const ray_t* r, v3 v0, v3 v1, v3 v2, float* t_out, float* bary) {
  const v3 vs[3] = {v0, v1, v2};
  const float org[3] = {r->o.x, r->o.y, r->o.z};
  float sx[3], sy[3], along[3];
  for (int i = 0; i < 3; ++i) {
    const float v[3] = {vs[i].x, vs[i].y, vs[i].z};
    float rel[3];
    for (int c = 0; c < 3; ++c) rel[c] = v[c] - org[c];
    along[i] = rel[r->k[2]];
    sx[i] = rel[r->k[0]] - r->shear[0] * along[i];
    sy[i] = rel[r->k[1]] - r->shear[1] * along[i];
  }
  float e[3];   /* e[i]: edge function of the edge opposite vertex i */
  for (int i = 0; i < 3; ++i) {
    int a = (i + 2) % 3, b = (i + 1) % 3;
    e[i] = sx[a] * sy[b] - sy[a] * sx[b];
  }
  if (e[0] == 0.0f || e[1] == 0.0f || e[2] == 0.0f)
    for (int i = 0; i < 3; ++i) {
      int a = (i + 2) % 3, b = (i + 1) % 3;
      e[i] = (float)((double)sx[a] * (double)sy[b] - (double)sy[a] * (double)sx[b]);
    }
  int below = e[0] < 0.0f || e[1] < 0.0f || e[2] < 0.0f;
  int above = e[0] > 0.0f || e[1] > 0.0f || e[2] > 0.0f;
  if (below && above) return 0;
  float det = e[0] + e[1] + e[2];
  if (det == 0.0f) return 0;
  float sz[3];
  for (int i = 0; i < 3; ++i) sz[i] = r->shear[2] * along[i];
  float T = e[0] * sz[0] + e[1] * sz[1] + e[2] * sz[2];
  /* the hit is in front when T has the sign of det */
  float Tp = det < 0.0f ? -T : T, detp = det < 0.0f ? -det : det;
  if (Tp <= 0.0f) return 0;
  float t = Tp / detp;
  /* deltaT: error bounds of the sheared coordinates, of the edge functions
     and of T, each the largest magnitude times gamma (PBRT Sec. 3.9.6) */
  float mx = 0.0f, my = 0.0f, mz = 0.0f, me = 0.0f;
  for (int i = 0; i < 3; ++i) {
    mx = fmaxf(mx, fabsf(sx[i]));
    my = fmaxf(my, fabsf(sy[i]));
    mz = fmaxf(mz, fabsf(sz[i]));
    me = fmaxf(me, fabsf(e[i]));
  }
  float err_z = gamma_f32(3) * mz;
  float err_x = gamma_f32(5) * (mx + mz);
  float err_y = gamma_f32(5) * (my + mz);
  float err_e = 2.0f * (gamma_f32(2) * mx * my + err_y * mx + err_x * my);
  float err_t = 3.0f * (gamma_f32(3) * me * mz + err_e * mz + err_z * me) / detp;
  if (!(t > err_t)) return 0;
  *t_out = t;
  if (bary)
    for (int i = 0; i < 3; ++i) bary[i] = e[i] / det;
  return 1;
}

/* Ray/sphere, with the discriminant taken from the distance between the
 * centre and the ray's line (Haines, Guenther and Akenine-Moeller, "Precision
 * Improvements for Ray/Sphere Intersection", Ray Tracing Gems, 2019).  d is
 * unit length.  Nearest t > 0. */
static int sph_hit(const ray_t* r, const float* sp, float* t_out) {
  const float org[3] = {r->o.x, r->o.y, r->o.z}, dir[3] = {r->d.x, r->d.y, r->d.z};
  const float R = sp[3];
  float oc[3], along = 0.0f, oc2 = 0.0f, perp2 = 0.0f;
  for (int c = 0; c < 3; ++c) oc[c] = org[c] - sp[c];
  for (int c = 0; c < 3; ++c) along += oc[c] * dir[c];
  for (int c = 0; c < 3; ++c) { float q = oc[c] - dir[c] * along; perp2 += q * q; }
  for (int c = 0; c < 3; ++c) oc2 += oc[c] * oc[c];
  float disc = R * R - perp2;
  if (disc < 0.0f) return 0;
  float root = along > 0.0f ? -along - sqrtf(disc) : -along + sqrtf(disc);
  if (root == 0.0f) return 0;
  float near = (oc2 - R * R) / root, far = root;
  if (near > far) { float t = near; near = far; far = t; }
  float t = near > 0.0f ? near : far;
  if (!(t > 0.0f)) return 0;
  *t_out = t;
  return 1;
}

static int isect_prim(const scene_t* s, const ray_t* r, int prim, float* t) {
  if (prim < s->nt) return tri_hit(r, tri_v(s, prim, 0), tri_v(s, prim, 1), tri_v(s, prim, 2), t, NULL);
  return sph_hit(r, s->sph + (size_t)(prim - s->nt) * 4, t);
}

/* ------------------------------------------------------------------------ */
/* BVH: recursive median split on the longest centroid axis (quickselect).  */
/* ------------------------------------------------------------------------ */
typedef struct { float bmin[3], bmax[3]; int left, right, first, count; } bnode_t;
typedef struct {
  bnode_t* nodes; int nn, cap;
  int* prims;
  float* pbmin; float* pbmax; float* cent;
} bvh_t;

static void prim_bounds(const scene_t* s, int p, float* mn, float* mx) {
  if (p < s->nt) {
    for (int c = 0; c < 3; ++c) { mn[c] = FLT_MAX; mx[c] = -FLT_MAX; }
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 3; ++c) {
        float v = s->tri[(size_t)p * 9 + k * 3 + c];
        if (v < mn[c]) mn[c] = v;
        if (v > mx[c]) mx[c] = v;
      }
  } else {
    const float* sp = s->sph + (size_t)(p - s->nt) * 4;
    for (int c = 0; c < 3; ++c) { mn[c] = sp[c] - sp[3]; mx[c] = sp[c] + sp[3]; }
  }
}

static int cent_less(const bvh_t* b, int axis, int p, int q) {
  float a = b->cent[(size_t)p * 3 + axis], c = b->cent[(size_t)q * 3 + axis];
  return a < c || (a == c && p < q);
}

static void quickselect(bvh_t* b, int axis, int lo, int hi, int kth) {
  /* partial ordering so that prims[kth] is the kth element of [lo, hi) */
  int* P = b->prims;
  while (hi - lo > 1) {
    int mid = lo + (hi - lo) / 2;
    int a = P[lo], m = P[mid], c = P[hi - 1];
    int piv;
    if (cent_less(b, axis, a, m)) piv = cent_less(b, axis, m, c) ? m : (cent_less(b, axis, a, c) ? c : a);
    else piv = cent_less(b, axis, a, c) ? a : (cent_less(b, axis, m, c) ? c : m);
    int i = lo, j = hi - 1;
    while (i <= j) {
      while (cent_less(b, axis, P[i], piv)) ++i;
      while (cent_less(b, axis, piv, P[j])) --j;
      if (i <= j) { int t = P[i]; P[i] = P[j]; P[j] = t; ++i; --j; }
    }
    if (kth <= j) hi = j + 1;
    else if (kth >= i) lo = i;
    else return;
  }
}

static int bvh_new_node(bvh_t* b) {
  if (b->nn == b->cap) {
    b->cap = b->cap ? b->cap * 2 : 1024;
    b->nodes = (bnode_t*)realloc(b->nodes, sizeof(bnode_t) * b->cap);
  }
  return b->nn++;
}

static int bvh_build_rec(bvh_t* b, int lo, int hi) {
  int id = bvh_new_node(b);
  bnode_t nd;
  float cmin[3], cmax[3];
  for (int c = 0; c < 3; ++c) { nd.bmin[c] = FLT_MAX; nd.bmax[c] = -FLT_MAX; cmin[c] = FLT_MAX; cmax[c] = -FLT_MAX; }
  for (int i = lo; i < hi; ++i) {
    int p = b->prims[i];
    for (int c = 0; c < 3; ++c) {
      if (b->pbmin[(size_t)p * 3 + c] < nd.bmin[c]) nd.bmin[c] = b->pbmin[(size_t)p * 3 + c];
      if (b->pbmax[(size_t)p * 3 + c] > nd.bmax[c]) nd.bmax[c] = b->pbmax[(size_t)p * 3 + c];
      float ce = b->cent[(size_t)p * 3 + c];
      if (ce < cmin[c]) cmin[c] = ce;
      if (ce > cmax[c]) cmax[c] = ce;
    }
  }
  nd.left = nd.right = -1;
  nd.first = lo;
  nd.count = hi - lo;
  if (hi - lo > 4) {
    int axis = 0;
    float ext = cmax[0] - cmin[0];
    for (int c = 1; c < 3; ++c) if (cmax[c] - cmin[c] > ext) { ext = cmax[c] - cmin[c]; axis = c; }
    int mid = lo + (hi - lo) / 2;
    quickselect(b, axis, lo, hi, mid);
    nd.count = 0;
    int l = bvh_build_rec(b, lo, mid);
    int r = bvh_build_rec(b, mid, hi);
    nd.left = l;
    nd.right = r;
  }
  b->nodes[id] = nd;
  return id;
}

static void bvh_build(bvh_t* b, const scene_t* s) {
  memset(b, 0, sizeof(*b));
  int n = s->nprim;
  b->prims = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  b->pbmin = (float*)malloc(sizeof(float) * 3 * (n > 0 ? n : 1));
  b->pbmax = (float*)malloc(sizeof(float) * 3 * (n > 0 ? n : 1));
  b->cent = (float*)malloc(sizeof(float) * 3 * (n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) {
    b->prims[i] = i;
    prim_bounds(s, i, b->pbmin + (size_t)i * 3, b->pbmax + (size_t)i * 3);
    for (int c = 0; c < 3; ++c)
      b->cent[(size_t)i * 3 + c] = 0.5f * (b->pbmin[(size_t)i * 3 + c] + b->pbmax[(size_t)i * 3 + c]);
  }
  if (n > 0) bvh_build_rec(b, 0, n);
}

static void bvh_free(bvh_t* b) { free(b->nodes); free(b->prims); free(b->pbmin); free(b->pbmax); free(b->cent); }

/* slab test; the far distance is widened by 1 + 2*gamma(3) (Pharr, Jakob,
 * Humphreys, PBRT 3rd ed., Sec. 3.9.2) so that the test stays conservative.
 * Near and far planes are chosen by the sign of the direction, so a zero
 * component of either sign with the origin on a plane gives a NaN distance
 * that fmaxf / fminf ignore, instead of one that flips the choice. */
static int box_hit(const float* mn, const float* mx, v3 o, v3 inv, float tmax) {
  float t0 = 0.0f, t1 = tmax;
  for (int a = 0; a < 3; ++a) {
    float oa = vget(o, a), ia = vget(inv, a);
    float tn = (mn[a] - oa) * ia;
    float tf = (mx[a] - oa) * ia;
    if (signbit(ia)) { float t = tn; tn = tf; tf = t; }
    tf *= 1.0000004f;
    t0 = fmaxf(t0, tn);
    t1 = fminf(t1, tf);
    if (t0 > t1) return 0;
  }
  return 1;
}

/* closest hit with t in (0, tmax); equal distances go to the lower primitive index */
static int trace_closest(const scene_t* s, const bvh_t* b, v3 o, v3 d, float tmax, float* t_out) {
  ray_t r = make_ray(o, d);
  v3 inv = mk3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  float best = tmax;
  int bestp = -1;
  if (s->nprim == 0) return -1;
  int stack[128];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const bnode_t* nd = &b->nodes[stack[--sp]];
    if (!box_hit(nd->bmin, nd->bmax, o, inv, best)) continue;
    if (nd->left < 0) {
      for (int i = 0; i < nd->count; ++i) {
        int p = b->prims[nd->first + i];
        float t;
        if (isect_prim(s, &r, p, &t) && (t < best || (t == best && bestp >= 0 && p < bestp))) {
          if (t < tmax) { best = t; bestp = p; }
        }
      }
    } else {
      stack[sp++] = nd->left;
      stack[sp++] = nd->right;
    }
  }
  *t_out = best;
  return bestp;
}

static int trace_brute(const scene_t* s, v3 o, v3 d, float tmax, float* t_out) {
  ray_t r = make_ray(o, d);
  float best = tmax;
  int bestp = -1;
  for (int p = 0; p < s->nprim; ++p) {
    float t;
    if (isect_prim(s, &r, p, &t) && t < tmax && (t < best || (t == best && bestp >= 0 && p < bestp))) {
      best = t;
      bestp = p;
    }
  }
  *t_out = best;
  return bestp;
}

static int trace_any(const scene_t* s, const bvh_t* b, v3 o, v3 d, float tmax) {
  ray_t r = make_ray(o, d);
  v3 inv = mk3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  if (s->nprim == 0) return 0;
  int stack[128];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const bnode_t* nd = &b->nodes[stack[--sp]];
    if (!box_hit(nd->bmin, nd->bmax, o, inv, tmax)) continue;
    if (nd->left < 0) {
      for (int i = 0; i < nd->count; ++i) {
        float t;
        if (isect_prim(s, &r, b->prims[nd->first + i], &t) && t < tmax) return 1;
      }
    } else {
      stack[sp++] = nd->left;
      stack[sp++] = nd->right;
    }
  }
  return 0;
}

/* Hit point and the bound that sizes the offset of the next ray's origin.
 * Triangles: the point b0 v0 + b1 v1 + b2 v2 from the barycentric weights of
 * the hit, with the bound gamma_7 (|b0 v0| + |b1 v1| + |b2 v2|) per component
 * (Pharr, Jakob and Humphreys, PBRT 3rd ed., Sec. 3.9.3).  Spheres: o + t d
 * with the bound gamma_5 |p| (spheres only end paths). */
static void hit_point(const scene_t* s, v3 o, v3 d, int prim, float t, v3* p, v3* err) {
  if (prim < s->nt) {
    ray_t r = make_ray(o, d);
    const v3 v[3] = {tri_v(s, prim, 0), tri_v(s, prim, 1), tri_v(s, prim, 2)};
    float tt, b[3];
    if (tri_hit(&r, v[0], v[1], v[2], &tt, b)) {
      float q[3] = {0.0f, 0.0f, 0.0f}, e[3] = {0.0f, 0.0f, 0.0f};
      for (int i = 0; i < 3; ++i) {
        const float vi[3] = {v[i].x, v[i].y, v[i].z};
        for (int c = 0; c < 3; ++c) {
          q[c] += vi[c] * b[i];
          e[c] += fabsf(vi[c] * b[i]);
        }
      }
      const float g7 = gamma_f32(7);
      *p = mk3(q[0], q[1], q[2]);
      *err = mk3(g7 * e[0], g7 * e[1], g7 * e[2]);
      return;
    }
  }
  *p = vadd(o, vmul(d, t));
  const float g5 = gamma_f32(5);
  *err = mk3(g5 * fabsf(p->x), g5 * fabsf(p->y), g5 * fabsf(p->z));
}

/* New ray origin: the hit point moved along the geometric normal, to the side
 * the new direction d leaves on, by twice the error bound projected on the
 * normal plus 1e-7. */
static v3 offset_origin(v3 p, v3 n, v3 err, v3 d) {
  v3 ns = vdot(n, d) >= 0.0f ? n : vneg(n);
  float e = 2.0f * (fabsf(n.x) * err.x + fabsf(n.y) * err.y + fabsf(n.z) * err.z) + 1e-7f;
  return vadd(p, vmul(ns, e));
}

/* ------------------------------------------------------------------------ */
/* materials                                                                */
/* ------------------------------------------------------------------------ */
static int mat_black(const mat_t* m) {
  return m->type == MT_DIFFUSE && m->albedo[0] <= 0.0f && m->albedo[1] <= 0.0f && m->albedo[2] <= 0.0f;
}
static int mat_delta(const mat_t* m) { return m->type == MT_DIELECTRIC; }

static float ggx_D(float alpha, float cos_h) {
  float a2 = alpha * alpha;
  float t = cos_h * cos_h * (a2 - 1.0f) + 1.0f;
  return a2 / ((float)PI_D * t * t);
}
static float ggx_G1(float alpha, float c) {
  float a2 = alpha * alpha;
  return 2.0f * c / (c + sqrtf(a2 + (1.0f - a2) * c * c));
}

/* BSDF value f(wo, wi) (FP64 colour); 0 for delta lobes and black surfaces. */
static c3 bsdf_eval(const mat_t* m, v3 n, v3 wo, v3 wi) {
  float co = vdot(n, wo), ci = vdot(n, wi);
  if (m->type == MT_DIFFUSE) {
    if (!(co * ci > 0.0f)) return ck(0, 0, 0);
    return ck(m->albedo[0] / PI_D, m->albedo[1] / PI_D, m->albedo[2] / PI_D);
  }
  if (m->type == MT_GGX) {
    if (!(co * ci > 0.0f)) return ck(0, 0, 0);
    v3 ns = co >= 0.0f ? n : vneg(n);
    float cos_o = fabsf(co), cos_i = fabsf(ci);
    v3 h = vnorm(vadd(wo, wi));
    float ch = vdot(ns, h);
    if (!(ch > 0.0f)) return ck(0, 0, 0);
    double D = ggx_D(m->alpha, ch);
    double G = (double)ggx_G1(m->alpha, cos_o) * (double)ggx_G1(m->alpha, cos_i);
    double x = 1.0 - fabs((double)vdot(wo, h));
    double x5 = x * x * x * x * x;
    double k = D * G / (4.0 * cos_o * cos_i);
    return ck((m->albedo[0] + (1.0 - m->albedo[0]) * x5) * k, (m->albedo[1] + (1.0 - m->albedo[1]) * x5) * k,
              (m->albedo[2] + (1.0 - m->albedo[2]) * x5) * k);
  }
  return ck(0, 0, 0);
}

/* Directional pdf of sampling wi given wo (solid angle; 1 for delta lobes). */
static double bsdf_pdf(const mat_t* m, v3 n, v3 wo, v3 wi) {
  float co = vdot(n, wo), ci = vdot(n, wi);
  if (m->type == MT_DIELECTRIC) return 1.0;
  if (!(co * ci > 0.0f)) return 0.0;
  if (m->type == MT_DIFFUSE) return fabs((double)ci) / PI_D;
  v3 ns = co >= 0.0f ? n : vneg(n);
  v3 h = vnorm(vadd(wo, wi));
  float ch = vdot(ns, h);
  if (!(ch > 0.0f)) return 0.0;
  return (double)ggx_D(m->alpha, ch) * (double)ch / (4.0 * fabs((double)vdot(wo, h)));
}

/* Samples wi given wo from random numbers u_lobe, u1, u2.  weight = f |cos| / pdf
 * (with the (eta_i/eta_t)^2 radiance scaling on refraction when `camera`).
 * Returns 0 if the sample is rejected. */
static int bsdf_sample(const mat_t* m, v3 n, v3 wo, float ul, float u1, float u2, int camera,
                       v3* wi, c3* weight) {
  float co = vdot(n, wo);
  v3 ns = co >= 0.0f ? n : vneg(n);
  if (m->type == MT_DIFFUSE) {
    float r = sqrtf(u1);
    float phi = TWO_PI_F * u2;
    float lz = sqrtf(fmaxf(0.0f, 1.0f - u1));
    *wi = from_local(ns, r * cosf(phi), r * sinf(phi), lz);
    if (!(lz > 0.0f)) return 0;
    *weight = ck(m->albedo[0], m->albedo[1], m->albedo[2]);
    return 1;
  }
  if (m->type == MT_DIELECTRIC) {
    int entering = co > 0.0f;
    float eta = entering ? 1.0f / m->ior : m->ior;
    float cos_i = vdot(ns, wo);
    float sin2_t = eta * eta * (1.0f - cos_i * cos_i);
    float F = 1.0f, cos_t = 0.0f;
    if (sin2_t < 1.0f) {
      cos_t = sqrtf(1.0f - sin2_t);
      float rs = (eta * cos_i - cos_t) / (eta * cos_i + cos_t);
      float rp = (cos_i - eta * cos_t) / (cos_i + eta * cos_t);
      F = 0.5f * (rs * rs + rp * rp);
    }
    if (ul < F) {
      *wi = vsub(vmul(ns, 2.0f * cos_i), wo);
      *weight = ck(1, 1, 1);
    } else {
      *wi = vadd(vmul(wo, -eta), vmul(ns, eta * cos_i - cos_t));
      double s = camera ? (double)eta * (double)eta : 1.0;
      *weight = ck(s, s, s);
    }
    return 1;
  }
  /* GGX conductor: half vector from D(h) cos(h) */
  {
    float a2 = m->alpha * m->alpha;
    float tan2 = a2 * u1 / (1.0f - u1);
    float ch = 1.0f / sqrtf(1.0f + tan2);
    float sh = sqrtf(fmaxf(0.0f, 1.0f - ch * ch));
    float phi = TWO_PI_F * u2;
    v3 h = from_local(ns, sh * cosf(phi), sh * sinf(phi), ch);
    float oh = vdot(wo, h);
    *wi = vsub(vmul(h, 2.0f * oh), wo);
    if (!(vdot(ns, *wi) > 0.0f) || !(co > 0.0f || co < 0.0f)) return 0;
    c3 f = bsdf_eval(m, n, wo, *wi);
    double pdf = bsdf_pdf(m, n, wo, *wi);
    if (!(pdf > 0.0)) return 0;
    double c = fabs((double)vdot(n, *wi)) / pdf;
    *weight = cscale(f, c);
    return 1;
  }
}

/* ------------------------------------------------------------------------ */
/* Density octree (Sec. 5): a sparse tree of cells, each holding the number */
/* of NEE vertices counted in it.  Written as an explicit tree of cells; the */
/* flat word layout of Sec. 5.5 (siblings in eight consecutive words, a      */
/* split cell holding the negated index of its first child) appears only in */
/* orc_octree_dump, where each cell's word index is its allocation order.    */
/* ------------------------------------------------------------------------ */

/* Plane/box intersection area, Eq. area (Sec. 5.3), in FP64.  Appendix A
 * derives it as the h-derivative of the box volume below the plane
 * <n, y> = h: over the d axes the normal is not perpendicular to,
 *   A = (prod of the box extents along the other axes)
 *       * | sum over the 2^d corners b of the box in those axes of
 *           eps_b max(0, h - <n, b>)^(d-1) | / ((d-1)! prod n_i),
 * with h = <n, p>, eps_b = +1 for an even and -1 for an odd number of upper
 * bounds among b's coordinates.  The paper's implementation decides d from
 * the FP32 normal: an axis whose |n_i| is within 1e-3 of 1 gives d = 1 and
 * the area of the box's face across that axis (the first such axis, in x, y,
 * z order); otherwise the first axis with |n_i| < 1e-4 is taken as
 * perpendicular (d = 2); otherwise d = 3.  These decisions are made on the
 * FP32 components, as the paper does. */
static double plane_box_area(const double lo[3], const double hi[3], const double p[3], const float n[3]) {
  int axes[3], d = 0;
  for (int i = 0; i < 3; ++i)
    if (fabsf(fabsf(n[i]) - 1.0f) < 1e-3f) {
      /* d = 1: the plane is taken as parallel to the face across axis i */
      double a = 1.0;
      for (int j = 0; j < 3; ++j) if (j != i) a *= hi[j] - lo[j];
      return a;
    }
  int dropped = -1;
  for (int i = 0; i < 3 && dropped < 0; ++i) if (fabsf(n[i]) < 1e-4f) dropped = i;
  for (int i = 0; i < 3; ++i) if (i != dropped) axes[d++] = i;
  double h = 0.0, prod_n = 1.0;
  for (int k = 0; k < d; ++k) { h += (double)n[axes[k]] * p[axes[k]]; prod_n *= (double)n[axes[k]]; }
  double sum = 0.0;
  for (int corner = 0; corner < (1 << d); ++corner) {
    double nb = 0.0;
    int uppers = 0;
    for (int k = 0; k < d; ++k) {
      int up = (corner >> k) & 1;
      uppers += up;
      nb += (double)n[axes[k]] * (up ? hi[axes[k]] : lo[axes[k]]);
    }
    double m = h - nb > 0.0 ? h - nb : 0.0;
    double term = d == 3 ? m * m : m;
    sum += (uppers & 1) ? -term : term;
  }
  double fact = d == 3 ? 2.0 : 1.0;  /* (d-1)! */
  double a = fabs(sum / (fact * prod_n));
  if (dropped >= 0) a *= hi[dropped] - lo[dropped];
  return a;
}

double orc_intersection_area(const float bmin[3], const float bmax[3], const float pos[3], const float n[3]) {
  double lo[3], hi[3], p[3];
  for (int c = 0; c < 3; ++c) { lo[c] = bmin[c]; hi[c] = bmax[c]; p[c] = pos[c]; }
  return plane_box_area(lo, hi, p, n);
}

typedef struct oct_cell {
  int32_t count;          /* vertices counted here (leaves) */
  int32_t word;           /* index in the flat layout (allocation order) */
  struct oct_cell* kids;  /* NULL for a leaf, else 8 cells in octant order x + 2y + 4z */
} oct_cell;

struct orc_octree {
  oct_cell root;
  int32_t words_used;     /* root + 8 per split; capacity + 1 once a split found no room */
  int32_t capacity;       /* words available: requested capacity rounded up to 8m + 1 */
  int32_t depth;          /* deepest level that holds a cell */
  float minb[3], size_inv[3], scene_scale;
  int split_factor;
  int iteration;          /* current 1-based iteration */
  int iter_clamp;         /* min(iteration, 1000): densities are divided by it */
  int32_t threshold;      /* a cell splits when its count reaches split_factor * iter_clamp */
  int32_t fresh_count;    /* count a cell created in this iteration starts with */
};

#define OCT_FILL_ITERATIONS 1000   /* counting stops after this many iterations (Appendix B) */
#define OCT_MAX_DEPTH 30           /* no cell below level 30: 2^30 cells per axis */

orc_octree* orc_octree_new(const float smin[3], const float smax[3], int capacity, int split_factor) {
  orc_octree* o = (orc_octree*)calloc(1, sizeof(orc_octree));
  /* the box is the scene's, grown by 0.2 % about its centre so that points on
     the scene's bounds fall inside (Appendix B) */
  float size[3];
  for (int c = 0; c < 3; ++c) size[c] = (smax[c] - smin[c]) * 1.002f;
  for (int c = 0; c < 3; ++c) {
    o->size_inv[c] = 1.0f / size[c];
    o->minb[c] = smin[c] - size[c] * (0.001f / 1.002f);
  }
  o->scene_scale = sqrtf(size[0] * size[0] + size[1] * size[1] + size[2] * size[2]);
  o->capacity = 8 * ((capacity + 7) / 8) + 1;
  o->root.word = 0;
  o->words_used = 1;
  o->split_factor = split_factor;
  return o;
}

static void cell_free(oct_cell* c) {
  if (!c->kids) return;
  for (int k = 0; k < 8; ++k) cell_free(&c->kids[k]);
  free(c->kids);
}

void orc_octree_free(orc_octree* o) {
  if (!o) return;
  cell_free(&o->root);
  free(o);
}

/* Counts are integrated over the iterations (Sec. 5.4): the split threshold
 * grows with the iteration and densities are divided by it.  A new cell
 * starts with a quarter of the split factor per iteration so far, since a
 * surface crosses about four of a cell's eight children (Sec. 5.2). */
void orc_octree_set_iteration(orc_octree* o, int iter) {
  o->iteration = iter;
  o->iter_clamp = iter < OCT_FILL_ITERATIONS ? iter : OCT_FILL_ITERATIONS;
  o->threshold = o->split_factor * o->iter_clamp;
  if (iter <= OCT_FILL_ITERATIONS)   /* no cell is created later */
    o->fresh_count = (o->split_factor * iter + 3) / 4;   /* ceil(split_factor * iter / 4) */
}

/* Position in units of the octree box, in FP32 as the paper computes it;
 * returns 0 outside [0, 1)^3. */
static int oct_unit_pos(const orc_octree* o, const float pos[3], float u[3]) {
  for (int c = 0; c < 3; ++c) {
    u[c] = (pos[c] - o->minb[c]) * o->size_inv[c];
    if (!(u[c] >= 0.0f && u[c] < 1.0f)) return 0;
  }
  return 1;
}

/* Octant at `level` (>= 1) of the cell holding unit position u: on the grid
 * of 2^level cells per axis the cell index is floor(u 2^level), and its
 * lowest bit tells which half of the parent cell it lies in. */
static int oct_octant(const float u[3], int level) {
  float scale = ldexpf(1.0f, level);
  int o = 0;
  for (int c = 0; c < 3; ++c) o |= ((int)(u[c] * scale) & 1) << c;
  return o;
}

static oct_cell* oct_leaf(const orc_octree* o, const float u[3], int* level) {
  oct_cell* c = (oct_cell*)&o->root;
  int L = 0;
  while (c->kids) { ++L; c = &c->kids[oct_octant(u, L)]; }
  *level = L;
  return c;
}

/* One NEE vertex (Sec. 5.1): one more in the leaf cell that holds it; the
 * vertex that brings a cell to the threshold splits it into eight children
 * (Sec. 5.2).  That vertex stays counted in the cell it split (whose count
 * is no longer read).  A split needs eight free words; when they are not
 * there the tree stops growing and the full cell keeps counting. */
void orc_octree_increment(orc_octree* o, const float pos[3]) {
  if (o->iteration > OCT_FILL_ITERATIONS) return;
  float u[3];
  if (!oct_unit_pos(o, pos, u)) return;
  int level;
  oct_cell* c = oct_leaf(o, u, &level);
  c->count += 1;
  if (c->count != o->threshold || level >= OCT_MAX_DEPTH) return;
  if (o->words_used + 8 > o->capacity) { o->words_used = o->capacity + 1; return; }
  c->kids = (oct_cell*)calloc(8, sizeof(oct_cell));
  for (int k = 0; k < 8; ++k) {
    c->kids[k].count = o->fresh_count;
    c->kids[k].word = o->words_used + k;
  }
  o->words_used += 8;
  if (level + 1 > o->depth) o->depth = level + 1;
}

/* Density at p for a plane with normal n (Eq. octdensity): the count of the
 * leaf cell holding p divided by the iteration count and by the area of the
 * plane inside the cell, the area kept above a small fraction of the squared
 * cell diagonal (0.1 of it for the centre query of the robust estimate, 0.01
 * otherwise).  Empty cells and points outside the box give 0.  *diag
 * receives the cell diagonal when the count is positive. */
static double oct_density(const orc_octree* o, const float pos[3], const float n[3], int centre, float* diag) {
  float u[3];
  if (!oct_unit_pos(o, pos, u)) return 0.0;
  int level;
  const oct_cell* c = oct_leaf(o, u, &level);
  if (c->count <= 0) return 0.0;
  double lo[3], hi[3], p[3];
  for (int a = 0; a < 3; ++a) {
    double extent = ldexp(1.0 / (double)o->size_inv[a], -level);
    double index = floor((double)u[a] * ldexp(1.0, level));
    lo[a] = index * extent;
    hi[a] = lo[a] + extent;
    p[a] = (double)pos[a] - (double)o->minb[a];
  }
  double area = plane_box_area(lo, hi, p, n);
  double cell_diag = ldexp((double)o->scene_scale, -level);
  double floor_area = cell_diag * cell_diag * (centre ? 0.1 : 0.01);
  if (diag) *diag = ldexpf(o->scene_scale, -level);
  return (double)c->count / ((double)o->iter_clamp * (area > floor_area ? area : floor_area));
}

static int cmp_float(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  return (x > y) - (x < y);
}

/* Robust density: the centre query and four more at 1.1 cell diagonals from
 * p along the two tangents (Duff et al. basis of the geometric normal); the
 * result is the median of the positive ones, the upper one of the middle two
 * for an even number, 0 when none is positive.  The displaced points and the
 * step are computed in FP32, as the paper does; the step is 1.1e-3 when the
 * centre cell is empty. */
static float oct_density_robust(const orc_octree* o, const float pos[3], const float n[3]) {
  float found[5];
  int nfound = 0;
  float step = 1e-3f;
  float d0 = (float)oct_density(o, pos, n, 1, &step);
  if (d0 > 0.0f) found[nfound++] = d0;
  step *= 1.1f;
  v3 t, b;
  onb(vload(n), &t, &b);
  const v3 dirs[4] = {t, vneg(t), b, vneg(b)};
  for (int k = 0; k < 4; ++k) {
    v3 q = vadd(vload(pos), vmul(dirs[k], step));
    float qq[3] = {q.x, q.y, q.z};
    float dk = (float)oct_density(o, qq, n, 0, NULL);
    if (dk > 0.0f) found[nfound++] = dk;
  }
  if (nfound == 0) return 0.0f;
  qsort(found, (size_t)nfound, sizeof(float), cmp_float);
  return found[nfound / 2];
}

float orc_octree_density(orc_octree* o, const float pos[3], const float n[3], int robust) {
  return robust ? oct_density_robust(o, pos, n) : (float)oct_density(o, pos, n, 0, NULL);
}

static void cell_dump(const oct_cell* c, int32_t* words, int n) {
  if (c->word >= n) return;
  words[c->word] = c->kids ? -c->kids[0].word : c->count;
  if (c->kids)
    for (int k = 0; k < 8; ++k) cell_dump(&c->kids[k], words, n);
}

/* The tree in the flat layout of Sec. 5.5, min(n, capacity) words: a leaf's
 * word holds its count, a split cell's word the negated index of its first
 * child; words no cell has taken hold the count a new cell would start with.
 * meta: words used (capacity + 1 after an overflow), depth, capacity. */
int orc_octree_dump(const orc_octree* o, int32_t* nodes, int n, int32_t meta[3]) {
  int m = n < o->capacity ? n : o->capacity;
  if (nodes) {
    for (int i = 0; i < m; ++i) nodes[i] = o->fresh_count;
    cell_dump(&o->root, nodes, m);
  }
  meta[0] = o->words_used;
  meta[1] = o->depth;
  meta[2] = o->capacity;
  return o->capacity;
}

/* Rebuilds the tree from the flat layout (the inverse of orc_octree_dump):
 * word 0 is the root; a negative word links to eight consecutive children.
 * words_used and depth are taken as given.  Returns 0, or -1 when a link
 * points outside [1, n - 8] or a word is reached twice. */
static int cell_load(oct_cell* c, const int32_t* words, int n, int w, char* seen) {
  if (w < 0 || w >= n || seen[w]) return -1;
  seen[w] = 1;
  c->word = w;
  if (words[w] >= 0) { c->count = words[w]; c->kids = NULL; return 0; }
  int first = -words[w];
  if (first < 1 || first > n - 8) return -1;
  c->kids = (oct_cell*)calloc(8, sizeof(oct_cell));
  for (int k = 0; k < 8; ++k)
    if (cell_load(&c->kids[k], words, n, first + k, seen) != 0) return -1;
  return 0;
}

int orc_octree_load(orc_octree* o, const int32_t* words, int n, int words_used, int depth) {
  cell_free(&o->root);
  memset(&o->root, 0, sizeof(o->root));
  char* seen = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  int rc = cell_load(&o->root, words, n, 0, seen);
  free(seen);
  o->words_used = words_used;
  o->depth = depth;
  return rc;
}

void orc_onb(const float n[3], float t[3], float b[3]) {
  v3 tt, bb;
  onb(vload(n), &tt, &bb);
  t[0] = tt.x; t[1] = tt.y; t[2] = tt.z;
  b[0] = bb.x; b[1] = bb.y; b[2] = bb.z;
}

int orc_light_selection(const double* power, int n, int n_samples, uint64_t seed, double* psel, int64_t* counts) {
  if (n < 1) return -1;
  float* prob = (float*)malloc(sizeof(float) * (size_t)n);
  int* alias = (int*)malloc(sizeof(int) * (size_t)n);
  alias_build(power, n, psel, prob, alias);
  rng_t g;
  g.key[0] = (uint32_t)seed;
  g.key[1] = (uint32_t)(seed >> 32);
  g.iter = 1;
  for (int i = 0; i < n; ++i) counts[i] = 0;
  for (int k = 0; k < n_samples; ++k)
    counts[alias_pick(prob, alias, n, rng_raw(&g, (uint32_t)k, 0, 0), rng_u(&g, (uint32_t)k, 0, 1))]++;
  free(prob);
  free(alias);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* explicit MIS over a full vertex list (Eq. misweight .. Eq. misw)           */
/* ------------------------------------------------------------------------ */
typedef struct {
  const mat_t* mat;  /* BSDF at this vertex (NULL for the camera) */
  v3 n_bsdf;         /* normal for BSDF evaluation */
  v3 n_in, n_out;    /* normal for cosines of the segment to v_{i-1} / to v_{i+1} */
  int delta;
} mv_t;

/* Path v_0 .. v_l: v_0 the camera, v_l the light point.  u[i], L[i] are the
 * unit direction and length of segment (v_i, v_{i+1}), i = 0 .. l-1.  p_l is
 * the NEE area pdf of v_l from v_{l-1}; rho the density at v_{l-1}; p_l_lp
 * the area pdf of v_l under light-photon emission and n_lp their number.
 * Fills p_e, p_E, nP[k] (k = 1 .. l-2, Eq. photonpdf times n_P) and nLP[k]
 * (k = 1 .. l-1, Eq. stdphotonpdf times n_LP; the light emits cosine-
 * weighted about its normal, so p_{l -> l-1} = cos_y / pi |cos_{l-1}| / L^2). */
static void path_pdfs(const mv_t* v, const v3* u, const float* L, int l, double p_l, double rho, double r,
                      uint32_t mask, double n_lp, double p_l_lp, double* p_e, double* p_E, double* nP,
                      double* nLP) {
  double F[64], R[64];
  F[1] = 1.0;
  for (int i = 2; i <= l; ++i) {
    const mv_t* a = &v[i - 1];
    double pdf = bsdf_pdf(a->mat, a->n_bsdf, vneg(u[i - 2]), u[i - 1]);
    double c = fabs((double)vdot(v[i].n_in, u[i - 1]));
    F[i] = pdf * c / ((double)L[i - 1] * (double)L[i - 1]);
  }
  for (int i = 1; i <= l - 2; ++i) {
    const mv_t* b = &v[i + 1];
    double pdf = bsdf_pdf(b->mat, b->n_bsdf, u[i + 1], vneg(u[i]));
    double c = fabs((double)vdot(v[i].n_out, u[i]));
    R[i] = pdf * c / ((double)L[i] * (double)L[i]);
  }
  double pe = 1.0;
  for (int i = 1; i <= l; ++i) pe *= F[i];
  *p_e = (mask & 1u) ? pe : 0.0;
  double pE = 0.0;
  if (l >= 2 && !v[l - 1].delta && (mask & 2u)) {
    pE = p_l;
    for (int i = 1; i <= l - 1; ++i) pE *= F[i];
  }
  *p_E = pE;
  for (int k = 1; k <= l - 2; ++k) {
    double x = 0.0;
    if (!v[k].delta && (mask & 4u) && rho > 0.0) {
      x = p_l * rho * PI_D * r * r;
      for (int i = k; i <= l - 2; ++i) x *= R[i];
      for (int i = 1; i <= k; ++i) x *= F[i];
    }
    nP[k] = x;
  }
  for (int k = 1; k <= l - 1; ++k) nLP[k] = 0.0;
  if ((mask & 8u) && n_lp > 0.0 && l >= 2) {
    double cos_y = (double)vdot(v[l].n_out, vneg(u[l - 1]));
    double c = fabs((double)vdot(v[l - 1].n_out, u[l - 1]));
    R[l - 1] = cos_y > 0.0 ? cos_y / PI_D * c / ((double)L[l - 1] * (double)L[l - 1]) : 0.0;
    for (int k = 1; k <= l - 1; ++k) {
      if (v[k].delta) continue;
      double x = n_lp * PI_D * r * r * p_l_lp;
      for (int i = k; i <= l - 1; ++i) x *= R[i];
      for (int i = 1; i <= k; ++i) x *= F[i];
      nLP[k] = x;
    }
  }
}

static double mis_weight(const mv_t* v, const v3* u, const float* L, int l, double p_l, double rho, double r,
                         uint32_t mask, double n_lp, double p_l_lp, int strategy /* 0 e, 1 E, 2 P, 3 LP */,
                         int kmerge) {
  double pe, pE, nP[64], nLP[64];
  path_pdfs(v, u, L, l, p_l, rho, r, mask, n_lp, p_l_lp, &pe, &pE, nP, nLP);
  double sum = pe + pE;
  for (int k = 1; k <= l - 2; ++k) sum += nP[k];
  for (int k = 1; k <= l - 1; ++k) sum += nLP[k];
  double own = strategy == 0 ? pe : (strategy == 1 ? pE : (strategy == 2 ? nP[kmerge] : nLP[kmerge]));
  return sum > 0.0 ? own / sum : 0.0;
}

static int mis_weights_impl(const float* verts, int n_verts, const float* light, float merge_radius, double rho,
                            uint32_t mask, double n_lp, double p_l_lp, int with_lp, double* w_out) {
  /* verts: [n_verts][7] = pos, normal, type (0 Lambertian albedo 1, 1 delta);
   * v_0 is the camera.  light: pos, normal, p_l (, p_l^LP).  w_out: [l+1] =
   * w_e, w_E, w_P1 .. w_P(l-2) with l = n_verts, then w_LP1 .. w_LP(l-1). */
  static mat_t lam = {MT_DIFFUSE, {1, 1, 1}, {0, 0, 0}, 1, 0};
  static mat_t gl = {MT_DIELECTRIC, {0, 0, 0}, {0, 0, 0}, 1.5f, 0};
  int l = n_verts;
  if (l < 1 || l > 60) return -1;
  mv_t v[64];
  v3 P[64], u[64];
  float L[64];
  for (int i = 0; i < n_verts; ++i) {
    P[i] = vload(verts + i * 7);
    v3 n = vload(verts + i * 7 + 3);
    int delta = verts[i * 7 + 6] > 0.5f;
    v[i].mat = delta ? &gl : &lam;
    v[i].n_bsdf = v[i].n_in = v[i].n_out = n;
    v[i].delta = delta;
  }
  P[l] = vload(light);
  v[l].mat = NULL;
  v[l].n_in = v[l].n_out = v[l].n_bsdf = vload(light + 3);
  v[l].delta = 0;
  for (int i = 0; i < l; ++i) {
    v3 d = vsub(P[i + 1], P[i]);
    L[i] = sqrtf(vdot(d, d));
    u[i] = vnorm(d);
  }
  double pe, pE, nP[64], nLP[64];
  path_pdfs(v, u, L, l, (double)light[6], rho, merge_radius, mask, n_lp, p_l_lp, &pe, &pE, nP, nLP);
  double sum = pe + pE;
  for (int k = 1; k <= l - 2; ++k) sum += nP[k];
  for (int k = 1; k <= l - 1; ++k) sum += nLP[k];
  w_out[0] = sum > 0 ? pe / sum : 0;
  w_out[1] = sum > 0 ? pE / sum : 0;
  for (int k = 1; k <= l - 2; ++k) w_out[1 + k] = sum > 0 ? nP[k] / sum : 0;
  if (with_lp)
    for (int k = 1; k <= l - 1; ++k) w_out[l - 1 + k] = sum > 0 ? nLP[k] / sum : 0;
  return 0;
}

int orc_mis_weights(const float* verts, int n_verts, const float* light, float merge_radius, double rho,
                    uint32_t mask, double* w_out) {
  return mis_weights_impl(verts, n_verts, light, merge_radius, rho, mask & 7u, 0.0, 0.0, 0, w_out);
}

int orc_mis_weights_lp(const float* verts, int n_verts, const float* light, float merge_radius, double rho,
                       uint32_t mask, double n_lp, double* w_out) {
  return mis_weights_impl(verts, n_verts, light, merge_radius, rho, mask, n_lp, (double)light[7], 1, w_out);
}

/* ------------------------------------------------------------------------ */
/* the NEB iteration                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  v3 pos, n;          /* hit point, geometric normal (unflipped) */
  v3 err;             /* error bound of pos */
  int prim, mat;
  int delta;
  v3 din;             /* direction of the segment arriving from v_{k-1} */
  float tin;          /* its length */
  c3 tau;             /* throughput up to this vertex */
  /* NEE data */
  int is_nee;
  int light;
  v3 y, ny, ldir;
  float ldist;
  double p_l;
  c3 dE;              /* zero if occluded or back-facing */
  float rho;
} cv_t;

typedef struct {
  int pixel, k;       /* random hit at vertex k of this pixel's path */
  c3 le;
} rh_t;

typedef struct { float x; int pixel, k; } mref_t;

static int mref_cmp(const void* a, const void* b) {
  const mref_t* p = (const mref_t*)a;
  const mref_t* q = (const mref_t*)b;
  if (p->x < q->x) return -1;
  if (p->x > q->x) return 1;
  if (p->pixel != q->pixel) return p->pixel < q->pixel ? -1 : 1;
  return p->k - q->k;
}

typedef struct {
  const scene_t* s;
  const bvh_t* b;
  const orc_config* cfg;
  rng_t rng;
  int W, H, D;
  float r;
  v3 eye, fwd, right, up;
  float tanh_, aspect;
} ctx_t;

static double sph_pdf_area(const scene_t* s, int prim, v3 y, v3 x) {
  const float* sp = s->sph + (size_t)(prim - s->nt) * 4;
  v3 c = vload(sp);
  double R = sp[3];
  if (!(vdot(vsub(y, c), vsub(x, c)) > 0.0f)) return 0.0;
  return 1.0 / (2.0 * PI_D * R * R);
}

/* p_l: NEE area pdf of point y on light `li` seen from x */
static double light_pdf(const scene_t* s, int li, v3 y, v3 x) {
  const light_t* L = &s->lights[li];
  if (L->kind == 0) return L->psel / (double)L->area;
  return L->psel * sph_pdf_area(s, L->prim, y, x);
}

/* area pdf of a light point under light-photon emission: the light chosen
 * as for NEE, the point uniform on the whole light surface */
static double lp_light_pdf(const scene_t* s, int li) {
  const light_t* L = &s->lights[li];
  if (L->kind == 0) return L->psel / (double)L->area;
  double R = s->sph[(size_t)(L->prim - s->nt) * 4 + 3];
  return L->psel / (4.0 * PI_D * R * R);
}

static int sample_light(const ctx_t* c, uint32_t pixel, uint32_t stream, v3 x, int* li, v3* y, v3* ny,
                        double* p_l) {
  const scene_t* s = c->s;
  if (s->nl == 0) return 0;
  int i = alias_pick(s->alias_prob, s->alias_idx, s->nl, rng_raw(&c->rng, pixel, stream, 0),
                     rng_u(&c->rng, pixel, stream, 1));
  float u2 = rng_u(&c->rng, pixel, stream, 2);
  float u3 = rng_u(&c->rng, pixel, stream, 3);
  const light_t* L = &s->lights[i];
  if (L->kind == 0) {
    float b1 = u2, b2 = u3;
    if (b1 + b2 > 1.0f) { b1 = 1.0f - b1; b2 = 1.0f - b2; }
    v3 a = tri_v(s, L->prim, 0), bb = tri_v(s, L->prim, 1), cc = tri_v(s, L->prim, 2);
    v3 e1 = vsub(bb, a), e2 = vsub(cc, a);
    *y = vadd(vadd(a, vmul(e1, b1)), vmul(e2, b2));
    *ny = vnorm(vcross(e1, e2));
  } else {
    const float* sp = s->sph + (size_t)(L->prim - s->nt) * 4;
    v3 ce = vload(sp);
    float R = sp[3];
    v3 w = vnorm(vsub(x, ce));
    float z = u2;
    float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float phi = TWO_PI_F * u3;
    v3 dir = from_local(w, rr * cosf(phi), rr * sinf(phi), z);
    *y = vadd(ce, vmul(dir, R));
    *ny = dir;
  }
  *li = i;
  *p_l = light_pdf(s, i, *y, x);
  return 1;
}

static c3 light_le(const scene_t* s, int prim) {
  const mat_t* m = &s->mats[s->prim_mat[prim]];
  return ck(m->emission[0], m->emission[1], m->emission[2]);
}

/* camera path of one pixel (pass 1) */
static int trace_camera(const ctx_t* c, int pixel, cv_t* path, int64_t* st, rh_t* rh, int* nrh,
                        orc_octree* oct) {
  const scene_t* s = c->s;
  int px = pixel % c->W, py = pixel / c->W;
  float ju = rng_u(&c->rng, (uint32_t)pixel, 0, 0);
  float jv = rng_u(&c->rng, (uint32_t)pixel, 0, 1);
  float sx = (((float)px + ju) / (float)c->W) * 2.0f - 1.0f;
  float sy = 1.0f - (((float)py + jv) / (float)c->H) * 2.0f;
  float a = sx * c->tanh_ * c->aspect;
  float bb = sy * c->tanh_;
  v3 d = vnorm(mk3(c->fwd.x + c->right.x * a + c->up.x * bb, c->fwd.y + c->right.y * a + c->up.y * bb,
                   c->fwd.z + c->right.z * a + c->up.z * bb));
  v3 o = c->eye;
  c3 tau = ck(1, 1, 1);
  int K = 0;
  for (int k = 1; k <= c->D; ++k) {
    float t;
    st[ORC_ST_CAMERA_RAYS]++;
    int prim = trace_closest(s, c->b, o, d, INFINITY, &t);
    if (prim < 0) break;
    cv_t* v = &path[k];
    memset(v, 0, sizeof(*v));
    hit_point(s, o, d, prim, t, &v->pos, &v->err);
    v->n = prim_normal(s, prim, v->pos);
    v->prim = prim;
    v->mat = s->prim_mat[prim];
    const mat_t* m = &s->mats[v->mat];
    v->delta = mat_delta(m);
    v->din = d;
    v->tin = t;
    v->tau = tau;
    v->rho = 0.0f;
    K = k;
    v3 wo = vneg(d);
    if (s->prim_light[prim] >= 0 && (prim >= s->nt || vdot(v->n, wo) > 0.0f)) {
      rh[*nrh].pixel = pixel;
      rh[*nrh].k = k;
      rh[*nrh].le = light_le(s, prim);
      (*nrh)++;
      st[ORC_ST_RANDOM_HITS]++;
    }
    if (mat_black(m)) { K = k; v->is_nee = 0; return -k; /* terminated on black */ }
    uint32_t stream = (uint32_t)k * 256u;
    if (k <= c->D - 1 && s->nl > 0) {
      v->is_nee = 1;
      st[ORC_ST_NEE_VERTICES]++;
      int li = 0;
      v3 y = mk3(0, 0, 0), ny = mk3(0, 0, 0);
      double p_l = 0.0;
      sample_light(c, (uint32_t)pixel, stream, v->pos, &li, &y, &ny, &p_l);
      v->light = li;
      v->y = y;
      v->ny = ny;
      v->p_l = p_l;
      v3 dd = vsub(y, v->pos);
      float dist2 = vdot(dd, dd);
      float dist = sqrtf(dist2);
      v->ldir = vmul(dd, 1.0f / dist);
      v->ldist = dist;
      float cos_y = -vdot(ny, v->ldir);
      v->dE = ck(0, 0, 0);
      if (cos_y > 0.0f && p_l > 0.0) {
        st[ORC_ST_SHADOW_RAYS]++;
        v3 so = offset_origin(v->pos, v->n, v->err, v->ldir);
        if (!trace_any(s, c->b, so, v->ldir, dist * (1.0f - 1e-4f))) {
          double cos_x = fabs((double)vdot(v->n, v->ldir));
          double g = cos_x * (double)cos_y / ((double)dist2 * p_l);
          v->dE = cscale(light_le(s, s->lights[li].prim), g);
        }
      }
      float pp[3] = {v->pos.x, v->pos.y, v->pos.z};
      orc_octree_increment(oct, pp);
    }
    if (k == c->D) break;
    float ul = rng_u(&c->rng, (uint32_t)pixel, stream, 4);
    float u1 = rng_u(&c->rng, (uint32_t)pixel, stream, 5);
    float u2 = rng_u(&c->rng, (uint32_t)pixel, stream, 6);
    v3 wi;
    c3 w;
    if (!bsdf_sample(m, v->n, wo, ul, u1, u2, 1, &wi, &w)) break;
    tau = cmul(tau, w);
    if (!(cmax(tau) > 0.0)) break;
    o = offset_origin(v->pos, v->n, v->err, wi);
    d = wi;
  }
  return K;
}

/* fill MIS vertex array for the camera prefix v_0 .. v_k of a path */
static void mv_camera(const scene_t* s, const cv_t* path, int k, mv_t* mv, v3* u, float* L) {
  mv[0].mat = NULL;
  mv[0].delta = 0;
  for (int i = 1; i <= k; ++i) {
    mv[i].mat = &s->mats[path[i].mat];
    mv[i].n_bsdf = mv[i].n_in = mv[i].n_out = path[i].n;
    mv[i].delta = path[i].delta;
    u[i - 1] = path[i].din;
    L[i - 1] = path[i].tin;
  }
}

int orc_render(const orc_scene* scene_in, const orc_config* cfg, int n_iter, double* accum, double* last_split,
               float* nee_rho, int64_t* stats) {
  if (cfg->max_depth < 1 || cfg->max_depth > 60 || cfg->width <= 0 || cfg->height <= 0) return -1;
  scene_t s;
  scene_init(&s, scene_in);
  bvh_t b;
  bvh_build(&b, &s);
  ctx_t c;
  memset(&c, 0, sizeof(c));
  c.s = &s;
  c.b = &b;
  c.cfg = cfg;
  c.W = cfg->width;
  c.H = cfg->height;
  c.D = cfg->max_depth;
  c.r = cfg->merge_radius;
  c.rng.key[0] = (uint32_t)(cfg->seed & 0xffffffffu);
  c.rng.key[1] = (uint32_t)(cfg->seed >> 32);
  {
    const float* cm = scene_in->cam;
    c.eye = vload(cm);
    v3 target = vload(cm + 3), upv = vload(cm + 6);
    c.fwd = vnorm(vsub(target, c.eye));
    c.right = vnorm(vcross(c.fwd, upv));
    c.up = vcross(c.right, c.fwd);
    c.tanh_ = tanf(cm[9] * 3.14159265358979323846f / 360.0f);
    c.aspect = (float)c.W / (float)c.H;
  }
  int P = c.W * c.H, D = c.D;
  int pb = cfg->pixel_begin > 0 ? cfg->pixel_begin : 0;
  int pe = cfg->pixel_end > 0 ? cfg->pixel_end : P;
  if (pe > P) pe = P;
  int np = pe - pb > 0 ? pe - pb : 0;
  orc_octree* oct = orc_octree_new(s.bmin, s.bmax, cfg->octree_capacity, cfg->split_factor);
  double* before = NULL;   /* the sums before the current iteration, for iter_images */
  if (cfg->iter_images) {
    before = (double*)malloc(sizeof(double) * (size_t)P * 3);
    memcpy(before, accum, sizeof(double) * (size_t)P * 3);
  }
  cv_t* paths = (cv_t*)calloc((size_t)np * (D + 1), sizeof(cv_t));
  int* plen = (int*)calloc((size_t)(np > 0 ? np : 1), sizeof(int));
  rh_t* rh = (rh_t*)calloc((size_t)np * D + 1, sizeof(rh_t));
  mref_t* mref = (mref_t*)calloc((size_t)np * D + 1, sizeof(mref_t));
  int64_t st[ORC_ST_COUNT];
  memset(st, 0, sizeof(st));
  memset(accum, 0, sizeof(double) * (size_t)P * 3);
  double kernel = 1.0 / (PI_D * (double)c.r * (double)c.r);
  float r2 = c.r * c.r;
  int first = cfg->first_iteration > 0 ? cfg->first_iteration : 1;
  const double n_lp = (cfg->strategy_mask & 8u) ? (double)(cfg->lp_photons > 0 ? cfg->lp_photons : 0) : 0.0;

  for (int it = 0; it < n_iter; ++it) {
    double t_start = now_seconds();
    int iter = first + it;
    int last = it == n_iter - 1;
    c.rng.iter = (uint32_t)iter;
    if (last && last_split) memset(last_split, 0, sizeof(double) * 4 * (size_t)P * 3);
    orc_octree_set_iteration(oct, iter);
    /* ---- pass 1: view paths, NEE vertices into the octree, random hits ---- */
    int nrh = 0;
    for (int q = 0; q < np; ++q) {
      int pixel = pb + q;
      int K = trace_camera(&c, pixel, paths + (size_t)q * (D + 1), st, rh, &nrh, oct);
      plen[q] = K < 0 ? -K : K;
    }
    /* ---- pass 2a: densities ---- */
    for (int q = 0; q < np; ++q) {
      cv_t* path = paths + (size_t)q * (D + 1);
      for (int k = 1; k <= plen[q]; ++k) {
        if (!path[k].is_nee) continue;
        float pp[3] = {path[k].pos.x, path[k].pos.y, path[k].pos.z};
        float nn[3] = {path[k].n.x, path[k].n.y, path[k].n.z};
        path[k].rho = orc_octree_density(oct, pp, nn, cfg->density_mode == 0);
      }
    }
    if (last && nee_rho) {
      for (int i = 0; i < P * (D - 1); ++i) nee_rho[i] = -1.0f;
      for (int q = 0; q < np; ++q) {
        cv_t* path = paths + (size_t)q * (D + 1);
        for (int k = 1; k <= plen[q] && k <= D - 1; ++k)
          if (path[k].is_nee) nee_rho[(size_t)(pb + q) * (D - 1) + (k - 1)] = path[k].rho;
      }
    }
    mv_t mv[64];
    v3 u[64];
    float L[64];
    /* ---- pass 2b: NEE contributions ---- */
    if (cfg->strategy_mask & 2u) {
      for (int q = 0; q < np; ++q) {
        cv_t* path = paths + (size_t)q * (D + 1);
        for (int k = 1; k <= plen[q]; ++k) {
          cv_t* v = &path[k];
          if (!v->is_nee || v->delta || !(cmax(v->dE) > 0.0)) continue;
          const mat_t* m = &s.mats[v->mat];
          c3 f = bsdf_eval(m, v->n, vneg(v->din), v->ldir);
          if (!(cmax(f) > 0.0)) continue;
          mv_camera(&s, path, k, mv, u, L);
          u[k] = v->ldir;
          L[k] = v->ldist;
          mv[k + 1].mat = NULL;
          mv[k + 1].n_in = mv[k + 1].n_out = mv[k + 1].n_bsdf = v->ny;
          mv[k + 1].delta = 0;
          double w = mis_weight(mv, u, L, k + 1, v->p_l, v->rho, c.r, cfg->strategy_mask, n_lp,
                                lp_light_pdf(&s, v->light), 1, 0);
          c3 contrib = cscale(cmul(cmul(v->tau, f), v->dE), w);
          double* a = accum + (size_t)(pb + q) * 3;
          a[0] += contrib.r; a[1] += contrib.g; a[2] += contrib.b;
          if (last && last_split) {
            double* ls = last_split + (size_t)1 * P * 3 + (size_t)(pb + q) * 3;
            ls[0] += contrib.r; ls[1] += contrib.g; ls[2] += contrib.b;
          }
        }
      }
    }
    /* ---- pass 2c: photons from NEE vertices, merged at view vertices ---- */
    if ((cfg->strategy_mask & 4u) && D >= 3) {
      int nm = 0;
      for (int q = 0; q < np; ++q) {
        cv_t* path = paths + (size_t)q * (D + 1);
        for (int k = 1; k <= plen[q] && k <= D - 2; ++k) {
          if (!path[k].is_nee || path[k].delta) continue;
          mref[nm].x = path[k].pos.x;
          mref[nm].pixel = pb + q;
          mref[nm].k = k;
          nm++;
        }
      }
      qsort(mref, (size_t)nm, sizeof(mref_t), mref_cmp);
      for (int q = 0; q < np; ++q) {
        cv_t* path = paths + (size_t)q * (D + 1);
        for (int m = 1; m <= plen[q]; ++m) {
          cv_t* nv = &path[m];
          if (!nv->is_nee || !(cmax(nv->dE) > 0.0) || !(nv->rho > 0.0f)) continue;
          st[ORC_ST_PHOTONS]++;
          int pixel = pb + q;
          c3 phi = cscale(nv->dE, 1.0 / (double)nv->rho);
          /* photon vertex list: ph[0] = NEE vertex, ph[j] = hit j */
          v3 ph_n[64], ph_dir[64];
          float ph_t[64];
          int ph_mat[64];
          ph_n[0] = nv->n;
          ph_mat[0] = nv->mat;
          v3 wo_ph = nv->ldir; /* towards where the light came from */
          v3 pos = nv->pos, nrm = nv->n, perr = nv->err;
          const mat_t* pm = &s.mats[nv->mat];
          for (int j = 1; j <= D - 2; ++j) {
            uint32_t stream = (uint32_t)m * 256u + 1u + (uint32_t)(j - 1);
            float ul = rng_u(&c.rng, (uint32_t)pixel, stream, 4);
            float u1 = rng_u(&c.rng, (uint32_t)pixel, stream, 5);
            float u2 = rng_u(&c.rng, (uint32_t)pixel, stream, 6);
            v3 wi;
            c3 w;
            if (!bsdf_sample(pm, nrm, wo_ph, ul, u1, u2, 0, &wi, &w)) break;
            phi = cmul(phi, w);
            if (!(cmax(phi) > 0.0)) break;
            v3 o = offset_origin(pos, nrm, perr, wi);
            float t;
            int prim = trace_closest(&s, &b, o, wi, INFINITY, &t);
            if (prim < 0) break;
            v3 hp, herr;
            hit_point(&s, o, wi, prim, t, &hp, &herr);
            v3 hn = prim_normal(&s, prim, hp);
            int hm = s.prim_mat[prim];
            const mat_t* hmat = &s.mats[hm];
            ph_n[j] = hn;
            ph_mat[j] = hm;
            ph_dir[j] = wi;
            ph_t[j] = t;
            if (mat_black(hmat)) break;
            st[ORC_ST_PHOTON_HITS]++;
            if (!mat_delta(hmat)) {
              /* range search: view vertices with |x - hp|^2 <= r^2 */
              int lo = 0, hi = nm;
              float xlo = hp.x - c.r;
              while (lo < hi) { int mid = (lo + hi) / 2; if (mref[mid].x < xlo) lo = mid + 1; else hi = mid; }
              for (int ci = lo; ci < nm && mref[ci].x <= hp.x + c.r; ++ci) {
                int cpix = mref[ci].pixel, kk = mref[ci].k;
                if (kk + j + 1 > D) continue;
                cv_t* cpath = paths + (size_t)(cpix - pb) * (D + 1);
                cv_t* cvx = &cpath[kk];
                float dx = cvx->pos.x - hp.x, dy = cvx->pos.y - hp.y, dz = cvx->pos.z - hp.z;
                float d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 <= r2)) continue;
                const mat_t* cm = &s.mats[cvx->mat];
                c3 f = bsdf_eval(cm, cvx->n, vneg(cvx->din), vneg(wi));
                if (!(cmax(f) > 0.0)) continue;
                /* full path: camera v_0..v_kk, photon vertices ph[j-1] .. ph[0], light */
                int l = kk + j + 1;
                mv_camera(&s, cpath, kk, mv, u, L);
                mv[kk].n_out = hn;  /* photon side of the merge vertex */
                for (int i = 1; i <= j; ++i) {
                  int pi = j - i; /* path vertex kk+i is photon vertex pi */
                  mv[kk + i].mat = &s.mats[ph_mat[pi]];
                  mv[kk + i].n_bsdf = mv[kk + i].n_in = mv[kk + i].n_out = ph_n[pi];
                  mv[kk + i].delta = mat_delta(&s.mats[ph_mat[pi]]);
                  /* segment (kk+i-1, kk+i) is photon segment pi+1 reversed */
                  u[kk + i - 1] = vneg(ph_dir[pi + 1]);
                  L[kk + i - 1] = ph_t[pi + 1];
                }
                u[l - 1] = nv->ldir;
                L[l - 1] = nv->ldist;
                mv[l].mat = NULL;
                mv[l].n_in = mv[l].n_out = mv[l].n_bsdf = nv->ny;
                mv[l].delta = 0;
                double wgt = mis_weight(mv, u, L, l, nv->p_l, nv->rho, c.r, cfg->strategy_mask, n_lp,
                                        lp_light_pdf(&s, nv->light), 2, kk);
                c3 contrib = cscale(cmul(cmul(cvx->tau, f), phi), kernel * wgt);
                st[ORC_ST_MERGES]++;
                double* a = accum + (size_t)cpix * 3;
                a[0] += contrib.r; a[1] += contrib.g; a[2] += contrib.b;
                if (last && last_split) {
                  double* ls = last_split + (size_t)2 * P * 3 + (size_t)cpix * 3;
                  ls[0] += contrib.r; ls[1] += contrib.g; ls[2] += contrib.b;
                }
              }
            }
            if (j == D - 2) break;
            pos = hp;
            nrm = hn;
            perr = herr;
            pm = hmat;
            wo_ph = vneg(wi);
          }
        }
      }
    }
    /* ---- pass 2d: conventional light photons (Sec. 6.1), merged at view vertices ---- */
    if (n_lp > 0.0 && s.nl > 0 && D >= 2) {
      int nm = 0;  /* view vertices x_k, 1 <= k <= D-1, non-delta */
      for (int q = 0; q < np; ++q) {
        cv_t* path = paths + (size_t)q * (D + 1);
        for (int k = 1; k <= plen[q] && k <= D - 1; ++k) {
          if (!path[k].is_nee || path[k].delta) continue;
          mref[nm].x = path[k].pos.x;
          mref[nm].pixel = pb + q;
          mref[nm].k = k;
          nm++;
        }
      }
      qsort(mref, (size_t)nm, sizeof(mref_t), mref_cmp);
      for (int i = 0; i < cfg->lp_photons; ++i) {
        const uint32_t lpix = (uint32_t)i, st0 = ORC_LP_STREAM;
        int li = alias_pick(s.alias_prob, s.alias_idx, s.nl, rng_raw(&c.rng, lpix, st0, 0),
                            rng_u(&c.rng, lpix, st0, 1));
        float u2 = rng_u(&c.rng, lpix, st0, 2), u3 = rng_u(&c.rng, lpix, st0, 3);
        const light_t* Lt = &s.lights[li];
        v3 y, ny, yerr;
        if (Lt->kind == 0) {
          float b1 = u2, b2 = u3;
          if (b1 + b2 > 1.0f) { b1 = 1.0f - b1; b2 = 1.0f - b2; }
          v3 a = tri_v(&s, Lt->prim, 0), bb = tri_v(&s, Lt->prim, 1), cc = tri_v(&s, Lt->prim, 2);
          v3 e1 = vsub(bb, a), e2 = vsub(cc, a);
          y = vadd(vadd(a, vmul(e1, b1)), vmul(e2, b2));
          ny = vnorm(vcross(e1, e2));
          yerr = mk3(gamma_f32(5) * (fabsf(a.x) + fabsf(e1.x * b1) + fabsf(e2.x * b2)),
                     gamma_f32(5) * (fabsf(a.y) + fabsf(e1.y * b1) + fabsf(e2.y * b2)),
                     gamma_f32(5) * (fabsf(a.z) + fabsf(e1.z * b1) + fabsf(e2.z * b2)));
        } else {
          const float* sp = s.sph + (size_t)(Lt->prim - s.nt) * 4;
          v3 ce = vload(sp);
          float z = 1.0f - 2.0f * u2;
          float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
          float ph = TWO_PI_F * u3;
          ny = mk3(rr * cosf(ph), rr * sinf(ph), z);
          y = vadd(ce, vmul(ny, sp[3]));
          yerr = mk3(gamma_f32(5) * (fabsf(ce.x) + sp[3]), gamma_f32(5) * (fabsf(ce.y) + sp[3]), gamma_f32(5) * (fabsf(ce.z) + sp[3]));
        }
        const double p_lp = lp_light_pdf(&s, li);
        float u4 = rng_u(&c.rng, lpix, st0, 4), u5 = rng_u(&c.rng, lpix, st0, 5);
        float er = sqrtf(u4), eph = TWO_PI_F * u5, ez = sqrtf(fmaxf(0.0f, 1.0f - u4));
        v3 w = from_local(ny, er * cosf(eph), er * sinf(eph), ez);
        if (!(ez > 0.0f)) continue;
        st[ORC_ST_PHOTONS]++;
        /* flux Le cos / (p_lp cos / pi) / n_LP */
        c3 phi = cscale(light_le(&s, Lt->prim), PI_D / (p_lp * n_lp));
        const v3 yl = offset_origin(y, ny, yerr, w);  /* the light vertex of every LP path */
        v3 o = yl;
        v3 ph_n[64], ph_dir[64];
        float ph_t[64];
        int ph_mat[64];
        v3 dir = w, hp1 = mk3(0, 0, 0);
        double rho1 = 0.0, p_l1 = 0.0;
        for (int j = 1; j <= D - 1; ++j) {
          float t;
          int prim = trace_closest(&s, &b, o, dir, INFINITY, &t);
          if (prim < 0) break;
          v3 hp, herr;
          hit_point(&s, o, dir, prim, t, &hp, &herr);
          v3 hn = prim_normal(&s, prim, hp);
          int hm = s.prim_mat[prim];
          const mat_t* hmat = &s.mats[hm];
          ph_n[j] = hn;
          ph_mat[j] = hm;
          ph_dir[j] = dir;
          ph_t[j] = t;
          if (mat_black(hmat)) break;
          st[ORC_ST_PHOTON_HITS]++;
          if (j == 1) {
            /* light end of every LP path of this photon: density, NEE pdf
             * and the light segment at the first hit */
            float pp[3] = {hp.x, hp.y, hp.z}, nn[3] = {hn.x, hn.y, hn.z};
            rho1 = orc_octree_density(oct, pp, nn, cfg->density_mode == 0);
            p_l1 = light_pdf(&s, li, yl, hp);
            hp1 = hp;
          }
          if (!mat_delta(hmat)) {
            int lo = 0, hi = nm;
            float xlo = hp.x - c.r;
            while (lo < hi) { int mid = (lo + hi) / 2; if (mref[mid].x < xlo) lo = mid + 1; else hi = mid; }
            for (int ci = lo; ci < nm && mref[ci].x <= hp.x + c.r; ++ci) {
              int cpix = mref[ci].pixel, kk = mref[ci].k;
              if (kk + j > D) continue;
              cv_t* cpath = paths + (size_t)(cpix - pb) * (D + 1);
              cv_t* cvx = &cpath[kk];
              float dx = cvx->pos.x - hp.x, dy = cvx->pos.y - hp.y, dz = cvx->pos.z - hp.z;
              float d2 = dx * dx + dy * dy + dz * dz;
              if (!(d2 <= r2)) continue;
              const mat_t* cm = &s.mats[cvx->mat];
              c3 f = bsdf_eval(cm, cvx->n, vneg(cvx->din), vneg(dir));
              if (!(cmax(f) > 0.0)) continue;
              /* camera v_0..v_kk, photon hits j-1 .. 1, light vertex o */
              int l = kk + j;
              mv_camera(&s, cpath, kk, mv, u, L);
              mv[kk].n_out = hn;
              for (int q2 = 1; q2 <= j - 1; ++q2) {
                int pi = j - q2;
                mv[kk + q2].mat = &s.mats[ph_mat[pi]];
                mv[kk + q2].n_bsdf = mv[kk + q2].n_in = mv[kk + q2].n_out = ph_n[pi];
                mv[kk + q2].delta = mat_delta(&s.mats[ph_mat[pi]]);
                u[kk + q2 - 1] = vneg(ph_dir[pi + 1]);
                L[kk + q2 - 1] = ph_t[pi + 1];
              }
              v3 ls = vsub(yl, hp1);
              u[l - 1] = vneg(w);
              L[l - 1] = sqrtf(vdot(ls, ls));
              mv[l].mat = NULL;
              mv[l].n_in = mv[l].n_out = mv[l].n_bsdf = ny;
              mv[l].delta = 0;
              double wgt = mis_weight(mv, u, L, l, p_l1, rho1, c.r, cfg->strategy_mask, n_lp, p_lp, 3, kk);
              c3 contrib = cscale(cmul(cmul(cvx->tau, f), phi), kernel * wgt);
              st[ORC_ST_MERGES]++;
              double* a = accum + (size_t)cpix * 3;
              a[0] += contrib.r; a[1] += contrib.g; a[2] += contrib.b;
              if (last && last_split) {
                double* ls3 = last_split + (size_t)3 * P * 3 + (size_t)cpix * 3;
                ls3[0] += contrib.r; ls3[1] += contrib.g; ls3[2] += contrib.b;
              }
            }
          }
          if (j == D - 1) break;
          float ul = rng_u(&c.rng, lpix, st0 + (uint32_t)j, 4);
          float ub1 = rng_u(&c.rng, lpix, st0 + (uint32_t)j, 5);
          float ub2 = rng_u(&c.rng, lpix, st0 + (uint32_t)j, 6);
          v3 wi;
          c3 wt;
          if (!bsdf_sample(hmat, hn, vneg(dir), ul, ub1, ub2, 0, &wi, &wt)) break;
          phi = cmul(phi, wt);
          if (!(cmax(phi) > 0.0)) break;
          o = offset_origin(hp, hn, herr, wi);
          dir = wi;
        }
      }
    }
    /* ---- pass 3: self emission of the stored random hits ---- */
    if (cfg->strategy_mask & 1u) {
      for (int e = 0; e < nrh; ++e) {
        int pixel = rh[e].pixel, k = rh[e].k;
        cv_t* path = paths + (size_t)(pixel - pb) * (D + 1);
        cv_t* v = &path[k];
        double w = 1.0;
        if (k >= 2) {
          cv_t* prev = &path[k - 1];
          int li = s.prim_light[v->prim];
          double p_l = light_pdf(&s, li, v->pos, prev->pos);
          mv_camera(&s, path, k, mv, u, L);
          mv[k].mat = NULL;
          mv[k].n_in = mv[k].n_out = mv[k].n_bsdf = v->n;
          mv[k].delta = 0;
          w = mis_weight(mv, u, L, k, p_l, prev->rho, c.r, cfg->strategy_mask, n_lp, lp_light_pdf(&s, li), 0, 0);
        }
        c3 contrib = cscale(cmul(v->tau, rh[e].le), w);
        double* a = accum + (size_t)pixel * 3;
        a[0] += contrib.r; a[1] += contrib.g; a[2] += contrib.b;
        if (last && last_split) {
          double* ls = last_split + (size_t)pixel * 3;
          ls[0] += contrib.r; ls[1] += contrib.g; ls[2] += contrib.b;
        }
      }
    }
    if (cfg->iter_seconds) cfg->iter_seconds[it] = now_seconds() - t_start;
    if (cfg->iter_images) {
      double* img = cfg->iter_images + (size_t)it * (size_t)P * 3;
      for (size_t j = 0; j < (size_t)P * 3; ++j) {
        img[j] = accum[j] - before[j];
        before[j] = accum[j];
      }
    }
  }
  free(before);
  st[ORC_ST_OCTREE_NODES] = oct->words_used < oct->capacity ? oct->words_used : oct->capacity;
  st[ORC_ST_OCTREE_DEPTH] = oct->depth;
  if (stats) memcpy(stats, st, sizeof(st));
  orc_octree_free(oct);
  free(paths); free(plen); free(rh); free(mref);
  bvh_free(&b);
  scene_free(&s);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* helpers for the pin tests                                                 */
/* ------------------------------------------------------------------------ */
int orc_trace(const orc_scene* scene_in, const float* rays, int n, int brute, int32_t* out_prim, float* out_t) {
  scene_t s;
  scene_init(&s, scene_in);
  bvh_t b;
  if (!brute) bvh_build(&b, &s);
  for (int i = 0; i < n; ++i) {
    v3 o = vload(rays + (size_t)i * 6), d = vload(rays + (size_t)i * 6 + 3);
    float t = INFINITY;
    int p = brute ? trace_brute(&s, o, d, INFINITY, &t) : trace_closest(&s, &b, o, d, INFINITY, &t);
    out_prim[i] = p;
    out_t[i] = p >= 0 ? t : INFINITY;
  }
  if (!brute) bvh_free(&b);
  scene_free(&s);
  return 0;
}

static int fcmp(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

void orc_density_naive(const float* pts, int n, float radius, float* out) {
  float r2 = radius * radius;
  double inv_area = 1.0 / (PI_D * (double)radius * (double)radius);
  for (int i = 0; i < n; ++i) {
    int cnt = 0;
    for (int j = 0; j < n; ++j) {
      float dx = pts[3 * j] - pts[3 * i], dy = pts[3 * j + 1] - pts[3 * i + 1], dz = pts[3 * j + 2] - pts[3 * i + 2];
      if (dx * dx + dy * dy + dz * dz <= r2) cnt++;
    }
    out[i] = (float)((double)cnt * inv_area);
  }
}

void orc_density_knn(const float* pts, int n, int k, float* out) {
  float* best = (float*)malloc(sizeof(float) * (size_t)(k > 0 ? k : 1));
  for (int i = 0; i < n; ++i) {
    int have = 0;  /* best[0..have) ascending, the k smallest so far */
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      float dx = pts[3 * j] - pts[3 * i], dy = pts[3 * j + 1] - pts[3 * i + 1], dz = pts[3 * j + 2] - pts[3 * i + 2];
      float d2 = dx * dx + dy * dy + dz * dz;
      if (have == k && !(d2 < best[k - 1])) continue;
      int at = have < k ? have++ : k - 1;
      while (at > 0 && best[at - 1] > d2) {
        best[at] = best[at - 1];
        at--;
      }
      best[at] = d2;
    }
    out[i] = have == k ? (float)((double)(k - 1) / (PI_D * (double)best[k - 1])) : 0.0f;
  }
  free(best);
}

void orc_count_neighbours(const float* pts, int n, const float* queries, int m, float r, int brute,
                          int32_t* out_count) {
  float r2 = r * r;
  if (brute) {
    for (int q = 0; q < m; ++q) {
      int cnt = 0;
      for (int i = 0; i < n; ++i) {
        float dx = pts[i * 3] - queries[q * 3], dy = pts[i * 3 + 1] - queries[q * 3 + 1],
              dz = pts[i * 3 + 2] - queries[q * 3 + 2];
        if (dx * dx + dy * dy + dz * dz <= r2) cnt++;
      }
      out_count[q] = cnt;
    }
    return;
  }
  /* sorted-window search as used by orc_render (x, then index) */
  float* xs = (float*)malloc(sizeof(float) * 4 * (n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) {
    xs[i * 4] = pts[i * 3];
    xs[i * 4 + 1] = pts[i * 3 + 1];
    xs[i * 4 + 2] = pts[i * 3 + 2];
    xs[i * 4 + 3] = 0;
  }
  qsort(xs, (size_t)n, sizeof(float) * 4, fcmp);
  for (int q = 0; q < m; ++q) {
    float hx = queries[q * 3], hy = queries[q * 3 + 1], hz = queries[q * 3 + 2];
    int lo = 0, hi = n;
    float xlo = hx - r;
    while (lo < hi) { int mid = (lo + hi) / 2; if (xs[mid * 4] < xlo) lo = mid + 1; else hi = mid; }
    int cnt = 0;
    for (int i = lo; i < n && xs[i * 4] <= hx + r; ++i) {
      float dx = xs[i * 4] - hx, dy = xs[i * 4 + 1] - hy, dz = xs[i * 4 + 2] - hz;
      if (dx * dx + dy * dy + dz * dz <= r2) cnt++;
    }
    out_count[q] = cnt;
  }
  free(xs);
}

/* BSDF sampling probe for the pin tests: material row m[12] (scenes layout),
 * geometric normal n, outgoing direction wo, random numbers u[3] (lobe, dir1,
 * dir2).  Writes wi[3], weight[3] (f |cos| / pdf) and returns 1, or 0 when the
 * sample is rejected.  pdf_out receives bsdf_pdf(wo -> wi), f_out f(wo, wi). */
int orc_bsdf_probe(const float* mrow, const float* n, const float* wo, const float* u, int camera, float* wi,
                   double* weight, double* pdf_out, double* f_out) {
  mat_t m;
  m.type = (int)mrow[0];
  for (int c = 0; c < 3; ++c) { m.albedo[c] = mrow[1 + c]; m.emission[c] = mrow[4 + c]; }
  m.ior = mrow[7];
  m.alpha = mrow[8];
  v3 w;
  c3 wt;
  int ok = bsdf_sample(&m, vload(n), vload(wo), u[0], u[1], u[2], camera, &w, &wt);
  wi[0] = w.x; wi[1] = w.y; wi[2] = w.z;
  weight[0] = wt.r; weight[1] = wt.g; weight[2] = wt.b;
  if (ok) {
    *pdf_out = bsdf_pdf(&m, vload(n), vload(wo), w);
    c3 f = bsdf_eval(&m, vload(n), vload(wo), w);
    f_out[0] = f.r; f_out[1] = f.g; f_out[2] = f.b;
  }
  return ok;
}

/* f(wo, wi) and pdf(wo -> wi) for arbitrary directions (pin tests). */
void orc_bsdf_eval_probe(const float* mrow, const float* n, const float* wo, const float* wi, double* f_out,
                         double* pdf_out) {
  mat_t m;
  m.type = (int)mrow[0];
  for (int c = 0; c < 3; ++c) { m.albedo[c] = mrow[1 + c]; m.emission[c] = mrow[4 + c]; }
  m.ior = mrow[7];
  m.alpha = mrow[8];
  c3 f = bsdf_eval(&m, vload(n), vload(wo), vload(wi));
  f_out[0] = f.r; f_out[1] = f.g; f_out[2] = f.b;
  *pdf_out = bsdf_pdf(&m, vload(n), vload(wo), vload(wi));
}
