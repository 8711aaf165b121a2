// neb_device.cuh -- device building blocks of the NEB pass (sm_103a).
//
// Everything here is written for FP32 IEEE rounding without contraction:
// the library is compiled with -fmad=false so that geometry, sampling
// decisions and the density octree round exactly like a plain C
// implementation of the same formulas.  Where a fused multiply-add is
// wanted it is written explicitly (__fmaf_rn).
#pragma once
#include <cfloat>
#include <cstdint>
#include <cuda_runtime.h>

#include "neb_types.h"

namespace neb {

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__host__ __device__ __forceinline__ float3 add(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ __forceinline__ float3 sub(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ __forceinline__ float3 mul(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__host__ __device__ __forceinline__ float3 cmul(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__host__ __device__ __forceinline__ float3 neg(float3 a) { return f3(-a.x, -a.y, -a.z); }
__host__ __device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float3 normalize(float3 a) {
  float l = sqrtf(dot(a, a));
  float inv = 1.0f / l;
  return mul(a, inv);
}
__host__ __device__ __forceinline__ float comp(float3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
__host__ __device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
__host__ __device__ __forceinline__ float maxc(float3 a) { return fmaxf(a.x, fmaxf(a.y, a.z)); }

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kInvPi = 0.318309886183790671538f;
constexpr float kPi = 3.14159265358979323846f;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64 bit multiplies with a Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
#ifdef __CUDA_ARCH__
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
#else
    uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
#endif
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Random numbers are addressed by (pixel, stream, dim, iteration):
// counter = (pixel, stream, dim / 4, iteration), lane dim % 4.
// stream = 256 k for view vertex k; 256 k + 1 + s for the s-th scattering of
// the photon that leaves NEE vertex k.  Dims per vertex: 0 light index,
// 1 alias acceptance, 2-3 point on the light, 4 lobe, 5-6 direction; the
// pixel jitter uses dims 0-1 of stream 0.
struct Rng4 {
  uint4 a;
};
__device__ __forceinline__ uint4 rng_block(uint2 key, uint32_t iter, uint32_t pixel, uint32_t stream, uint32_t blk) {
  return philox4x32_10(make_uint4(pixel, stream, blk, iter), key);
}
__host__ __device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }

// ---------------------------------------------------------------------------
// orthonormal basis (Duff et al., "Building an Orthonormal Basis, Revisited", JCGT 2017)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
  float sign = copysignf(1.0f, n.z);
  float a = -1.0f / (sign + n.z);
  float bb = n.x * n.y * a;
  t = f3(1.0f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
  b = f3(bb, sign + n.y * n.y * a, -n.y);
}
__device__ __forceinline__ float3 from_local(float3 n, float lx, float ly, float lz) {
  float3 t, b;
  onb(n, t, b);
  return add(add(mul(t, lx), mul(b, ly)), mul(n, lz));
}

// ---------------------------------------------------------------------------
// materials
// ---------------------------------------------------------------------------
struct Mat {
  int type;
  float3 albedo, emission;
  float ior, alpha;
};
__device__ __forceinline__ Mat load_mat(const float4* __restrict__ mats, int m) {
  float4 a = __ldg(mats + 3 * m), b = __ldg(mats + 3 * m + 1), c = __ldg(mats + 3 * m + 2);
  Mat r;
  r.type = __float_as_int(a.x);
  r.albedo = f3(a.y, a.z, a.w);
  r.emission = f3(b.x, b.y, b.z);
  r.ior = b.w;
  r.alpha = c.x;
  return r;
}
__device__ __forceinline__ bool mat_black(const Mat& m) {
  return m.type == MAT_DIFFUSE && m.albedo.x <= 0.0f && m.albedo.y <= 0.0f && m.albedo.z <= 0.0f;
}
__device__ __forceinline__ bool mat_delta(const Mat& m) { return m.type == MAT_DIELECTRIC; }

__device__ __forceinline__ float ggx_D(float alpha, float ch) {
  float a2 = alpha * alpha;
  float t = ch * ch * (a2 - 1.0f) + 1.0f;
  return a2 / (kPi * t * t);
}
__device__ __forceinline__ float ggx_G1(float alpha, float c) {
  float a2 = alpha * alpha;
  return 2.0f * c / (c + sqrtf(a2 + (1.0f - a2) * c * c));
}

// BSDF value f(wo, wi); zero for delta lobes.
__device__ __forceinline__ float3 bsdf_eval(const Mat& m, float3 n, float3 wo, float3 wi) {
  float co = dot(n, wo), ci = dot(n, wi);
  if (!(co * ci > 0.0f)) return f3(0, 0, 0);
  if (m.type == MAT_DIFFUSE) return mul(m.albedo, kInvPi);
  if (m.type == MAT_GGX) {
    float3 ns = co >= 0.0f ? n : neg(n);
    float cos_o = fabsf(co), cos_i = fabsf(ci);
    float3 h = normalize(add(wo, wi));
    float ch = dot(ns, h);
    if (!(ch > 0.0f)) return f3(0, 0, 0);
    float D = ggx_D(m.alpha, ch);
    float G = ggx_G1(m.alpha, cos_o) * ggx_G1(m.alpha, cos_i);
    float x = 1.0f - fabsf(dot(wo, h));
    float x5 = x * x * x * x * x;
    float k = D * G / (4.0f * cos_o * cos_i);
    return f3((m.albedo.x + (1.0f - m.albedo.x) * x5) * k, (m.albedo.y + (1.0f - m.albedo.y) * x5) * k,
              (m.albedo.z + (1.0f - m.albedo.z) * x5) * k);
  }
  return f3(0, 0, 0);
}

// Directional pdf of sampling wi given wo; 1 for the delta lobes (the lobe
// probability times a Dirac is common to every strategy that can create the
// path and cancels in the MIS weights).
__device__ __forceinline__ float bsdf_pdf(const Mat& m, float3 n, float3 wo, float3 wi) {
  if (m.type == MAT_DIELECTRIC) return 1.0f;
  float co = dot(n, wo), ci = dot(n, wi);
  if (!(co * ci > 0.0f)) return 0.0f;
  if (m.type == MAT_DIFFUSE) return fabsf(ci) * kInvPi;
  float3 ns = co >= 0.0f ? n : neg(n);
  float3 h = normalize(add(wo, wi));
  float ch = dot(ns, h);
  if (!(ch > 0.0f)) return 0.0f;
  return ggx_D(m.alpha, ch) * ch / (4.0f * fabsf(dot(wo, h)));
}

// Samples wi given wo.  weight = f |cos| / pdf (with the (eta_i/eta_t)^2
// radiance scaling on refraction for camera paths), pdf_fwd = pdf(wo->wi),
// pdf_rev = pdf(wi->wo).  Returns false when the sample is rejected.
__device__ __forceinline__ bool bsdf_sample(const Mat& m, float3 n, float3 wo, float ul, float u1, float u2,
                                            bool camera, float3& wi, float3& weight, float& pdf_fwd,
                                            float& pdf_rev) {
  float co = dot(n, wo);
  float3 ns = co >= 0.0f ? n : neg(n);
  if (m.type == MAT_DIFFUSE) {
    float r = sqrtf(u1);
    float phi = kTwoPi * u2;
    float lz = sqrtf(fmaxf(0.0f, 1.0f - u1));
    wi = from_local(ns, r * cosf(phi), r * sinf(phi), lz);
    if (!(lz > 0.0f)) return false;
    weight = m.albedo;
    pdf_fwd = bsdf_pdf(m, n, wo, wi);
    pdf_rev = bsdf_pdf(m, n, wi, wo);
    return true;
  }
  if (m.type == MAT_DIELECTRIC) {
    bool entering = co > 0.0f;
    float eta = entering ? 1.0f / m.ior : m.ior;
    float cos_i = dot(ns, wo);
    float sin2_t = eta * eta * (1.0f - cos_i * cos_i);
    float F = 1.0f, cos_t = 0.0f;
    if (sin2_t < 1.0f) {
      cos_t = sqrtf(1.0f - sin2_t);
      float rs = (eta * cos_i - cos_t) / (eta * cos_i + cos_t);
      float rp = (cos_i - eta * cos_t) / (cos_i + eta * cos_t);
      F = 0.5f * (rs * rs + rp * rp);
    }
    if (ul < F) {
      wi = sub(mul(ns, 2.0f * cos_i), wo);
      weight = f3(1, 1, 1);
    } else {
      wi = add(mul(wo, -eta), mul(ns, eta * cos_i - cos_t));
      float s = camera ? eta * eta : 1.0f;
      weight = f3(s, s, s);
    }
    pdf_fwd = 1.0f;
    pdf_rev = 1.0f;
    return true;
  }
  // GGX conductor: half vector from D(h) cos(h)
  float a2 = m.alpha * m.alpha;
  float tan2 = a2 * u1 / (1.0f - u1);
  float ch = 1.0f / sqrtf(1.0f + tan2);
  float sh = sqrtf(fmaxf(0.0f, 1.0f - ch * ch));
  float phi = kTwoPi * u2;
  float3 h = from_local(ns, sh * cosf(phi), sh * sinf(phi), ch);
  float oh = dot(wo, h);
  wi = sub(mul(h, 2.0f * oh), wo);
  if (!(dot(ns, wi) > 0.0f) || !(co > 0.0f || co < 0.0f)) return false;
  float3 f = bsdf_eval(m, n, wo, wi);
  float pdf = bsdf_pdf(m, n, wo, wi);
  if (!(pdf > 0.0f)) return false;
  float c = fabsf(dot(n, wi)) / pdf;
  weight = mul(f, c);
  pdf_fwd = pdf;
  pdf_rev = bsdf_pdf(m, n, wi, wo);
  return true;
}

// ---------------------------------------------------------------------------
// ray / primitive intersection
// ---------------------------------------------------------------------------
#define NEB_GAMMA2 1.19209304e-07f
#define NEB_GAMMA3 1.78813966e-07f
#define NEB_GAMMA5 2.98023313e-07f
#define NEB_GAMMA7 4.17232688e-07f

// Octahedral unit-vector code with 16 bits per coordinate (Meyer et al.,
// "On Floating-Point Normal Vectors", EGSR 2010): project onto the octahedron
// |x| + |y| + |z| = 1, fold the lower half over the diagonals, round each
// coordinate to a signed 16-bit integer.  Angular error about 3e-5 rad.
__device__ __forceinline__ float2 oct_fold(float px, float py) {
  return make_float2((1.0f - fabsf(py)) * (px >= 0.0f ? 1.0f : -1.0f),
                     (1.0f - fabsf(px)) * (py >= 0.0f ? 1.0f : -1.0f));
}
__device__ __forceinline__ uint32_t oct_encode16(float3 n) {
  float s = fabsf(n.x) + fabsf(n.y) + fabsf(n.z);
  float px = n.x / s, py = n.y / s;
  if (n.z < 0.0f) {
    float2 f = oct_fold(px, py);
    px = f.x;
    py = f.y;
  }
  int qx = __float2int_rn(fminf(fmaxf(px, -1.0f), 1.0f) * 32767.0f);
  int qy = __float2int_rn(fminf(fmaxf(py, -1.0f), 1.0f) * 32767.0f);
  return (uint32_t)(qx & 0xffff) | ((uint32_t)(qy & 0xffff) << 16);
}
__device__ __forceinline__ float3 oct_decode16(uint32_t v) {
  float px = (float)(short)(v & 0xffffu) * (1.0f / 32767.0f), py = (float)(short)(v >> 16) * (1.0f / 32767.0f);
  float nz = 1.0f - fabsf(px) - fabsf(py);
  if (nz < 0.0f) {
    float2 f = oct_fold(px, py);
    px = f.x;
    py = f.y;
  }
  float l = sqrtf(px * px + py * py + nz * nz);
  return make_float3(px / l, py / l, nz / l);
}

// Bucket of grid cell (x, y, z) in a hash table of mask + 1 buckets (Teschner
// et al., "Optimized Spatial Hashing for Collision Detection of Deformable
// Objects", VMV 2003).  The merge grid, its builder and the stand-alone point
// grids all use this one function.
// Cell index of grid coordinate g (position / cell size): floor(g), held
// within +-2^30 so that far points or a tiny cell cannot overflow the
// integer; points beyond that all share the boundary cell, and since every
// candidate is checked by its distance, counts stay exact.
__device__ __forceinline__ int grid_cell_index(float g) {
  return (int)fminf(fmaxf(floorf(g), -1073741824.0f), 1073741824.0f);
}

__device__ __forceinline__ uint32_t grid_hash(int x, int y, int z, uint32_t mask) {
  return (((uint32_t)x * 73856093u) ^ ((uint32_t)y * 19349663u) ^ ((uint32_t)z * 83492791u)) & mask;
}

struct RayPre {
  float3 o, d, inv;
  int kx, ky, kz;
  float Sx, Sy, Sz;
  int oct;  // bit a set when direction component a has its sign bit set
};

__device__ __forceinline__ RayPre make_ray(float3 o, float3 d) {
  RayPre r;
  r.o = o;
  r.d = d;
  r.inv = f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  r.oct = (signbit(d.x) ? 1 : 0) | (signbit(d.y) ? 2 : 0) | (signbit(d.z) ? 4 : 0);
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  if (comp(d, kz) < 0.0f) { int t = kx; kx = ky; ky = t; }
  r.kx = kx; r.ky = ky; r.kz = kz;
  float dz = comp(d, kz);
  r.Sx = comp(d, kx) / dz;
  r.Sy = comp(d, ky) / dz;
  r.Sz = 1.0f / dz;
  return r;
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013) with its
// FP64 re-evaluation of zero edge functions and the conservative lower bound
// deltaT on t of PBRT 3rd ed. Sec. 3.9.6 (hits within the test's own rounding
// error of the origin are rejected).  Returns t > deltaT or -1.
__device__ __forceinline__ float isect_tri(const RayPre& r, float3 v0, float3 v1, float3 v2, float* bary) {
  float3 A = sub(v0, r.o), B = sub(v1, r.o), C = sub(v2, r.o);
  float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
  float Ax = comp(A, r.kx) - r.Sx * Akz;
  float Ay = comp(A, r.ky) - r.Sy * Akz;
  float Bx = comp(B, r.kx) - r.Sx * Bkz;
  float By = comp(B, r.ky) - r.Sy * Bkz;
  float Cx = comp(C, r.kx) - r.Sx * Ckz;
  float Cy = comp(C, r.ky) - r.Sy * Ckz;
  float U = Cx * By - Cy * Bx;
  float V = Ax * Cy - Ay * Cx;
  float W = Bx * Ay - By * Ax;
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
    V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
    W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
  float det = U + V + W;
  if (det == 0.0f) return -1.0f;
  float Az = r.Sz * Akz, Bz = r.Sz * Bkz, Cz = r.Sz * Ckz;
  float T = U * Az + V * Bz + W * Cz;
  float Ts = T, dets = det;
  if (dets < 0.0f) { Ts = -Ts; dets = -dets; }
  if (Ts <= 0.0f) return -1.0f;
  float t = Ts / dets;
  float maxZ = fmaxf(fabsf(Az), fmaxf(fabsf(Bz), fabsf(Cz)));
  float maxX = fmaxf(fabsf(Ax), fmaxf(fabsf(Bx), fabsf(Cx)));
  float maxY = fmaxf(fabsf(Ay), fmaxf(fabsf(By), fabsf(Cy)));
  float maxE = fmaxf(fabsf(U), fmaxf(fabsf(V), fabsf(W)));
  float dZ = NEB_GAMMA3 * maxZ;
  float dX = NEB_GAMMA5 * (maxX + maxZ);
  float dY = NEB_GAMMA5 * (maxY + maxZ);
  float dE = 2.0f * (NEB_GAMMA2 * maxX * maxY + dY * maxX + dX * maxY);
  float dT = 3.0f * (NEB_GAMMA3 * maxE * maxZ + dE * maxZ + dZ * maxE) / dets;
  if (!(t > dT)) return -1.0f;
  if (bary) { bary[0] = U / det; bary[1] = V / det; bary[2] = W / det; }
  return t;
}

// Ray/sphere with the cancellation-free discriminant of Haines et al.,
// "Precision Improvements for Ray/Sphere Intersection" (Ray Tracing Gems 2019).
__device__ __forceinline__ float isect_sph(const RayPre& r, float4 sp) {
  float3 c = xyz(sp);
  float R = sp.w;
  float3 oc = sub(r.o, c);
  float b = dot(oc, r.d);
  float3 qv = sub(oc, mul(r.d, b));
  float disc = R * R - dot(qv, qv);
  if (disc < 0.0f) return -1.0f;
  float c2 = dot(oc, oc) - R * R;
  float sq = sqrtf(disc);
  float q = (b > 0.0f) ? (-b - sq) : (-b + sq);
  if (q == 0.0f) return -1.0f;
  float t0 = c2 / q, t1 = q;
  if (t0 > t1) { float t = t0; t0 = t1; t1 = t; }
  float t = (t0 > 0.0f) ? t0 : t1;
  if (!(t > 0.0f)) return -1.0f;
  return t;
}

// slab test, far distance widened by 1 + 2 gamma_3 (PBRT 3rd ed. Sec. 3.9.2)
__device__ __forceinline__ bool box_hit(float3 lo, float3 hi, const RayPre& r, float tmax, float& tnear) {
  float t0 = 0.0f, t1 = tmax;
  {
    float tn = (lo.x - r.o.x) * r.inv.x, tf = (hi.x - r.o.x) * r.inv.x;
    if (tn > tf) { float t = tn; tn = tf; tf = t; }
    tf *= 1.0000004f;
    t0 = fmaxf(t0, tn);
    t1 = fminf(t1, tf);
  }
  {
    float tn = (lo.y - r.o.y) * r.inv.y, tf = (hi.y - r.o.y) * r.inv.y;
    if (tn > tf) { float t = tn; tn = tf; tf = t; }
    tf *= 1.0000004f;
    t0 = fmaxf(t0, tn);
    t1 = fminf(t1, tf);
  }
  {
    float tn = (lo.z - r.o.z) * r.inv.z, tf = (hi.z - r.o.z) * r.inv.z;
    if (tn > tf) { float t = tn; tn = tf; tf = t; }
    tf *= 1.0000004f;
    t0 = fmaxf(t0, tn);
    t1 = fminf(t1, tf);
  }
  tnear = t0;
  return t0 <= t1;
}

// ---------------------------------------------------------------------------
// scene view + BVH traversal
// ---------------------------------------------------------------------------
struct SceneView {
  const float4* __restrict__ tv0;  // xyz v0, w = material (int bits)
  const float4* __restrict__ tv1;
  const float4* __restrict__ tv2;
  const float4* __restrict__ sph;  // centre, radius
  const int* __restrict__ sph_mat;
  const float4* __restrict__ mats; // 3 float4 per material
  const BVH4Node* __restrict__ nodes;
  const int* __restrict__ prim_light;
  const int* __restrict__ light_prim;
  const float* __restrict__ light_psel;
  const float* __restrict__ light_inv_area;  // triangles: 1/area
  const float* __restrict__ alias_prob;
  const int* __restrict__ alias_idx;
  int nt, ns, nl;
};

__device__ __forceinline__ int prim_mat(const SceneView& s, int p) {
  return p < s.nt ? __float_as_int(__ldg(&s.tv0[p].w)) : __ldg(&s.sph_mat[p - s.nt]);
}

__device__ __forceinline__ float isect_prim(const SceneView& s, const RayPre& r, int p) {
  if (p < s.nt) return isect_tri(r, xyz(__ldg(s.tv0 + p)), xyz(__ldg(s.tv1 + p)), xyz(__ldg(s.tv2 + p)), nullptr);
  return isect_sph(r, __ldg(s.sph + (p - s.nt)));
}

// ---- BVH4 traversal --------------------------------------------------------------
// A 4-wide node keeps, per axis, the low and the high bounds of its four
// children in one float4 each.  On axis a the entry plane of every child is
// its low bound when the ray's direction component is positive and its high
// bound when it is negative, so the walk loads the entry and exit planes
// directly by the ray's octant and needs no per-child compare and swap.  The
// slab distances are those of box_hit: the decisions are the same for every
// non-zero direction component (a zero component gives NaN planes, which
// both forms ignore).
struct Node4Oct {
  float4 nx, fx, ny, fy, nz, fz;  // entry / exit planes per axis, children 0-3
  int4 ch;
};
__device__ __forceinline__ Node4Oct load_node4_oct(const BVH4Node* __restrict__ nodes, int i, int oct) {
  const float4* p = reinterpret_cast<const float4*>(nodes + i);
  const int ox = oct & 1, oy = (oct >> 1) & 1, oz = (oct >> 2) & 1;
  Node4Oct n;
  n.nx = __ldg(p + ox);
  n.fx = __ldg(p + (1 - ox));
  n.ny = __ldg(p + 2 + oy);
  n.fy = __ldg(p + 3 - oy);
  n.nz = __ldg(p + 4 + oz);
  n.fz = __ldg(p + 5 - oz);
  n.ch = __ldg(reinterpret_cast<const int4*>(p + 6));
  return n;
}
__device__ __forceinline__ float comp4(float4 v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w)); }
__device__ __forceinline__ int comp4i(int4 v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w)); }

// Walks take only rays with a finite origin and direction.  The slab test
// drops NaN distances, so a ray with a NaN component would enter every child
// slot, the empty ones (inverted infinite boxes) included; such a ray hits
// nothing and is settled before its walk, as a walk of it would settle it.
__device__ __forceinline__ bool ray_finite(float3 o, float3 d) {
  return fabsf(o.x) <= FLT_MAX && fabsf(o.y) <= FLT_MAX && fabsf(o.z) <= FLT_MAX && fabsf(d.x) <= FLT_MAX &&
         fabsf(d.y) <= FLT_MAX && fabsf(d.z) <= FLT_MAX;
}

// Three-input FP32 minimum and maximum (sm_100 and later); NaN inputs drop
// out as they do from nested fminf / fmaxf.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Slab distances (plane - o) * inv of two children on one axis, with one
// packed FP32x2 add and one packed multiply: each half rounds like the scalar
// subtract and multiply (plane + (-o) is plane - o exactly).
__device__ __forceinline__ float2 slab2(float a, float b, float no, float inv) {
  return __fmul2_rn(__fadd2_rn(make_float2(a, b), make_float2(no, no)), make_float2(inv, inv));
}

// Slab tests of the four children: entry = max(0, entry planes), exit =
// min(tmax, exit planes widened by 1 + 2 gamma_3); NaN distances drop out of
// the minimum and maximum.  Returns the mask of children whose box is hit
// before tmax and their entry distances.
__device__ __forceinline__ uint32_t child_hits4(const Node4Oct& n, const RayPre& r, float tmax, float (&tn)[4]) {
  const float nox = -r.o.x, noy = -r.o.y, noz = -r.o.z;
  const float2 nx01 = slab2(n.nx.x, n.nx.y, nox, r.inv.x), nx23 = slab2(n.nx.z, n.nx.w, nox, r.inv.x);
  const float2 ny01 = slab2(n.ny.x, n.ny.y, noy, r.inv.y), ny23 = slab2(n.ny.z, n.ny.w, noy, r.inv.y);
  const float2 nz01 = slab2(n.nz.x, n.nz.y, noz, r.inv.z), nz23 = slab2(n.nz.z, n.nz.w, noz, r.inv.z);
  const float2 fx01 = slab2(n.fx.x, n.fx.y, nox, r.inv.x), fx23 = slab2(n.fx.z, n.fx.w, nox, r.inv.x);
  const float2 fy01 = slab2(n.fy.x, n.fy.y, noy, r.inv.y), fy23 = slab2(n.fy.z, n.fy.w, noy, r.inv.y);
  const float2 fz01 = slab2(n.fz.x, n.fz.y, noz, r.inv.z), fz23 = slab2(n.fz.z, n.fz.w, noz, r.inv.z);
  const float ex[4] = {nx01.x, nx01.y, nx23.x, nx23.y}, ey[4] = {ny01.x, ny01.y, ny23.x, ny23.y},
              ez[4] = {nz01.x, nz01.y, nz23.x, nz23.y};
  const float gx[4] = {fx01.x, fx01.y, fx23.x, fx23.y}, gy[4] = {fy01.x, fy01.y, fy23.x, fy23.y},
              gz[4] = {fz01.x, fz01.y, fz23.x, fz23.y};
  uint32_t m = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float t0 = fmaxf(fmax3(ex[c], ey[c], ez[c]), 0.0f);
    const float t1 = fminf(fmin3(gx[c], gy[c], gz[c]) * 1.0000004f, tmax);
    tn[c] = t0;
    if (t0 <= t1) m |= 1u << c;
  }
  return m;
}

// Sort key of a hit inner child: its entry distance (>= 0, so the float bits
// order like the distances) with the two low bits replaced by the child slot.
// The masked distance is at most the entry distance.
constexpr uint32_t kNoKey = 0xffffffffu;
__device__ __forceinline__ uint32_t child_key(float tn, int c) { return (__float_as_uint(tn) & ~3u) | (uint32_t)c; }
__device__ __forceinline__ float key_dist(uint32_t k) { return __uint_as_float(k & ~3u); }
__device__ __forceinline__ void key_swap(uint32_t& a, uint32_t& b) {
  uint32_t lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// One node step of the closest-hit walk over the BVH4.  Leaf children whose
// box is hit are tested in one loop after the box tests, so the lanes of a
// warp run their first, second, ... leaf test together; hit inner children
// that still start before the closest hit are visited near-first (the others
// pushed far-to-near), ordered by a sorting network over their keys so the
// step keeps no per-thread array.  Returns true when the walk is over.
__device__ __forceinline__ bool closest_step4(const SceneView& s, const RayPre& r, float tmax, int& node, int& sp,
                                              int* stack, float* stack_t, float& best_t, int& best, uint32_t* status,
                                              uint32_t& visits, uint32_t& ptests) {
  Node4Oct n = load_node4_oct(s.nodes, node, r.oct);
  ++visits;
  uint32_t k0 = kNoKey, k1 = kNoKey, k2 = kNoKey, k3 = kNoKey;
  int leaves = 0;
  float tn[4];
  const uint32_t hit = child_hits4(n, r, best_t, tn);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int ref = comp4i(n.ch, c);
    if (!(hit & (1u << c))) continue;  // empty slots hold boxes no ray hits
    if (ref < 0) {
      leaves |= 1 << c;
    } else {
      uint32_t k = child_key(tn[c], c);
      if (c == 0) k0 = k;
      else if (c == 1) k1 = k;
      else if (c == 2) k2 = k;
      else k3 = k;
    }
  }
  const float bt = best_t;
  while (leaves) {
    int c = __ffs(leaves) - 1;
    leaves &= leaves - 1;
    int p = ~comp4i(n.ch, c);
    ++ptests;
    float t = isect_prim(s, r, p);
    if (t > 0.0f && t < tmax && (t < best_t || (t == best_t && best >= 0 && p < best))) {
      best_t = t;
      best = p;
    }
  }
  // a child entered beyond a closer hit found here holds no closer hit (the
  // box tests already dropped the children entered beyond the earlier one)
  if (best_t < bt) {
    if (k0 != kNoKey && key_dist(k0) > best_t) k0 = kNoKey;
    if (k1 != kNoKey && key_dist(k1) > best_t) k1 = kNoKey;
    if (k2 != kNoKey && key_dist(k2) > best_t) k2 = kNoKey;
    if (k3 != kNoKey && key_dist(k3) > best_t) k3 = kNoKey;
  }
  key_swap(k0, k1);
  key_swap(k2, k3);
  key_swap(k0, k2);
  key_swap(k1, k3);
  key_swap(k1, k2);
  if (k0 == kNoKey) {
    while (sp > 0) {
      --sp;
      if (stack_t[sp] <= best_t) {
        node = stack[sp];
        return false;
      }
    }
    return true;
  }
  if (k3 != kNoKey) {
    if (sp < 64) {
      stack_t[sp] = key_dist(k3);
      stack[sp++] = comp4i(n.ch, k3 & 3);
    }
    else atomicOr(status, NEB_STATUS_STACK_OVERFLOW);
  }
  if (k2 != kNoKey) {
    if (sp < 64) {
      stack_t[sp] = key_dist(k2);
      stack[sp++] = comp4i(n.ch, k2 & 3);
    }
    else atomicOr(status, NEB_STATUS_STACK_OVERFLOW);
  }
  if (k1 != kNoKey) {
    if (sp < 64) {
      stack_t[sp] = key_dist(k1);
      stack[sp++] = comp4i(n.ch, k1 & 3);
    }
    else atomicOr(status, NEB_STATUS_STACK_OVERFLOW);
  }
  node = comp4i(n.ch, k0 & 3);
  return false;
}

// Closest hit with t in (deltaT, tmax); equal distances go to the lower
// primitive index.
__device__ __forceinline__ int trace_closest(const SceneView& s, const RayPre& r, float tmax, float& t_out,
                                             uint32_t* status, uint32_t& visits, uint32_t& ptests) {
  int best = -1;
  float best_t = tmax;
  if (s.nt + s.ns == 0 || !ray_finite(r.o, r.d)) { t_out = tmax; return -1; }
  int stack[64];
  float stack_t[64];
  int sp = 0, node = 0;
  while (!closest_step4(s, r, tmax, node, sp, stack, stack_t, best_t, best, status, visits, ptests)) {
  }
  t_out = best_t;
  return best;
}

// Hit point and its floating-point error bound: triangles are rebuilt from
// the watertight test's barycentrics (b0 v0 + b1 v1 + b2 v2, bound
// gamma_7 sum |b_i v_i|, PBRT 3rd ed. Sec. 3.9.3); spheres use o + t d with
// the bound gamma_5 |p|.
__device__ __forceinline__ void hit_point(const SceneView& s, const RayPre& r, int prim, float t, float3& p,
                                          float3& err, float3& n) {
  if (prim < s.nt) {
    float3 v0 = xyz(__ldg(s.tv0 + prim)), v1 = xyz(__ldg(s.tv1 + prim)), v2 = xyz(__ldg(s.tv2 + prim));
    float b[3];
    float tt = isect_tri(r, v0, v1, v2, b);
    n = normalize(cross(sub(v1, v0), sub(v2, v0)));
    if (tt > 0.0f) {
      p = add(add(mul(v0, b[0]), mul(v1, b[1])), mul(v2, b[2]));
      err = f3(NEB_GAMMA7 * (fabsf(v0.x * b[0]) + fabsf(v1.x * b[1]) + fabsf(v2.x * b[2])),
               NEB_GAMMA7 * (fabsf(v0.y * b[0]) + fabsf(v1.y * b[1]) + fabsf(v2.y * b[2])),
               NEB_GAMMA7 * (fabsf(v0.z * b[0]) + fabsf(v1.z * b[1]) + fabsf(v2.z * b[2])));
      return;
    }
    p = add(r.o, mul(r.d, t));
    err = f3(NEB_GAMMA5 * fabsf(p.x), NEB_GAMMA5 * fabsf(p.y), NEB_GAMMA5 * fabsf(p.z));
    return;
  }
  p = add(r.o, mul(r.d, t));
  err = f3(NEB_GAMMA5 * fabsf(p.x), NEB_GAMMA5 * fabsf(p.y), NEB_GAMMA5 * fabsf(p.z));
  n = normalize(sub(p, xyz(__ldg(s.sph + (prim - s.nt)))));
}

// new ray origin: hit point moved to the side of d by twice the projected
// error bound plus 1e-7
__device__ __forceinline__ float3 offset_origin(float3 p, float3 n, float3 err, float3 d) {
  float3 ns = dot(n, d) >= 0.0f ? n : neg(n);
  float e = 2.0f * (fabsf(n.x) * err.x + fabsf(n.y) * err.y + fabsf(n.z) * err.z) + 1e-7f;
  return add(p, mul(ns, e));
}

// ---------------------------------------------------------------------------
// warp-aggregated append (ballot + population count prefix)
// ---------------------------------------------------------------------------
// All 32 lanes of the warp must call it together.  Returns the slot of this
// lane in [base, base + popc(ballot)) or -1 when pred is false; slots past
// `cap` are dropped and raise NEB_STATUS_QUEUE_OVERFLOW.
__device__ __forceinline__ int warp_append(int* counter, bool pred, int cap, uint32_t* status) {
  unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (mask == 0) return -1;
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (!pred) return -1;
  int slot = base + __popc(mask & ((1u << lane) - 1u));
  if (slot >= cap) {
    atomicOr(status, NEB_STATUS_QUEUE_OVERFLOW);
    return -1;
  }
  return slot;
}

}  // namespace neb
