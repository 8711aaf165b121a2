// neb_api.cu -- the C ABI of libneb.so: context lifetime, scene upload
// (materials, light list and alias table), iteration, readback, statistics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "neb_device.cuh"
#include "neb_internal.h"

using namespace neb;

namespace neb {
SceneView scene_view(const neb_ctx* c) {
  SceneView s;
  s.tv0 = c->tv0;
  s.tv1 = c->tv1;
  s.tv2 = c->tv2;
  s.sph = c->sph;
  s.sph_mat = c->sph_mat;
  s.mats = c->mats;
  s.nodes = c->nodes;
  s.prim_light = c->prim_light;
  s.light_prim = c->light_prim;
  s.light_psel = c->light_psel;
  s.light_inv_area = c->light_inv_area;
  s.alias_prob = c->alias_prob;
  s.alias_idx = c->alias_idx;
  s.nt = c->nt;
  s.ns = c->ns;
  s.nl = c->nl;
  return s;
}
}  // namespace neb

static int fail(neb_ctx* c, int code, const char* what, cudaError_t e = cudaSuccess) {
  if (c) {
    char buf[512];
    if (e != cudaSuccess)
      snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    else
      snprintf(buf, sizeof(buf), "%s", what);
    c->err = buf;
  }
  return code;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count);
}

static void free_scene(neb_ctx* c) {
  cudaFree(c->tv0); cudaFree(c->tv1); cudaFree(c->tv2); cudaFree(c->sph); cudaFree(c->mats); cudaFree(c->sph_mat);
  cudaFree(c->prim_light); cudaFree(c->light_prim); cudaFree(c->alias_idx); cudaFree(c->light_psel);
  cudaFree(c->light_inv_area); cudaFree(c->alias_prob); cudaFree(c->nee_lights); cudaFree(c->alias_slots);
  cudaFree(c->nodes);
  cudaFree(c->prim_start);
  cudaFree(c->oct_nodes);
  cudaFree(c->oct_state);
  c->tv0 = c->tv1 = c->tv2 = c->sph = c->mats = nullptr;
  c->sph_mat = c->prim_light = c->light_prim = c->alias_idx = nullptr;
  c->light_psel = c->light_inv_area = c->alias_prob = nullptr;
  c->nee_lights = nullptr;
  c->alias_slots = nullptr;
  c->nodes = nullptr;
  c->prim_start = nullptr;
  c->oct_nodes = nullptr;
  c->oct_state = nullptr;
  c->scene_ready = c->bvh_ready = false;
}

static bool config_ok(const neb_config* cfg) {
  return cfg->width >= 1 && cfg->height >= 1 && cfg->max_depth >= 1 && cfg->max_depth <= kMaxDepth &&
         cfg->merge_radius > 0.0f && cfg->octree_capacity >= 1 && cfg->split_factor >= 2 &&
         (cfg->octree_mode == 0 || cfg->octree_mode == 1) && (cfg->density_mode == 0 || cfg->density_mode == 1) &&
         !(cfg->strategy_mask & ~15u) && cfg->lp_photons >= 0 && cfg->lp_photons <= (1 << 26) &&
         (cfg->bvh_builder == 0 || cfg->bvh_builder == 1) &&
         (cfg->photon_records == 0 || cfg->photon_records == 1) &&
         (cfg->density_all == 0 || cfg->density_all == 1) &&
         cfg->merge_mode >= 0 && cfg->merge_mode <= 2 && cfg->merge_hits >= 0 &&
         (long long)cfg->width * cfg->height <= (1ll << 28);
}

static bool photon_grouping(const neb_config* cfg, size_t cap_ph) {
  return cfg->photon_records == 0 && cap_ph >= ((size_t)1 << 20);
}

// Queue capacities and hash-table size of a configuration (neb_create).
struct Capacities {
  size_t P, cap_cam, cap_nee, cap_rh, cap_ph, cap_mh;
  uint32_t table, ptable;
};
static Capacities capacities(const neb_config* cfg) {
  Capacities k;
  size_t D = (size_t)cfg->max_depth;
  k.P = (size_t)cfg->width * cfg->height;
  k.cap_cam = k.P;
  k.cap_nee = k.P * (D > 1 ? D - 1 : 1);
  k.cap_rh = k.P * D;
  k.cap_ph = k.cap_nee;
  // buckets of the view-vertex grid: one per NEE vertex, at most 2^22 (16 MB of
  // counts and 16 MB of starts stay in L2; more vertices share buckets)
  k.table = 1024;
  while (k.table < (uint32_t)k.cap_nee && k.table < (1u << 22)) k.table <<= 1;
  // staged photon hits of the per-cell merge (none when every hit merges on
  // its own); the photon table has a bucket per four staged hits
  const size_t mh = cfg->merge_hits > 0 ? (size_t)cfg->merge_hits : 2 * k.cap_ph;
  k.cap_mh = cfg->merge_mode != 1 ? (mh < ((size_t)1 << 30) ? mh : ((size_t)1 << 30)) : 0;
  k.ptable = 1024;
  while (k.ptable < k.table && (size_t)k.ptable * 4 < k.cap_mh) k.ptable <<= 1;
  return k;
}

extern "C" int neb_job_device_bytes(const neb_config* cfg, int n_tri, int n_sph, int n_mat, int n_lights,
                                    uint64_t* out) {
  if (!cfg || !out || !config_ok(cfg) || n_tri < 0 || n_sph < 0 || n_mat < 1 || n_lights < 0 ||
      n_lights > n_tri + n_sph || n_tri + n_sph < 1)
    return NEB_ERR_ARG;
  // the buffers of neb_create, neb_scene_upload and neb_build_bvh, in that order
  const Capacities k = capacities(cfg);
  const size_t D = (size_t)cfg->max_depth, nee_rows = k.P * (D > 1 ? D - 1 : 1);
  uint64_t b = 0;
  b += 3 * k.P * sizeof(CamRay) + 2 * sizeof(DevCounters);
  b += 2 * (7 * k.cap_nee * sizeof(float4) + 2 * k.cap_nee * sizeof(int) + k.cap_rh * sizeof(RHEvent) +
            (cfg->octree_mode == 1 ? nee_rows * sizeof(int) : 0));
  b += 2 * k.cap_ph * sizeof(PhotonRay) + k.cap_cam * sizeof(int2) + k.cap_ph * sizeof(int2);
  b += k.cap_nee * (sizeof(MergeRec) + sizeof(int)) + 2 * ((size_t)k.table + 1) * sizeof(int) +
       (size_t)k.table * sizeof(uint32_t);
  b += scan_scratch_ints((size_t)k.table + 1) * sizeof(int) + k.P * 3 * (2 * sizeof(double) + sizeof(float));
  b += cfg->keep_split ? k.P * 12 * sizeof(double) : 0;
  b += 2 * k.cap_nee * (sizeof(ShadowRay) + sizeof(int)) + group_counter_ints() * sizeof(int);
  b += photon_grouping(cfg, k.cap_ph) ? k.cap_ph * sizeof(PhotonRay) + group_counter_ints() * sizeof(int) : 0;
  b += k.cap_mh * (sizeof(MergeHit) + sizeof(int) + sizeof(int2)) +
       (k.cap_mh ? 2 * ((size_t)k.ptable + 1) * sizeof(int) : 0);
  const size_t nt = (size_t)n_tri, ns = (size_t)n_sph, nl = (size_t)n_lights, np = nt + ns;
  b += 3 * nt * sizeof(float4) + ns * (sizeof(float4) + sizeof(int)) + 3 * (size_t)n_mat * sizeof(float4);
  b += np * sizeof(int) + nl * (2 * sizeof(int) + 3 * sizeof(float) + sizeof(NeeLight) + sizeof(int2));
  b += (1 + (((size_t)cfg->octree_capacity + 7) & ~(size_t)7)) * sizeof(int) + sizeof(OctreeState);
  b += (np > 1 ? np - 1 : 1) * sizeof(BVH4Node) + np * sizeof(int);
  *out = b;
  return NEB_OK;
}

extern "C" int neb_create(const neb_config* cfg, void* cuda_stream, neb_ctx** out) {
  if (!cfg || !out) return NEB_ERR_ARG;
  *out = nullptr;
  if (!config_ok(cfg)) return NEB_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return NEB_ERR_NO_DEVICE;
  neb_ctx* c = new (std::nothrow) neb_ctx();
  if (!c) return NEB_ERR_OOM;
  c->cfg = *cfg;
  c->W = cfg->width;
  c->H = cfg->height;
  c->D = cfg->max_depth;
  c->P = c->W * c->H;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return NEB_ERR_CUDA;
    }
    c->own_stream = true;
  }
  size_t P = (size_t)c->P, D = (size_t)c->D;
  const Capacities k = capacities(cfg);
  c->cap_cam = (int)k.cap_cam;
  c->cap_nee = (int)k.cap_nee;
  c->cap_rh = (int)k.cap_rh;
  c->cap_ph = (int)k.cap_ph;
  c->cap_mh = (int)k.cap_mh;
  c->ptable_size = k.ptable;
  uint32_t t = k.table;
  c->table_size = t;
  c->scan_scratch.n = scan_scratch_ints((size_t)t + 1);
  bool ok = dalloc(&c->camq[0], P) == cudaSuccess && dalloc(&c->camq[1], P) == cudaSuccess &&
            dalloc(&c->camq_grouped, P) == cudaSuccess &&
            dalloc(&c->counters, 2) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k) {
    IterSlot& sl = c->slots[k];
    sl.cnt = c->counters + k;
    ok = dalloc(&sl.nv.pos, c->cap_nee) == cudaSuccess && dalloc(&sl.nv.nrm, c->cap_nee) == cudaSuccess &&
         dalloc(&sl.nv.wo, c->cap_nee) == cudaSuccess && dalloc(&sl.nv.tau, c->cap_nee) == cudaSuccess &&
         dalloc(&sl.nv.err, c->cap_nee) == cudaSuccess && dalloc(&sl.nv.ldir, c->cap_nee) == cudaSuccess &&
         dalloc(&sl.nv.dE, c->cap_nee) == cudaSuccess && dalloc(&sl.nv.lit, c->cap_nee) == cudaSuccess &&
         dalloc(&sl.nv.prim, c->cap_nee) == cudaSuccess &&
         dalloc(&sl.rh, c->cap_rh) == cudaSuccess &&
         (cfg->octree_mode != 1 || dalloc(&sl.slot_map, P * (D > 1 ? D - 1 : 1)) == cudaSuccess);
  }
  ok = ok && dalloc(&c->phq[0], c->cap_ph) == cudaSuccess && dalloc(&c->phq[1], c->cap_ph) == cudaSuccess &&
       dalloc(&c->hits, (size_t)c->cap_cam) == cudaSuccess && dalloc(&c->hits_ph, (size_t)c->cap_ph) == cudaSuccess &&
       dalloc(&c->mrec, c->cap_nee) == cudaSuccess && dalloc(&c->vert_bucket, c->cap_nee) == cudaSuccess &&
       dalloc(&c->bucket_count, (size_t)t + 1) == cudaSuccess &&
       dalloc(&c->bucket_start, (size_t)t + 1) == cudaSuccess && dalloc(&c->cell_bits, (size_t)t) == cudaSuccess &&
       dalloc(&c->scan_scratch.data, c->scan_scratch.n) == cudaSuccess && dalloc(&c->accum, P * 6) == cudaSuccess &&
       dalloc(&c->frame, P * 3) == cudaSuccess &&
       (!cfg->keep_split || dalloc(&c->split, P * 12) == cudaSuccess);
  ok = ok && dalloc(&c->shadow_rays, c->cap_nee) == cudaSuccess && dalloc(&c->shadow_start, c->cap_nee) == cudaSuccess &&
       dalloc(&c->shadow_rays_b, c->cap_nee) == cudaSuccess && dalloc(&c->shadow_start_b, c->cap_nee) == cudaSuccess &&
       dalloc(&c->group_counters, group_counter_ints()) == cudaSuccess;
  // photon rays are regrouped before each walk when the queue can be large
  // (for small jobs the three extra launches per bounce cost more than the
  // walk gains); FP32 records only
  if (ok && photon_grouping(cfg, (size_t)c->cap_ph))
    ok = dalloc(&c->phq_grouped, (size_t)c->cap_ph) == cudaSuccess &&
         dalloc(&c->ph_group_counters, group_counter_ints()) == cudaSuccess;
  if (ok && c->cap_mh > 0)
    ok = dalloc(&c->mh, (size_t)c->cap_mh) == cudaSuccess && dalloc(&c->mh_sorted, (size_t)c->cap_mh) == cudaSuccess &&
         dalloc(&c->mh_tile, (size_t)c->cap_mh) == cudaSuccess &&
         dalloc(&c->pb_count, (size_t)c->ptable_size + 1) == cudaSuccess &&
         dalloc(&c->pb_start, (size_t)c->ptable_size + 1) == cudaSuccess;
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  ok = ok && cudaStreamCreateWithPriority(&c->stream_hi, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
       cudaEventCreateWithFlags(&c->ev_caller, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&c->stream_b, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&c->stream_cap, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k)
    ok = cudaEventCreateWithFlags(&c->ev_pass1[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_pass23[k], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->ev_frame, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    neb_destroy(c);
    return NEB_ERR_OOM;
  }
  cudaMemsetAsync(c->bucket_count, 0, sizeof(int) * ((size_t)t + 1), c->stream);
  if (c->pb_count) cudaMemsetAsync(c->pb_count, 0, sizeof(int) * ((size_t)c->ptable_size + 1), c->stream);
  if (c->ph_group_counters) cudaMemsetAsync(c->ph_group_counters, 0, sizeof(int) * group_counter_ints(), c->stream);
  cudaMemsetAsync(c->accum, 0, sizeof(double) * P * 6, c->stream);
  cudaMemsetAsync(c->counters, 0, 2 * sizeof(DevCounters), c->stream);
  cudaMemsetAsync(c->group_counters, 0, sizeof(int) * group_counter_ints(), c->stream);
  if (c->split) cudaMemsetAsync(c->split, 0, sizeof(double) * P * 12, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    neb_destroy(c);
    return NEB_ERR_CUDA;
  }
  *out = c;
  return NEB_OK;
}

extern "C" void neb_destroy(neb_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_scene(c);
  cudaFree(c->camq[0]); cudaFree(c->camq[1]); cudaFree(c->camq_grouped);
  if (c->stream_b) cudaStreamSynchronize(c->stream_b);
  if (c->stream_hi) cudaStreamSynchronize(c->stream_hi);
  for (IterSlot& sl : c->slots) {
    cudaFree(sl.nv.pos); cudaFree(sl.nv.nrm); cudaFree(sl.nv.wo); cudaFree(sl.nv.tau); cudaFree(sl.nv.err);
    cudaFree(sl.nv.ldir); cudaFree(sl.nv.dE); cudaFree(sl.nv.lit); cudaFree(sl.nv.prim); cudaFree(sl.rh); cudaFree(sl.slot_map);
  }
  cudaFree(c->phq[0]); cudaFree(c->phq[1]); cudaFree(c->hits); cudaFree(c->hits_ph); cudaFree(c->mrec);
  cudaFree(c->vert_bucket); cudaFree(c->bucket_count); cudaFree(c->bucket_start); cudaFree(c->cell_bits); cudaFree(c->scan_scratch.data);
  cudaFree(c->accum); cudaFree(c->frame); cudaFree(c->split); cudaFree(c->counters);
  if (c->ev_frame) cudaEventDestroy(c->ev_frame);
  cudaFree(c->shadow_rays); cudaFree(c->shadow_start); cudaFree(c->shadow_rays_b); cudaFree(c->shadow_start_b);
  cudaFree(c->group_counters);
  cudaFree(c->phq_grouped); cudaFree(c->ph_group_counters);
  cudaFree(c->mh); cudaFree(c->mh_sorted); cudaFree(c->mh_tile); cudaFree(c->pb_count); cudaFree(c->pb_start);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  for (int k = 0; k < 2; ++k) {
    if (c->ev_pass1[k]) cudaEventDestroy(c->ev_pass1[k]);
    if (c->ev_pass23[k]) cudaEventDestroy(c->ev_pass23[k]);
  }
  for (int k = 0; k < 2; ++k) {
    if (c->graph_pass1[k]) cudaGraphExecDestroy(c->graph_pass1[k]);
    if (c->graph_pass23[k]) cudaGraphExecDestroy(c->graph_pass23[k]);
  }
  if (c->stream_b) cudaStreamDestroy(c->stream_b);
  if (c->stream_hi) cudaStreamDestroy(c->stream_hi);
  if (c->ev_caller) cudaEventDestroy(c->ev_caller);
  if (c->stream_cap) cudaStreamDestroy(c->stream_cap);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" const char* neb_last_error(const neb_ctx* c) { return c ? c->err.c_str() : "null context"; }

static float i2f(int i) {
  float f;
  memcpy(&f, &i, sizeof(f));
  return f;
}

static float3 hnorm(float3 a) {
  float l = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
  float inv = 1.0f / l;
  return make_float3(a.x * inv, a.y * inv, a.z * inv);
}
static float3 hcross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static float3 hsub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }

// Floats as ints that order like the floats (for atomicMin / atomicMax).
__host__ __device__ static inline int ordered_int(float f) {
  int i;
  memcpy(&i, &f, sizeof(i));
  return i >= 0 ? i : i ^ 0x7fffffff;
}
static float ordered_float(int i) {
  int j = i >= 0 ? i : i ^ 0x7fffffff;
  float f;
  memcpy(&f, &j, sizeof(f));
  return f;
}

namespace neb {
__global__ void k_bounds_init(int* b) {
  for (int k = 0; k < 3; ++k) {
    b[k] = 0x7fffffff;
    b[3 + k] = (int)0x80000000;
  }
}

// Caller triangles [nt][3][3] + materials -> the v0 / v1 / v2 float4 arrays
// (material index in v0.w), and the bounds of all vertices (ordered ints).
__global__ void k_pack_triangles(const float* __restrict__ tri, const uint32_t* __restrict__ mat, int nt,
                                 float4* v0, float4* v1, float4* v2, int* bounds) {
  float lo[3] = {3.402823466e+38f, 3.402823466e+38f, 3.402823466e+38f};
  float hi[3] = {-3.402823466e+38f, -3.402823466e+38f, -3.402823466e+38f};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
    const float* t = tri + 9 * (size_t)i;
    float v[9];
    for (int k = 0; k < 9; ++k) v[k] = t[k];
    v0[i] = make_float4(v[0], v[1], v[2], __int_as_float((int)mat[i]));
    v1[i] = make_float4(v[3], v[4], v[5], 0.0f);
    v2[i] = make_float4(v[6], v[7], v[8], 0.0f);
    for (int q = 0; q < 3; ++q)
      for (int k = 0; k < 3; ++k) {
        lo[k] = fminf(lo[k], v[3 * q + k]);
        hi[k] = fmaxf(hi[k], v[3 * q + k]);
      }
  }
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 3; ++k) {
      atomicMin(bounds + k, ordered_int(lo[k]));
      atomicMax(bounds + 3 + k, ordered_int(hi[k]));
    }
}

__global__ void k_mark_lights(const int* __restrict__ light_prim, int nl, int* prim_light) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x)
    prim_light[light_prim[i]] = i;
}

static void launch_pack_triangles(const float* tri, const uint32_t* mat, int nt, float4* v0, float4* v1, float4* v2,
                                  int* bounds, cudaStream_t st) {
  k_bounds_init<<<1, 1, 0, st>>>(bounds);
  int blocks = (nt + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_pack_triangles<<<blocks, 256, 0, st>>>(tri, mat, nt, v0, v1, v2, bounds);
}

// The NEE light records and alias slots: the same values the per-light
// arrays hold (the area pdf is the same FP32 product psel * (1 / area) the
// light pdf forms), gathered per light into one 64-byte line.
__global__ void k_nee_lights(const int* __restrict__ light_prim, const float* __restrict__ psel,
                             const float* __restrict__ inv_area, const float* __restrict__ alias_prob,
                             const int* __restrict__ alias_idx, const float4* __restrict__ tv0,
                             const float4* __restrict__ tv1, const float4* __restrict__ tv2,
                             const float4* __restrict__ sph, const int* __restrict__ sph_mat,
                             const float4* __restrict__ mats, int nt, int nl, NeeLight* out, int2* slots) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
    const int prim = light_prim[i];
    const float pa = psel[i] * inv_area[i];
    NeeLight L;
    int mat;
    if (prim < nt) {
      float4 a = tv0[prim], b = tv1[prim], cc = tv2[prim];
      mat = __float_as_int(a.w);
      L.a = make_float4(a.x, a.y, a.z, 0.0f);
      L.b = make_float4(b.x, b.y, b.z, pa);
      L.c = make_float4(cc.x, cc.y, cc.z, __int_as_float(prim));
    } else {
      mat = sph_mat[prim - nt];
      L.a = sph[prim - nt];
      L.b = make_float4(0.0f, 0.0f, 0.0f, pa);
      L.c = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(prim));
    }
    float4 e = mats[3 * mat + 1];
    L.e = make_float4(e.x, e.y, e.z, 0.0f);
    out[i] = L;
    slots[i] = make_int2(__float_as_int(alias_prob[i]), alias_idx[i]);
  }
}

static void launch_nee_lights(neb_ctx* c, cudaStream_t st) {
  int blocks = (c->nl + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_nee_lights<<<blocks, 256, 0, st>>>(c->light_prim, c->light_psel, c->light_inv_area, c->alias_prob, c->alias_idx,
                                       c->tv0, c->tv1, c->tv2, c->sph, c->sph_mat, c->mats, c->nt, c->nl,
                                       c->nee_lights, c->alias_slots);
}

static void launch_mark_lights(const int* light_prim, int nl, int* prim_light, cudaStream_t st) {
  int blocks = (nl + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_mark_lights<<<blocks, 256, 0, st>>>(light_prim, nl, prim_light);
}
}  // namespace neb

extern "C" int neb_scene_upload(neb_ctx* c, const float* tri, const uint32_t* tri_mat, int nt, const float* sph,
                                const uint32_t* sph_mat, int ns, const float* mats, int nm, const float* cam) {
  if (!c) return NEB_ERR_ARG;
  if (nt < 0 || ns < 0 || nm < 1 || !mats || !cam || (nt > 0 && (!tri || !tri_mat)) ||
      (ns > 0 && (!sph || !sph_mat)) || nt + ns < 1)
    return fail(c, NEB_ERR_ARG, "neb_scene_upload: bad arguments");
  // per-material mean emission; the material check and the light list take
  // one pass over the primitives' material indices
  std::vector<double> mat_le(nm);
  for (int m = 0; m < nm; ++m) {
    const float* e = mats + 12 * (size_t)m + 4;
    mat_le[m] = ((double)e[0] + (double)e[1] + (double)e[2]) / 3.0;
  }
  for (int i = 0; i < nt; ++i)
    if (tri_mat[i] >= (uint32_t)nm) return fail(c, NEB_ERR_ARG, "neb_scene_upload: triangle material out of range");
  for (int i = 0; i < ns; ++i)
    if (sph_mat[i] >= (uint32_t)nm) return fail(c, NEB_ERR_ARG, "neb_scene_upload: sphere material out of range");
  cudaStreamSynchronize(c->stream);
  free_scene(c);
  c->nt = nt;
  c->ns = ns;
  c->nm = nm;
  // ---- host-side repacking of the small arrays (triangles are repacked on the device)
  std::vector<float4> sp(ns), mt(3 * (size_t)nm);
  std::vector<int> smat(ns);
  for (int i = 0; i < ns; ++i) {
    sp[i] = make_float4(sph[4 * i], sph[4 * i + 1], sph[4 * i + 2], sph[4 * i + 3]);
    smat[i] = (int)sph_mat[i];
  }
  for (int m = 0; m < nm; ++m) {
    const float* r = mats + 12 * (size_t)m;
    mt[3 * m] = make_float4(i2f((int)r[0]), r[1], r[2], r[3]);
    mt[3 * m + 1] = make_float4(r[4], r[5], r[6], r[7]);
    mt[3 * m + 2] = make_float4(r[8], 0.0f, 0.0f, 0.0f);
  }
  // ---- light list: emissive triangles in index order, then emissive spheres
  int np = nt + ns;
  std::vector<int> light_prim;
  std::vector<double> power;
  std::vector<float> inv_area;
  const double PI = 3.14159265358979323846;
  for (int p = 0; p < np; ++p) {
    int m = p < nt ? (int)tri_mat[p] : (int)sph_mat[p - nt];
    double le = mat_le[m];
    if (le <= 0.0) continue;
    if (p < nt) {
      const float* t = tri + 9 * (size_t)p;
      float3 a = make_float3(t[0], t[1], t[2]), b = make_float3(t[3], t[4], t[5]), cc = make_float3(t[6], t[7], t[8]);
      float3 cr = hcross(hsub(b, a), hsub(cc, a));
      double area = 0.5 * sqrt((double)cr.x * cr.x + (double)cr.y * cr.y + (double)cr.z * cr.z);
      float fa = (float)area;
      power.push_back(PI * area * le);
      inv_area.push_back(1.0f / fa);
    } else {
      double R = sph[4 * (size_t)(p - nt) + 3];
      power.push_back(4.0 * PI * PI * R * R * le);
      inv_area.push_back((float)(1.0 / (2.0 * PI * R * R)));
    }
    light_prim.push_back(p);
  }
  int nl = (int)light_prim.size();
  c->nl = nl;
  // alias table, Vose (1991): worklists used as stacks filled in index order
  std::vector<float> psel(nl), aprob(nl);
  std::vector<int> aidx(nl);
  if (nl > 0) {
    double total = 0.0;
    for (int i = 0; i < nl; ++i) total += power[i];
    std::vector<double> pp(nl);
    std::vector<int> small, large;
    for (int i = 0; i < nl; ++i) {
      psel[i] = (float)(power[i] / total);
      pp[i] = power[i] * (double)nl / total;
      aidx[i] = i;
      if (pp[i] < 1.0) small.push_back(i); else large.push_back(i);
    }
    while (!small.empty() && !large.empty()) {
      int l = small.back(); small.pop_back();
      int g = large.back(); large.pop_back();
      aprob[l] = (float)pp[l];
      aidx[l] = g;
      pp[g] = (pp[g] + pp[l]) - 1.0;
      if (pp[g] < 1.0) small.push_back(g); else large.push_back(g);
    }
    while (!large.empty()) { aprob[large.back()] = 1.0f; large.pop_back(); }
    while (!small.empty()) { aprob[small.back()] = 1.0f; small.pop_back(); }
  }
  // scene bounds: spheres here, triangle vertices on the device (merged below)
  for (int k = 0; k < 3; ++k) { c->bmin[k] = 3.402823466e+38f; c->bmax[k] = -3.402823466e+38f; }
  for (int i = 0; i < ns; ++i)
    for (int k = 0; k < 3; ++k) {
      float ce = sph[4 * (size_t)i + k], r = sph[4 * (size_t)i + 3];
      if (ce - r < c->bmin[k]) c->bmin[k] = ce - r;
      if (ce + r > c->bmax[k]) c->bmax[k] = ce + r;
    }
  // camera basis (pinhole)
  {
    float3 eye = make_float3(cam[0], cam[1], cam[2]), target = make_float3(cam[3], cam[4], cam[5]),
           up = make_float3(cam[6], cam[7], cam[8]);
    c->cam.eye = eye;
    c->cam.fwd = hnorm(hsub(target, eye));
    c->cam.right = hnorm(hcross(c->cam.fwd, up));
    c->cam.up = hcross(c->cam.right, c->cam.fwd);
    c->cam.tanh_ = tanf(cam[9] * 3.14159265358979323846f / 360.0f);
    c->cam.aspect = (float)c->W / (float)c->H;
  }
  // ---- device copies
  cudaStream_t st = c->stream;
  bool ok = dalloc(&c->tv0, nt) == cudaSuccess && dalloc(&c->tv1, nt) == cudaSuccess &&
            dalloc(&c->tv2, nt) == cudaSuccess && dalloc(&c->sph, ns) == cudaSuccess &&
            dalloc(&c->sph_mat, ns) == cudaSuccess && dalloc(&c->mats, 3 * (size_t)nm) == cudaSuccess &&
            dalloc(&c->prim_light, np) == cudaSuccess && dalloc(&c->light_prim, nl) == cudaSuccess &&
            dalloc(&c->light_psel, nl) == cudaSuccess && dalloc(&c->light_inv_area, nl) == cudaSuccess &&
            dalloc(&c->alias_prob, nl) == cudaSuccess && dalloc(&c->alias_idx, nl) == cudaSuccess &&
            dalloc(&c->nee_lights, nl) == cudaSuccess && dalloc(&c->alias_slots, nl) == cudaSuccess;
  c->oct_cap = octree_params(c->bmin, c->bmax, c->cfg.octree_capacity, c->cfg.split_factor).capacity;
  ok = ok && dalloc(&c->oct_nodes, (size_t)c->oct_cap) == cudaSuccess && dalloc(&c->oct_state, 1) == cudaSuccess;
  // the caller's triangle arrays, copied as they are and repacked on the device
  float* d_tri = nullptr;
  uint32_t* d_tmat = nullptr;
  int* d_bounds = nullptr;
  ok = ok && cudaMallocAsync(&d_tri, sizeof(float) * 9 * (size_t)(nt > 0 ? nt : 1), st) == cudaSuccess &&
       cudaMallocAsync(&d_tmat, sizeof(uint32_t) * (size_t)(nt > 0 ? nt : 1), st) == cudaSuccess &&
       cudaMallocAsync(&d_bounds, sizeof(int) * 6, st) == cudaSuccess;
  if (!ok) {
    cudaFreeAsync(d_tri, st); cudaFreeAsync(d_tmat, st); cudaFreeAsync(d_bounds, st);
    cudaStreamSynchronize(st);
    cudaGetLastError();
    free_scene(c);
    return fail(c, NEB_ERR_OOM, "neb_scene_upload: device allocation failed");
  }
  int hb[6];
  if (nt) {
    cudaMemcpyAsync(d_tri, tri, sizeof(float) * 9 * (size_t)nt, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_tmat, tri_mat, sizeof(uint32_t) * (size_t)nt, cudaMemcpyHostToDevice, st);
    launch_pack_triangles(d_tri, d_tmat, nt, c->tv0, c->tv1, c->tv2, d_bounds, st);
    cudaMemcpyAsync(hb, d_bounds, sizeof(hb), cudaMemcpyDeviceToHost, st);
  }
  cudaMemsetAsync(c->prim_light, 0xff, sizeof(int) * (size_t)np, st);  // -1: not a light
  cudaFreeAsync(d_tri, st);
  cudaFreeAsync(d_tmat, st);
  cudaFreeAsync(d_bounds, st);
  if (ns) {
    cudaMemcpyAsync(c->sph, sp.data(), sizeof(float4) * ns, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->sph_mat, smat.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st);
  }
  cudaMemcpyAsync(c->mats, mt.data(), sizeof(float4) * 3 * nm, cudaMemcpyHostToDevice, st);
  if (nl) {
    cudaMemcpyAsync(c->light_prim, light_prim.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, st);
    launch_mark_lights(c->light_prim, nl, c->prim_light, st);
    cudaMemcpyAsync(c->light_psel, psel.data(), sizeof(float) * nl, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->light_inv_area, inv_area.data(), sizeof(float) * nl, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->alias_prob, aprob.data(), sizeof(float) * nl, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->alias_idx, aidx.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, st);
    launch_nee_lights(c, st);
  }
  OctreeState s0{1, 0, 0, 0};
  cudaMemsetAsync(c->oct_nodes, 0, sizeof(int) * (size_t)c->oct_cap, st);
  cudaMemcpyAsync(c->oct_state, &s0, sizeof(s0), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(c->accum, 0, sizeof(double) * 6 * (size_t)c->P, st);
  cudaMemsetAsync(c->counters, 0, 2 * sizeof(DevCounters), st);
  c->iteration = 0;
  c->launches = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_scene_upload", e);
  if (nt) {
    for (int k = 0; k < 3; ++k) {
      c->bmin[k] = fminf(c->bmin[k], ordered_float(hb[k]));
      c->bmax[k] = fmaxf(c->bmax[k], ordered_float(hb[3 + k]));
    }
  }
  c->oct = octree_params(c->bmin, c->bmax, c->cfg.octree_capacity, c->cfg.split_factor);
  c->scene_ready = true;
  return NEB_OK;
}

extern "C" int neb_build_bvh(neb_ctx* c) {
  if (!c) return NEB_ERR_ARG;
  if (!c->scene_ready) return fail(c, NEB_ERR_ARG, "neb_build_bvh: no scene uploaded");
  cudaError_t e = build_bvh(c);
  if (e != cudaSuccess) return fail(c, e == cudaErrorMemoryAllocation ? NEB_ERR_OOM : NEB_ERR_CUDA, "neb_build_bvh", e);
  c->bvh_ready = true;
  return NEB_OK;
}

extern "C" int neb_bvh_cost(neb_ctx* c, double* out) {
  if (!c || !out) return NEB_ERR_ARG;
  if (!c->bvh_ready) return fail(c, NEB_ERR_ARG, "neb_bvh_cost: no BVH");
  double s[3] = {0.0, 0.0, 0.0};
  cudaError_t e = bvh_area_sums(c, s);
  if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_bvh_cost", e);
  out[0] = s[2] > 0.0 ? 1.0 + s[0] / s[2] : 0.0;
  out[1] = s[2] > 0.0 ? s[1] / s[2] : 0.0;
  return NEB_OK;
}

// Passes 2-3 of an iteration overlap pass 1 of the next one (two streams, two
// buffer slots); stage timing keeps everything on one stream.
static int iterate_one(neb_ctx* c) {
  cudaError_t e = run_iteration(c, c->iteration + 1, !c->profiling);
  if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_iterate", e);
  c->iteration += 1;
  return NEB_OK;
}

// The caller's stream waits for the last iteration, so work enqueued on it
// afterwards sees every result.
static int join(neb_ctx* c) {
  if (c->profiling || c->iteration == 0) return NEB_OK;
  cudaError_t e = cudaStreamWaitEvent(c->stream, c->ev_pass23[c->iteration & 1], 0);
  return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_iterate", e);
}

extern "C" int neb_iterate(neb_ctx* c, int n_iterations) {
  if (!c || n_iterations < 0) return NEB_ERR_ARG;
  if (!c->bvh_ready) return fail(c, NEB_ERR_ARG, "neb_iterate: call neb_scene_upload and neb_build_bvh first");
  for (int i = 0; i < n_iterations; ++i) {
    int rc = iterate_one(c);
    if (rc != NEB_OK) return rc;
  }
  return n_iterations > 0 ? join(c) : NEB_OK;
}

extern "C" int neb_iterate_read(neb_ctx* c, int n_iterations, float* rgb_host) {
  if (!c || n_iterations < 0 || (n_iterations > 0 && !rgb_host)) return NEB_ERR_ARG;
  if (!c->bvh_ready) return fail(c, NEB_ERR_ARG, "neb_iterate_read: call neb_scene_upload and neb_build_bvh first");
  const size_t bytes = sizeof(float) * 3 * (size_t)c->P;
  for (int i = 0; i < n_iterations; ++i) {
    int rc = iterate_one(c);
    if (rc != NEB_OK) return rc;
    // the frame of this iteration follows its passes 2-3 on their stream, so
    // pass 1 of the next iteration is not held back by it
    cudaStream_t st2 = c->profiling ? c->stream : c->stream_b;
    cudaError_t e = launch_resolve(c->accum, c->P, c->iteration, c->frame, st2);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rgb_host, c->frame, bytes, cudaMemcpyDeviceToHost, st2);
    if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_iterate_read", e);
  }
  if (n_iterations > 0 && !c->profiling) {
    cudaError_t e = cudaEventRecord(c->ev_frame, c->stream_b);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_frame, 0);
    if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_iterate_read", e);
  }
  return NEB_OK;
}

extern "C" int neb_iterate_batch(neb_ctx* const* ctxs, int n, int n_iterations) {
  if (n < 0 || n_iterations < 0 || (n > 0 && !ctxs)) return NEB_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return NEB_ERR_ARG;
    if (!ctxs[i]->bvh_ready)
      return fail(ctxs[i], NEB_ERR_ARG, "neb_iterate_batch: every job needs its scene and BVH first");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] || ctxs[j]->stream == ctxs[i]->stream)
        return fail(ctxs[i], NEB_ERR_ARG, "neb_iterate_batch: jobs must be distinct contexts on distinct streams");
  }
  // Round-robin: iteration t of every job is enqueued before iteration t + 1
  // of any, so the jobs' kernels overlap on the GPU; each job's own order and
  // results are those of neb_iterate.
  for (int t = 0; t < n_iterations; ++t)
    for (int i = 0; i < n; ++i) {
      int rc = iterate_one(ctxs[i]);
      if (rc != NEB_OK) return rc;
    }
  for (int i = 0; i < n && n_iterations > 0; ++i) {
    int rc = join(ctxs[i]);
    if (rc != NEB_OK) return rc;
  }
  return NEB_OK;
}

static bool tuning_ok(const neb_tuning* t) {
  auto in = [](int v, int lo, int hi) { return v >= lo && v <= hi; };
  return in(t->cam_origin_bits, 0, 4) && in(t->cam_dir_bits, 0, 4) && in(t->shadow_origin_bits, 0, 4) &&
         in(t->shadow_light_bits, 0, 4) && 3 * (t->cam_origin_bits + t->cam_dir_bits) <= 12 &&
         3 * (t->shadow_origin_bits + t->shadow_light_bits) <= 12 && in(t->shade_blocks_per_sm, 1, 32) &&
         in(t->photon_grouping, 0, 1);
}

extern "C" int neb_get_tuning(const neb_ctx* c, neb_tuning* out) {
  if (!c || !out) return NEB_ERR_ARG;
  *out = c->tune;
  return NEB_OK;
}

extern "C" int neb_set_tuning(neb_ctx* c, const neb_tuning* t) {
  if (!c || !t || !tuning_ok(t)) return NEB_ERR_ARG;
  c->tune = *t;
  return NEB_OK;
}

// Milliseconds of n overlapped iterations with the current settings.
static int time_iterations(neb_ctx* c, int n, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_autotune");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, NEB_ERR_CUDA, "neb_autotune");
  }
  cudaEventRecord(e0, c->stream);
  int rc = neb_iterate(c, n);
  cudaEventRecord(e1, c->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (rc == NEB_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != NEB_OK) return rc;
  return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_autotune", e);
}

extern "C" int neb_autotune(neb_ctx* c, int iterations_per_candidate, neb_tuning* chosen) {
  if (!c || iterations_per_candidate < 1) return NEB_ERR_ARG;
  if (!c->bvh_ready) return fail(c, NEB_ERR_ARG, "neb_autotune: call neb_scene_upload and neb_build_bvh first");
  const int cams[][2] = {{1, 3}, {0, 3}, {1, 2}, {2, 2}, {0, 4}};
  const int shadows[][2] = {{2, 2}, {1, 2}, {2, 1}, {1, 1}};
  const int blocks[] = {8, 4, 16};
  neb_tuning best = c->tune;
  for (int axis = 0; axis < 3; ++axis) {
    const int n = axis == 0 ? 5 : (axis == 1 ? 4 : 3);
    float best_ms = 0.0f;
    neb_tuning pick = best;
    for (int i = 0; i < n; ++i) {
      neb_tuning t = best;
      if (axis == 0) { t.cam_origin_bits = cams[i][0]; t.cam_dir_bits = cams[i][1]; }
      if (axis == 1) { t.shadow_origin_bits = shadows[i][0]; t.shadow_light_bits = shadows[i][1]; }
      if (axis == 2) t.shade_blocks_per_sm = blocks[i];
      c->tune = t;
      float ms = 0.0f;
      int rc = time_iterations(c, iterations_per_candidate, &ms);
      if (rc != NEB_OK) {
        c->tune = best;
        return rc;
      }
      if (i == 0 || ms < best_ms) {
        best_ms = ms;
        pick = t;
      }
    }
    best = pick;
  }
  c->tune = best;
  if (chosen) *chosen = best;
  return NEB_OK;
}

extern "C" int neb_resolve(neb_ctx* c, float* rgb_out, int out_is_device) {
  if (!c || !rgb_out) return NEB_ERR_ARG;
  size_t n = (size_t)c->P * 3;
  if (out_is_device) {
    cudaError_t e = launch_resolve(c->accum, c->P, c->iteration, rgb_out, c->stream);
    return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_resolve", e);
  }
  float* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(float) * n, c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_OOM, "neb_resolve", e);
  launch_resolve(c->accum, c->P, c->iteration, d, c->stream);
  cudaMemcpyAsync(rgb_out, d, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d, c->stream);
  e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_resolve", e);
}

extern "C" int neb_synchronize(neb_ctx* c) {
  if (!c) return NEB_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_synchronize", e);
}

extern "C" int neb_error_estimate(neb_ctx* c, double* rel_rmse) {
  if (!c || !rel_rmse) return NEB_ERR_ARG;
  const int n = c->iteration, n_odd = (n + 1) / 2, n_even = n / 2;
  if (n_even < 1) return fail(c, NEB_ERR_ARG, "neb_error_estimate: needs at least two iterations");
  double* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, 2 * sizeof(double), c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_OOM, "neb_error_estimate", e);
  launch_error_sums(c->accum, c->P, n_even, n_odd, d, c->stream);
  double h[2] = {0.0, 0.0};
  cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d, c->stream);
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_error_estimate", e);
  const double var_of_mean = h[0] * (double)n_even * (double)n_odd / ((double)n * (double)n);
  *rel_rmse = h[1] > 0.0 ? sqrt(var_of_mean / h[1]) : 0.0;
  return NEB_OK;
}

extern "C" int neb_read_accum(neb_ctx* c, double* out) {
  if (!c || !out) return NEB_ERR_ARG;
  double* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(double) * 3 * (size_t)c->P, c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_OOM, "neb_read_accum", e);
  launch_sum_halves(c->accum, c->P, d, c->stream);
  cudaMemcpyAsync(out, d, sizeof(double) * 3 * (size_t)c->P, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d, c->stream);
  e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_read_accum", e);
}

extern "C" int neb_read_split(neb_ctx* c, double* out) {
  if (!c || !out) return NEB_ERR_ARG;
  if (!c->split) return fail(c, NEB_ERR_ARG, "neb_read_split: context created without keep_split");
  cudaMemcpyAsync(out, c->split, sizeof(double) * 12 * (size_t)c->P, cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_read_split", e);
}

extern "C" int neb_read_nee_rho(neb_ctx* c, float* out) {
  if (!c || !out) return NEB_ERR_ARG;
  if (c->D < 2) return fail(c, NEB_ERR_ARG, "neb_read_nee_rho: max_depth < 2 has no NEE vertices");
  size_t n = (size_t)c->P * (c->D - 1);
  float* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(float) * n, c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_OOM, "neb_read_nee_rho", e);
  launch_read_rho(c, d);
  cudaMemcpyAsync(out, d, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d, c->stream);
  e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_read_nee_rho", e);
}

extern "C" int neb_read_nee_vertices(neb_ctx* c, float* pos, float* nrm, int cap, int* count) {
  if (!c || !count || cap < 0 || (cap > 0 && (!pos || !nrm))) return NEB_ERR_ARG;
  const IterSlot& sl = c->slots[c->iteration & 1];  // slot of the last iteration
  DevCounters h;
  cudaMemcpyAsync(&h, sl.cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_read_nee_vertices", e);
  const int n = c->iteration > 0 ? (h.nee_count < c->cap_nee ? h.nee_count : c->cap_nee) : 0;
  *count = n;
  const int m = n < cap ? n : cap;
  if (m == 0) return NEB_OK;
  std::vector<float4> p(m), q(m);
  cudaMemcpyAsync(p.data(), sl.nv.pos, sizeof(float4) * (size_t)m, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(q.data(), sl.nv.nrm, sizeof(float4) * (size_t)m, cudaMemcpyDeviceToHost, c->stream);
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_read_nee_vertices", e);
  for (int i = 0; i < m; ++i) {
    pos[3 * i] = p[i].x; pos[3 * i + 1] = p[i].y; pos[3 * i + 2] = p[i].z;
    nrm[3 * i] = q[i].x; nrm[3 * i + 1] = q[i].y; nrm[3 * i + 2] = q[i].z;
  }
  return NEB_OK;
}

extern "C" int neb_get_stats(neb_ctx* c, neb_stats* out) {
  if (!c || !out) return NEB_ERR_ARG;
  DevCounters hs[2];
  OctreeState os{};
  cudaMemcpyAsync(hs, c->counters, sizeof(hs), cudaMemcpyDeviceToHost, c->stream);
  if (c->oct_state) cudaMemcpyAsync(&os, c->oct_state, sizeof(os), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_get_stats", e);
  // the two slots' counters together cover every iteration
  DevCounters h = hs[0];
  const DevCounters& h1 = hs[1];
  h.status |= h1.status;
  h.camera_rays += h1.camera_rays;
  h.nee_vertices += h1.nee_vertices;
  h.shadow_rays += h1.shadow_rays;
  h.photons += h1.photons;
  h.photon_hits += h1.photon_hits;
  h.merge_tests += h1.merge_tests;
  h.merges += h1.merges;
  h.random_hits += h1.random_hits;
  h.octree_inserts += h1.octree_inserts;
  h.octree_queries += h1.octree_queries;
  h.node_visits += h1.node_visits;
  h.prim_tests += h1.prim_tests;
  h.merge_hits_staged += h1.merge_hits_staged;
  for (int i = 0; i < 3; ++i) {
    h.visits_by[i] += h1.visits_by[i];
    h.ptests_by[i] += h1.ptests_by[i];
  }
  memset(out, 0, sizeof(*out));
  out->iterations = c->iteration;
  out->camera_rays = (int64_t)h.camera_rays;
  out->nee_vertices = (int64_t)h.nee_vertices;
  out->shadow_rays = (int64_t)h.shadow_rays;
  out->photons = (int64_t)h.photons;
  out->photon_hits = (int64_t)h.photon_hits;
  out->merge_tests = (int64_t)h.merge_tests;
  out->merges = (int64_t)h.merges;
  out->random_hits = (int64_t)h.random_hits;
  out->octree_inserts = (int64_t)h.octree_inserts;
  out->octree_queries = (int64_t)h.octree_queries;
  out->bvh_node_visits = (int64_t)h.node_visits;
  out->prim_tests = (int64_t)h.prim_tests;
  out->kernel_launches = c->launches;
  for (int i = 0; i < 3; ++i) {
    out->stage_node_visits[i] = (int64_t)h.visits_by[i];
    out->stage_prim_tests[i] = (int64_t)h.ptests_by[i];
  }
  out->octree_nodes = os.alloc < c->oct_cap ? os.alloc : c->oct_cap;
  out->octree_depth = os.depth;
  out->status = h.status | os.status;
  out->merge_hits_staged = (int64_t)h.merge_hits_staged;
  if (out->status & NEB_STATUS_SPIN_TIMEOUT) return fail(c, NEB_ERR_DEVICE_TIMEOUT, "octree insert spin timed out");
  if (out->status & (NEB_STATUS_QUEUE_OVERFLOW | NEB_STATUS_STACK_OVERFLOW))
    return fail(c, NEB_ERR_QUEUE_OVERFLOW, "device queue or traversal stack overflowed");
  return NEB_OK;
}

static const char* kStageNames[STAGE_COUNT] = {"rearm",      "camera",   "trace_camera", "extend",
                                               "shadow",     "octree_insert", "density", "nee_emit",
                                               "grid_build", "emission", "trace_photon", "photon",
                                               "group",      "merge"};

extern "C" int neb_set_profiling(neb_ctx* c, int enable) {
  if (!c) return NEB_ERR_ARG;
  if (enable && !c->ev[0]) {
    for (auto& ev : c->ev)
      if (cudaEventCreate(&ev) != cudaSuccess) return fail(c, NEB_ERR_CUDA, "neb_set_profiling");
  }
  c->profiling = enable != 0;
  for (int i = 0; i < STAGE_COUNT; ++i) {
    c->stage_ms[i] = 0.0;
    c->stage_launches[i] = 0;
  }
  return NEB_OK;
}

extern "C" int neb_get_stage_times(neb_ctx* c, double* ms, int64_t* launches, char* names, int max_stages) {
  if (!c) return NEB_ERR_ARG;
  int n = max_stages < STAGE_COUNT ? max_stages : STAGE_COUNT;
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = c->stage_ms[i];
    if (launches) launches[i] = c->stage_launches[i];
    if (names) {
      strncpy(names + 32 * i, kStageNames[i], 31);
      names[32 * i + 31] = 0;
    }
  }
  return STAGE_COUNT;
}

extern "C" int neb_trace_closest(neb_ctx* c, const float* rays, int n, int32_t* out_prim, float* out_t) {
  if (!c || n < 0 || (n > 0 && (!rays || !out_prim || !out_t))) return NEB_ERR_ARG;
  if (!c->bvh_ready) return fail(c, NEB_ERR_ARG, "neb_trace_closest: no BVH");
  if (n == 0) return NEB_OK;
  float* d = nullptr;
  size_t bytes = sizeof(float) * 6 * (size_t)n + sizeof(int) * (size_t)n + sizeof(float) * (size_t)n;
  cudaError_t e = cudaMallocAsync(&d, bytes, c->stream);
  if (e != cudaSuccess) return fail(c, NEB_ERR_OOM, "neb_trace_closest", e);
  int* dp = reinterpret_cast<int*>(d + 6 * (size_t)n);
  float* dt = reinterpret_cast<float*>(dp + n);
  cudaMemcpyAsync(d, rays, sizeof(float) * 6 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
  launch_trace_debug(scene_view(c), d, n, dp, dt, &c->counters->status, c->stream);
  cudaMemcpyAsync(out_prim, dp, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(out_t, dt, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d, c->stream);
  e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? NEB_OK : fail(c, NEB_ERR_CUDA, "neb_trace_closest", e);
}

extern "C" int neb_philox(const uint32_t* ctr, int n, const uint32_t key[2], uint32_t* out) {
  if (n < 0 || (n > 0 && (!ctr || !out || !key))) return NEB_ERR_ARG;
  if (n == 0) return NEB_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return NEB_ERR_NO_DEVICE;
  uint32_t* d = nullptr;
  if (cudaMalloc(&d, sizeof(uint32_t) * 8 * (size_t)n) != cudaSuccess) return NEB_ERR_OOM;
  cudaMemcpy(d, ctr, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyHostToDevice);
  launch_philox(d, n, make_uint2(key[0], key[1]), d + 4 * (size_t)n, 0);
  cudaError_t e = cudaMemcpy(out, d + 4 * (size_t)n, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? NEB_OK : NEB_ERR_CUDA;
}

extern "C" int neb_plane_box_area(const float* boxes, const float* pos, const float* nrm, int n, double* out) {
  if (n < 0 || (n > 0 && (!boxes || !pos || !nrm || !out))) return NEB_ERR_ARG;
  if (n == 0) return NEB_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return NEB_ERR_NO_DEVICE;
  float* d = nullptr;
  double* dout = nullptr;
  if (cudaMalloc(&d, sizeof(float) * 12 * (size_t)n) != cudaSuccess) return NEB_ERR_OOM;
  if (cudaMalloc(&dout, sizeof(double) * (size_t)n) != cudaSuccess) { cudaFree(d); return NEB_ERR_OOM; }
  cudaMemcpy(d, boxes, sizeof(float) * 6 * (size_t)n, cudaMemcpyHostToDevice);
  cudaMemcpy(d + 6 * (size_t)n, pos, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice);
  cudaMemcpy(d + 9 * (size_t)n, nrm, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice);
  launch_area(d, d + 6 * (size_t)n, d + 9 * (size_t)n, n, dout, 0);
  cudaError_t e = cudaMemcpy(out, dout, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  cudaFree(dout);
  return e == cudaSuccess ? NEB_OK : NEB_ERR_CUDA;
}

extern "C" int neb_count_neighbours(const float* pts, int n, const float* queries, int m, float r, int32_t* out) {
  if (n < 0 || m < 0 || !(r > 0.0f) || (n > 0 && !pts) || (m > 0 && (!queries || !out))) return NEB_ERR_ARG;
  if (m == 0) return NEB_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return NEB_ERR_NO_DEVICE;
  float *dp = nullptr, *dq = nullptr;
  int* dout = nullptr;
  if (cudaMalloc(&dp, sizeof(float) * 3 * (size_t)(n > 0 ? n : 1)) != cudaSuccess ||
      cudaMalloc(&dq, sizeof(float) * 3 * (size_t)m) != cudaSuccess ||
      cudaMalloc(&dout, sizeof(int) * (size_t)m) != cudaSuccess) {
    cudaFree(dp); cudaFree(dq); cudaFree(dout);
    return NEB_ERR_OOM;
  }
  if (n > 0) cudaMemcpy(dp, pts, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice);
  cudaMemcpy(dq, queries, sizeof(float) * 3 * (size_t)m, cudaMemcpyHostToDevice);
  cudaError_t e = count_neighbours_device(dp, n, dq, m, r, dout, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost);
  cudaFree(dp); cudaFree(dq); cudaFree(dout);
  return e == cudaSuccess ? NEB_OK : NEB_ERR_CUDA;
}
