// neb_trace.cu -- persistent BVH traversal kernels with dynamic ray fetch.
//
// Each warp keeps 32 rays in flight.  A lane that finishes its ray becomes
// idle; once enough lanes are idle (or none is busy) the warp fetches that
// many new rays with one atomic on a per-launch counter, so a few long rays
// no longer hold idle lanes until they finish (Aila and Laine, "Understanding
// the Efficiency of Ray Traversal on GPUs", HPG 2009: persistent threads with
// dynamic fetch).  Closest-hit warps check every kSteps node steps; any-hit
// warps vote after every step (measured: voting every step slows the
// closest-hit walk, 10.4 -> 11.0 ms per iteration on the many-lights scene,
// and speeds the any-hit walk, 6.0 -> 5.85 ms).  The traversal itself is the
// stack walk of trace_closest / trace_any cut into single node steps so lanes
// can be refilled between steps.
#include <cfloat>

#include "neb_device.cuh"
#include "neb_internal.h"

namespace neb {

constexpr int kTraceThreads = 256;
constexpr int kRefill = 8;        // refill when at least this many lanes are idle
constexpr int kSteps = 24;        // node steps between refill checks (closest hit)
constexpr int kShadowSteps = 64;  // node steps at most between refills (any hit; it votes every step)
constexpr int kShadowFlush = 28;  // any hit: lanes ready to test their queued leaves before the warp tests
constexpr int kIdle = -1, kDone = -2;

// Traversal state.  Both walks run over the 4-wide BVH.  Closest-hit walks
// test the leaf primitives of a node right after its box tests.  Shadow (any-hit) walks
// queue leaf primitives, and the warp tests its queued primitives together
// once kShadowFlush lanes have two queued or nothing left to walk, so the
// long triangle test runs with most lanes active ("while-while" with
// speculative traversal, Aila and Laine 2009).
struct Walk {
  int node;  // next inner node, -1 when the stack is exhausted
  int sp, best;
  float best_t;
  int npend;
  int pend[5];
  int start, skip;  // any hit: the subtree walked first, and the subtree the second walk leaves out (0: none)
};

__device__ __forceinline__ void walk_init(Walk& w) {
  w.node = 0;
  w.sp = 0;
  w.best = -1;
  w.best_t = FLT_MAX;
  w.npend = 0;
  w.start = 0;
  w.skip = 0;
}

// One inner-node step of the any-hit walk over the 4-wide tree: leaf children
// whose box is hit are queued (at most four, so a walk steps with at most one
// queued primitive), the first hit inner child is visited next and the others
// are pushed; the inner child w.skip (a subtree already walked) is left out.
// Leaf links are negative and the root, 0, is no node's child, so w.skip = 0
// leaves nothing out.
__device__ __forceinline__ void inner_step4(const SceneView& s, const RayPre& r, float tbound, Walk& w, int* stack,
                                           uint32_t* status, uint32_t& visits) {
  Node4Oct n = load_node4_oct(s.nodes, w.node, r.oct);
  ++visits;
  int next = -1;
  float tn[4];
  const uint32_t hit = child_hits4(n, r, tbound, tn);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int ref = comp4i(n.ch, c);
    if (ref == w.skip || !(hit & (1u << c))) continue;  // empty slots hold boxes no ray hits
    if (ref < 0) {
      w.pend[w.npend++] = ~ref;
    } else if (next < 0) {
      next = ref;
    } else if (w.sp < 64) {
      stack[w.sp++] = ref;
    } else {
      atomicOr(status, NEB_STATUS_STACK_OVERFLOW);
    }
  }
  w.node = next >= 0 ? next : (w.sp > 0 ? stack[--w.sp] : -1);
}

__device__ __forceinline__ void warp_total(unsigned long long* dst, uint32_t v) {
  uint32_t t = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && t) atomicAdd(dst, (unsigned long long)t);
}

// Warp-aggregated fetch of new rays for the idle lanes; all lanes call it.
// Returns the new ray index of an idle lane, kDone when the queue is empty.
__device__ __forceinline__ int fetch_rays(int cur, int* fetch, int count, int refill) {
  const unsigned FULL = 0xffffffffu;
  int lane = threadIdx.x & 31;
  bool idle = cur == kIdle;
  unsigned im = __ballot_sync(FULL, idle);
  unsigned bm = __ballot_sync(FULL, cur >= 0);
  if (im == 0 || (__popc(im) < refill && bm != 0)) return cur;
  int leader = __ffs(im) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(fetch, __popc(im));
  base = __shfl_sync(FULL, base, leader);
  if (!idle) return cur;
  int r = base + __popc(im & ((1u << lane) - 1u));
  return r < count ? r : kDone;
}

// Closest hit for a queue of 64-byte records (origin in float4 0, direction in
// float4 1: CamRay and PhotonRay).  hits[i] = (prim, t bits), prim -1 on a miss.
// packed: records are PackedPhoton (48 bytes, direction in the octahedral
// word) instead of 64-byte records with the direction in float4 1.
__global__ void __launch_bounds__(kTraceThreads, 4) k_trace_closest(SceneView s, const float4* __restrict__ recs,
                                                                 const int* __restrict__ count_ptr, int cap,
                                                                 int* __restrict__ fetch, int2* __restrict__ hits,
                                                                 DevCounters* cnt, int which, int packed) {
  const int count = min(*count_ptr, cap);
  int ray = kIdle;
  RayPre r;
  Walk w;
  int stack[64];
  float stack_t[64];
  uint32_t visits = 0, ptests = 0;
  while (true) {
    int nr = fetch_rays(ray, fetch, count, kRefill);
    if (ray == kIdle && nr >= 0) {
      const float4* rec = recs + (packed ? 3 : 4) * (size_t)nr;
      float4 o = __ldg(rec);
      float3 d = packed ? oct_decode16(__ldg(reinterpret_cast<const uint4*>(rec + 2)).x) : xyz(__ldg(rec + 1));
      r = make_ray(xyz(o), d);
      walk_init(w);
      if (s.nt + s.ns == 0 || !ray_finite(r.o, r.d)) {  // a miss without a walk
        hits[nr] = make_int2(-1, __float_as_int(FLT_MAX));
        nr = kIdle;
      }
    }
    ray = nr;
    if (__all_sync(0xffffffffu, ray == kDone)) break;
    for (int step = 0; step < kSteps && ray >= 0; ++step) {
      if (closest_step4(s, r, FLT_MAX, w.node, w.sp, stack, stack_t, w.best_t, w.best, &cnt->status, visits, ptests)) {
        hits[ray] = make_int2(w.best, __float_as_int(w.best_t));
        ray = kIdle;
      }
    }
  }
  warp_total(&cnt->node_visits, visits);
  warp_total(&cnt->prim_tests, ptests);
  warp_total(&cnt->visits_by[which], visits);
  warp_total(&cnt->ptests_by[which], ptests);
}

// Shadow rays (any hit with tmax = (1 - 1e-4) dist from the offset origin):
// the NEE vertices whose ray reaches the light are appended to the lit list,
// the only record of visibility that passes 2-3 read.  Most shadow rays are
// blocked, often by geometry next to their origin (the far side of the same
// building), so there are two walks.  Phase 0 walks each ray through the
// subtree a few levels above the node that holds its origin's primitive;
// rays with no blocker there (and a subtree short of the whole tree) are
// appended to a second queue.  Phase 1 walks those from the root, leaving
// that subtree out.  Every leaf is tested once at most and the answer is that
// of one walk from the root; splitting the walks keeps walks of similar
// length together in a warp.  Phase 2 is the single walk from the root, used
// for small trees, where the second launch would cost more than it saves.
__global__ void __launch_bounds__(kTraceThreads) k_trace_shadow(SceneView s, NeeStore nv,
                                                                const ShadowRay* __restrict__ srays,
                                                                const int* __restrict__ sstart,
                                                                const int* __restrict__ count_ptr, int cap,
                                                                int* __restrict__ fetch, DevCounters* cnt, int phase,
                                                                ShadowRay* __restrict__ rays_b,
                                                                int* __restrict__ start_b) {
  const int count = min(*count_ptr, cap);
  int ray = kIdle;  // NEE id of the lane's shadow ray
  RayPre r;
  Walk w;
  float tmax = 0.0f;
  int stack[64];
  uint32_t visits = 0, ptests = 0, rays = 0;
  const bool no_geometry = s.nt + s.ns == 0;
  while (true) {
    int nr = fetch_rays(ray, fetch, count, kRefill);
    bool lit0 = false;
    int lit0_id = 0;
    if (ray == kIdle && nr >= 0) {
      float4 so = __ldg(&srays[nr].o), sd = __ldg(&srays[nr].d);
      const int first = __ldg(sstart + nr);
      nr = __float_as_int(sd.w);
      r = make_ray(xyz(so), xyz(sd));
      tmax = so.w;
      walk_init(w);
      w.start = phase == 2 ? 0 : first;
      w.node = phase == 0 ? first : 0;
      w.skip = phase == 1 ? first : 0;
      if (phase != 1) ++rays;
      if (no_geometry || !ray_finite(r.o, r.d)) {  // nothing can block it
        lit0 = true;
        lit0_id = nr;
        nr = kIdle;
      }
    }
    if (__any_sync(0xffffffffu, lit0)) {
      int slot = warp_append(&cnt->lit_count, lit0, cap, &cnt->status);
      if (slot >= 0) nv.lit[slot] = lit0_id;
    }
    ray = nr;
    if (__all_sync(0xffffffffu, ray == kDone)) break;
    for (int step = 0; step < kShadowSteps; ++step) {
      if (ray >= 0 && w.node >= 0 && w.npend <= 1) inner_step4(s, r, tmax, w, stack, &cnt->status, visits);
      bool ready = ray < 0 || w.npend >= 2 || w.node < 0;
      // the queued leaves are tested once 28 lanes are ready (the others test
      // what they have queued and walk on): waiting for all 32 leaves most
      // lanes idle behind the last few (many lights: 5.82 -> 5.58 ms)
      if (__popc(__ballot_sync(0xffffffffu, ready)) >= kShadowFlush) {
        bool lit = false, defer = false;
        int id = 0;
        if (ray >= 0) {
          bool hit = false;
          for (int q = 0; q < w.npend; ++q) {
            ++ptests;
            float t = isect_prim(s, r, w.pend[q]);
            hit |= t > 0.0f && t < tmax;
          }
          w.npend = 0;
          if (!hit && w.node < 0) {
            id = ray;
            if (phase == 0 && w.start > 0) defer = true;  // the rest of the tree is still to walk
            else lit = true;
          }
          if (hit || w.node < 0) ray = kIdle;
        }
        int slot = warp_append(&cnt->lit_count, lit, cap, &cnt->status);
        if (slot >= 0) nv.lit[slot] = id;
        if (phase == 0) {
          int b = warp_append(&cnt->shadow_count_b, defer, cap, &cnt->status);
          if (b >= 0) {
            ShadowRay sr;
            sr.o = make_float4(r.o.x, r.o.y, r.o.z, tmax);
            sr.d = make_float4(r.d.x, r.d.y, r.d.z, __int_as_float(id));
            rays_b[b] = sr;
            start_b[b] = w.start;
          }
        }
        if (__all_sync(0xffffffffu, ray < 0)) break;
      }
      // leave for a refill once enough lanes can take a new ray
      if (__popc(__ballot_sync(0xffffffffu, ray == kIdle)) >= kRefill) break;
    }
  }
  warp_total(&cnt->shadow_rays, rays);
  warp_total(&cnt->node_visits, visits);
  warp_total(&cnt->prim_tests, ptests);
  warp_total(&cnt->visits_by[1], visits);
  warp_total(&cnt->ptests_by[1], ptests);
}

// Persistent grid: the SM count times the resident blocks per SM of `kernel`.
template <typename K>
static int trace_blocks(K kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kTraceThreads, 0);
  return (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 4);
}

cudaError_t launch_trace_closest(neb_ctx* c, const float4* recs, const int* count_ptr, int cap, int2* hits,
                                 int which, DevCounters* cnt, cudaStream_t st, int packed) {
  static const int closest_blocks = trace_blocks(k_trace_closest);
  int* fetch = &cnt->fetch[which];
  cudaMemsetAsync(fetch, 0, sizeof(int), st);
  k_trace_closest<<<capped_blocks(cap, kTraceThreads, closest_blocks), kTraceThreads, 0, st>>>(scene_view(c), recs, count_ptr, cap, fetch, hits, cnt,
                                                            which, packed);
  return cudaGetLastError();
}

// Trees of fewer nodes are walked from the root in one launch.
constexpr int kLocalFirstMinNodes = 8192;

int shadow_walk_launches(const neb_ctx* c) { return c->n_nodes4 >= kLocalFirstMinNodes ? 2 : 1; }

cudaError_t launch_trace_shadow(neb_ctx* c, const IterSlot& sl, cudaStream_t st) {
  static const int shadow_blocks = trace_blocks(k_trace_shadow);
  const int blocks = capped_blocks(c->cap_nee, kTraceThreads, shadow_blocks);
  int* fetch = &sl.cnt->fetch[1];   // phase 0 (or the single walk)
  int* fetch_b = &sl.cnt->fetch[3];  // phase 1
  cudaMemsetAsync(fetch, 0, sizeof(int), st);
  if (shadow_walk_launches(c) == 1) {
    k_trace_shadow<<<blocks, kTraceThreads, 0, st>>>(scene_view(c), sl.nv, c->shadow_rays, c->shadow_start,
                                                     &sl.cnt->shadow_count, c->cap_nee, fetch, sl.cnt, 2, nullptr,
                                                     nullptr);
    return cudaGetLastError();
  }
  cudaMemsetAsync(fetch_b, 0, sizeof(int), st);
  k_trace_shadow<<<blocks, kTraceThreads, 0, st>>>(scene_view(c), sl.nv, c->shadow_rays, c->shadow_start,
                                                   &sl.cnt->shadow_count, c->cap_nee, fetch, sl.cnt, 0,
                                                   c->shadow_rays_b, c->shadow_start_b);
  k_trace_shadow<<<blocks, kTraceThreads, 0, st>>>(scene_view(c), sl.nv, c->shadow_rays_b, c->shadow_start_b,
                                                   &sl.cnt->shadow_count_b, c->cap_nee, fetch_b, sl.cnt, 1,
                                                   nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace neb
