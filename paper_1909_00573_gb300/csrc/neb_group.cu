// neb_group.cu -- regrouping of ray queues before they are traced: camera
// rays after the first bounce, shadow rays and photon rays, by a counting
// sort over spatial groups (origin cell and direction or light-point cell).
#include <cfloat>

#include "neb_device.cuh"
#include "neb_internal.h"

namespace neb {

// ---- ray grouping ---------------------------------------------------------------
// Rays are traced faster when the 32 rays of a warp start close together and
// run in about the same direction: the lanes walk the same nodes and
// consecutive warps find them in cache.  Three queues are regrouped by a
// counting sort over kGroups spatial groups before they are traced:
//  - shadow rays, which leave in the order of their NEE vertices, so that a
//    warp's rays usually aim at different lights: grouped by the cell of the
//    origin and of the light point in the scene box (default 4 x 4 x 4 each);
//  - camera rays after the first bounce, which start in one area but go in
//    all directions: grouped by the cell of the origin and of the direction
//    in [-1, 1]^3 (default 2 x 2 x 2 and 8 x 8 x 8: on the city scene the
//    direction matters more than the origin);
//  - photon rays (64-byte records, as the camera rays) before each photon
//    walk, with the camera rays' cells.
// The cell resolutions are launch settings of the context (neb_tuning).
// The sort has three launches.  Count: each block builds a shared-memory
// histogram of its contiguous chunk of the queue and adds its non-zero
// groups to global counters (at most one atomic per block and group).  Scan:
// one block turns the counters into group offsets and re-zeroes them.
// Scatter: each block reads back the histogram its chunk got in the count
// launch (same chunks, same grid), reserves one range per non-zero group from
// the global cursors and ranks its rays inside the range with shared-memory
// atomics (reading the histogram back instead of counting the chunk again:
// grouping 2.27 -> 1.91 ms per iteration on the many-lights scene).  The order inside a group is that of the
// atomics; it changes no result.  The scatter moves the records, so the
// walks read their rays coalesced; shadow rays are written as 32-byte records
// and vertices without a shadow ray are dropped.
constexpr int kGroupBits = 12;
constexpr int kGroups = 1 << kGroupBits;
constexpr int kGroupBlocks = 152;
constexpr int kGroupThreads = 1024;
constexpr int kScanThreads = 1024;

// counters, cursors, then each count block's histogram (the scatter of the
// same queue splits it into the same block chunks and reads its histogram
// back instead of counting its chunk again)
size_t group_counter_ints() { return (2 + (size_t)kGroupBlocks) * (size_t)kGroups; }

struct CellGrid {
  float3 lo, unit;  // box minimum, 1 / extent per axis
};

// A grouping key: the scene box and the log2 cells per axis of its two parts
// (origin, then light point or direction); 3 (a + b) <= kGroupBits.
struct GroupSpec {
  CellGrid g;
  int a, b;
};

// Morton index of p's cell in a grid of 2^bits (bits <= 4) cells per axis over the box
__device__ __forceinline__ int grid_cell(const CellGrid& g, float3 p, int bits) {
  const int n = 1 << bits;
  int ix = min(max((int)((p.x - g.lo.x) * g.unit.x * (float)n), 0), n - 1);
  int iy = min(max((int)((p.y - g.lo.y) * g.unit.y * (float)n), 0), n - 1);
  int iz = min(max((int)((p.z - g.lo.z) * g.unit.z * (float)n), 0), n - 1);
  int m = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (b < bits)
      m |= (((ix >> b) & 1) << (3 * b)) | (((iy >> b) & 1) << (3 * b + 1)) | (((iz >> b) & 1) << (3 * b + 2));
  return m;
}

__device__ __forceinline__ int shadow_group(const GroupSpec& k, float3 p, float3 y) {
  return (grid_cell(k.g, p, k.a) << (3 * k.b)) + grid_cell(k.g, y, k.b);
}

__device__ __forceinline__ int camera_group(const GroupSpec& k, float3 o, float3 d) {
  const CellGrid dg = {f3(-1.0f, -1.0f, -1.0f), f3(0.5f, 0.5f, 0.5f)};
  return (grid_cell(k.g, o, k.a) << (3 * k.b)) + grid_cell(dg, d, k.b);
}

// Contiguous chunk [lo, hi) of a queue of n entries for this block.
__device__ __forceinline__ void block_chunk(int n, int& lo, int& hi) {
  const int chunk = (n + gridDim.x - 1) / gridDim.x;
  lo = min(n, blockIdx.x * chunk);
  hi = min(n, lo + chunk);
}

// h = shared histogram (kGroups ints).  Adds the block's non-zero groups to
// the global counters.
__device__ __forceinline__ void flush_counts(const int* h, int* counts) {
  for (int i = threadIdx.x; i < kGroups; i += blockDim.x)
    if (h[i]) atomicAdd(counts + i, h[i]);
}

// Turns the block's histogram h into its first output slot per group by
// reserving ranges from the global cursors.
__device__ __forceinline__ void reserve_ranges(int* h, int* cursors) {
  for (int i = threadIdx.x; i < kGroups; i += blockDim.x)
    if (h[i]) h[i] = atomicAdd(cursors + i, h[i]);
}

__device__ __forceinline__ void clear_hist(int* h) {
  for (int i = threadIdx.x; i < kGroups; i += blockDim.x) h[i] = 0;
}

// The block's histogram in the counter array (after the counters and cursors).
__device__ __forceinline__ int* block_hist(int* counters) { return counters + (2 + blockIdx.x) * kGroups; }
__device__ __forceinline__ void save_hist(const int* h, int* counters) {
  int* dst = block_hist(counters);
  for (int i = threadIdx.x; i < kGroups; i += blockDim.x) dst[i] = h[i];
}
__device__ __forceinline__ void load_hist(int* h, int* counters) {
  const int* src = block_hist(counters);
  for (int i = threadIdx.x; i < kGroups; i += blockDim.x) h[i] = src[i];
}

// One block: cursors = exclusive scan of counts, counts reset to zero;
// *total (if non-null) receives the sum.
__global__ void __launch_bounds__(kScanThreads) k_group_scan(int* __restrict__ counts, int* __restrict__ cursors,
                                                             int* total) {
  constexpr int kPer = kGroups / kScanThreads;
  __shared__ int warp_sums[kScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  int v[kPer];
  int sum = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    v[j] = counts[t * kPer + j];
    counts[t * kPer + j] = 0;
    sum += v[j];
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int x = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += x;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;  // exclusive warp offsets
    if (lane == 31 && total) *total = wi;
  }
  __syncthreads();
  int run = warp_sums[wid] + incl - sum;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    cursors[t * kPer + j] = run;
    run += v[j];
  }
}
static_assert(kGroups % kScanThreads == 0, "scan covers the groups evenly");

__device__ __forceinline__ bool nee_has_shadow(const NeeStore& nv, int i) {
  return (__float_as_int(nv.nrm[i].w) >> NV_FLAG_SHIFT) & NV_SHADOW;
}
__device__ __forceinline__ float3 nee_light_point(const NeeStore& nv, int i) {
  float3 p = xyz(nv.pos[i]);
  float4 ld = nv.ldir[i];
  float dist = nv.err[i].w;
  return f3(p.x + ld.x * dist, p.y + ld.y * dist, p.z + ld.z * dist);
}

__global__ void __launch_bounds__(kGroupThreads) k_shadow_count(NeeStore nv, const DevCounters* cnt, int cap,
                                                                GroupSpec g, int* __restrict__ counts) {
  __shared__ int h[kGroups];
  clear_hist(h);
  __syncthreads();
  int lo, hi;
  block_chunk(min(cnt->nee_count, cap), lo, hi);
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
    if (nee_has_shadow(nv, i)) atomicAdd(&h[shadow_group(g, xyz(nv.pos[i]), nee_light_point(nv, i))], 1);
  __syncthreads();
  flush_counts(h, counts);
  save_hist(h, counts);
}

// Each shadow ray also gets the subtree its walk starts in: the one
// kShadowLift levels above the node that holds its origin's primitive
// (precomputed per primitive when the tree is built).
__global__ void __launch_bounds__(kGroupThreads) k_shadow_scatter(NeeStore nv, const DevCounters* cnt, int cap,
                                                                  GroupSpec g, int* __restrict__ cursors,
                                                                  ShadowRay* __restrict__ rays,
                                                                  const int* __restrict__ prim_start,
                                                                  int* __restrict__ start) {
  __shared__ int h[kGroups];
  load_hist(h, cursors - kGroups);
  __syncthreads();
  int lo, hi;
  block_chunk(min(cnt->nee_count, cap), lo, hi);
  reserve_ranges(h, cursors);
  __syncthreads();
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    if (!nee_has_shadow(nv, i)) continue;
    int slot = atomicAdd(&h[shadow_group(g, xyz(nv.pos[i]), nee_light_point(nv, i))], 1);
    float4 pp = nv.pos[i], nn = nv.nrm[i], ee = nv.err[i], ld = nv.ldir[i];
    float3 ldir = xyz(ld);
    float3 o = offset_origin(xyz(pp), xyz(nn), xyz(ee), ldir);
    ShadowRay sr;
    sr.o = make_float4(o.x, o.y, o.z, ee.w * (1.0f - 1e-4f));
    sr.d = make_float4(ldir.x, ldir.y, ldir.z, __int_as_float(i));
    rays[slot] = sr;
    start[slot] = __ldg(prim_start + nv.prim[i]);
  }
}

__global__ void __launch_bounds__(kGroupThreads) k_cam_group_count(const CamRay* __restrict__ q,
                                                                   const int* __restrict__ count_ptr, int cap,
                                                                   GroupSpec g, int* __restrict__ counts) {
  __shared__ int h[kGroups];
  clear_hist(h);
  __syncthreads();
  int lo, hi;
  block_chunk(min(*count_ptr, cap), lo, hi);
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
    atomicAdd(&h[camera_group(g, xyz(__ldg(&q[i].o)), xyz(__ldg(&q[i].d)))], 1);
  __syncthreads();
  flush_counts(h, counts);
  save_hist(h, counts);
}

__global__ void __launch_bounds__(kGroupThreads) k_cam_group_scatter(const CamRay* __restrict__ q,
                                                                     const int* __restrict__ count_ptr, int cap,
                                                                     GroupSpec g, int* __restrict__ cursors,
                                                                     CamRay* __restrict__ out) {
  __shared__ int h[kGroups];
  load_hist(h, cursors - kGroups);
  __syncthreads();
  int lo, hi;
  block_chunk(min(*count_ptr, cap), lo, hi);
  reserve_ranges(h, cursors);
  __syncthreads();
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    CamRay r = q[i];
    out[atomicAdd(&h[camera_group(g, xyz(r.o), xyz(r.d))], 1)] = r;
  }
}

static CellGrid scene_grid(const neb_ctx* c) {
  CellGrid g;
  g.lo = f3(c->bmin[0], c->bmin[1], c->bmin[2]);
  float un[3];
  for (int a = 0; a < 3; ++a) {
    float ext = c->bmax[a] - c->bmin[a];
    un[a] = ext > 0.0f ? 1.0f / ext : 0.0f;
  }
  g.unit = f3(un[0], un[1], un[2]);
  return g;
}

static int group_blocks(int cap) { return capped_blocks(cap, kGroupThreads, kGroupBlocks); }

cudaError_t launch_group_camera(neb_ctx* c, const CamRay* q, const int* count_ptr, CamRay* out, cudaStream_t st) {
  GroupSpec g = {scene_grid(c), c->tune.cam_origin_bits, c->tune.cam_dir_bits};
  int* counts = c->group_counters;
  int* cursors = c->group_counters + kGroups;
  k_cam_group_count<<<group_blocks(c->cap_cam), kGroupThreads, 0, st>>>(q, count_ptr, c->cap_cam, g, counts);
  k_group_scan<<<1, kScanThreads, 0, st>>>(counts, cursors, nullptr);
  k_cam_group_scatter<<<group_blocks(c->cap_cam), kGroupThreads, 0, st>>>(q, count_ptr, c->cap_cam, g, cursors, out);
  return cudaGetLastError();
}

// Photon records share the camera records' layout in their first two float4
// (origin, direction), which is all the grouping reads; it moves whole
// 64-byte records.
static_assert(sizeof(PhotonRay) == sizeof(CamRay), "photon and camera records are both 64 bytes");
cudaError_t launch_group_photons(neb_ctx* c, const PhotonRay* q, const int* count_ptr, PhotonRay* out,
                                 cudaStream_t st) {
  GroupSpec g = {scene_grid(c), c->tune.cam_origin_bits, c->tune.cam_dir_bits};
  int* counts = c->ph_group_counters;
  int* cursors = c->ph_group_counters + kGroups;
  const CamRay* qc = reinterpret_cast<const CamRay*>(q);
  CamRay* oc = reinterpret_cast<CamRay*>(out);
  k_cam_group_count<<<group_blocks(c->cap_ph), kGroupThreads, 0, st>>>(qc, count_ptr, c->cap_ph, g, counts);
  k_group_scan<<<1, kScanThreads, 0, st>>>(counts, cursors, nullptr);
  k_cam_group_scatter<<<group_blocks(c->cap_ph), kGroupThreads, 0, st>>>(qc, count_ptr, c->cap_ph, g, cursors, oc);
  return cudaGetLastError();
}

cudaError_t launch_group_shadow(neb_ctx* c, const IterSlot& sl, cudaStream_t st) {
  GroupSpec g = {scene_grid(c), c->tune.shadow_origin_bits, c->tune.shadow_light_bits};
  int* counts = c->group_counters;
  int* cursors = c->group_counters + kGroups;
  k_shadow_count<<<group_blocks(c->cap_nee), kGroupThreads, 0, st>>>(sl.nv, sl.cnt, c->cap_nee, g, counts);
  k_group_scan<<<1, kScanThreads, 0, st>>>(counts, cursors, &sl.cnt->shadow_count);
  k_shadow_scatter<<<group_blocks(c->cap_nee), kGroupThreads, 0, st>>>(sl.nv, sl.cnt, c->cap_nee, g, cursors,
                                                             c->shadow_rays, c->prim_start, c->shadow_start);
  return cudaGetLastError();
}

}  // namespace neb
