// neb_internal.h -- host-side context and the launchers shared between the
// translation units of libneb.so.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "neb_device.cuh"
#include "neb_types.h"

namespace neb {

// ---- wavefront records -------------------------------------------------------

// Camera ray in flight from x_{k-1} to x_k (64 bytes).
struct __align__(16) CamRay {
  float4 o;    // origin xyz, w: pixel (int bits)
  float4 d;    // direction xyz, w: pdf_fwd = solid-angle pdf of d at x_{k-1} (1: camera or delta)
  float4 tau;  // throughput up to x_k (rgb), w: cos_prev = |n_{k-1} . d|
  float4 mis;  // x: C'_k = C_{k-1} + [x_{k-1} non-delta], y: C_{k-1},
               // z: NEE id of x_{k-1} (int bits, -1 none), w: flags (int bits)
};
enum { RAY_FROM_CAMERA = 1, RAY_PREV_DELTA = 2 };

// Random hit of an emitter at x_l = y, finished in pass 3 (48 bytes).
struct __align__(16) RHEvent {
  float4 L;     // rgb tau * Le, w: F_l = pdf_fwd |cos_y| / t^2 (0 when l == 1)
  float4 y;     // hit point, w: light index (int bits)
  int4 info;    // x pixel, y NEE id of x_{l-1} (-1 when l == 1), z flags, w C_{l-1} (float bits)
};

// Photon ray leaving a photon vertex (64 bytes).
struct __align__(16) PhotonRay {
  float4 o;    // origin, w: pixel of the path that owns the NEE vertex (int bits)
  float4 d;    // direction, w: pdf_dir (solid angle, 1 for delta)
  float4 phi;  // flux rgb, w: cos_orig = |n_origin . d|
  float4 mis;  // x E0, y pA, z pB, w: k_nee | (j << 8), j = index of the next hit
};

// Packed photon ray (48 bytes): origin and MIS factors in FP32; the RGB flux
// as three FP16 mantissas of a shared power-of-two scale; the direction as
// two 16-bit octahedral coordinates (Meyer et al. 2010).
struct __align__(16) PackedPhoton {
  float4 o;    // origin, w: pixel (int bits)
  float4 mis;  // E0, pA, pB, pdf_dir
  uint4 q;     // x: direction (u16 x, u16 y); y: flux r, g (FP16); z: flux b, cos_orig (FP16);
               // w: k_nee | j << 8 | (flux exponent + 128) << 16
};

// One light of the NEE light choice (64 bytes): what a light sample at a
// camera vertex reads once the alias slot has picked the light, so that the
// choice costs two dependent loads (slot, then this line) instead of five.
struct __align__(16) NeeLight {
  float4 a;  // triangle: v0; sphere: centre, w radius
  float4 b;  // triangle: v1; w: area pdf of the choice, psel / area (sphere: psel / (2 pi R^2))
  float4 c;  // triangle: v2; w: primitive index (int bits)
  float4 e;  // emission rgb of the light's material
};

// Shadow ray of an NEE vertex in light-grouped order (32 bytes).
struct __align__(16) ShadowRay {
  float4 o;  // offset origin, w: tmax = (1 - 1e-4) distance to the light point
  float4 d;  // direction to the light point, w: NEE id (int bits)
};

// Grid-ordered entry of a mergeable view vertex (16 bytes): its position and
// its NEE id; the merge reads the rest of the vertex from the NEE store for
// the few candidates within the radius.
struct __align__(16) MergeRec {
  float4 pos;  // xyz, w: NEE id (int bits)
};

// Photon hit staged for the per-cell merge (48 bytes): everything the merge
// of this hit with a view vertex x_k reads, with the hit's 1 / w written as
// c0 (1 + c1' pdfF + c2' pdfC Cfac) and c0 folded into the flux (c0 = 1 for
// NEB photons, so their terms are the ones the per-hit merge computes).
struct __align__(16) MergeHit {
  float4 key;  // hit point xyz, w: kmax | (channel - 2) << 8 (int bits)
  float4 dir;  // -photon direction (towards where it came from), w: c1'
  float4 phi;  // flux / c0 (rgb), w: c2'
};

// NEE vertex store, structure of arrays (one float4 per field).
struct NeeStore {
  float4* pos;   // xyz, w: Cfac_k = C'_k cos_prev / (pdf_fwd |cos_k|)
  float4* nrm;   // geometric normal (unflipped), w: mat | k << 20 | flags << 26 (int bits)
  float4* wo;    // xyz, w: pixel (int bits)
  float4* tau;   // rgb, w: g_y = cos_y / (dist^2 p_l)
  float4* err;   // hit point error bound, w: ldist
  float4* ldir;  // direction to the light point, w: rho after the density pass (-2 where not evaluated)
  float4* dE;    // unoccluded irradiance rgb (zero if back-facing; read only for vertices of the lit list),
                 // w: the light point's light-photon pdf
  int* lit;      // ids of the vertices whose shadow ray reached the light (DevCounters::lit_count of them)
  int* prim;     // primitive the vertex lies on
};
enum { NV_DELTA = 1, NV_MERGEABLE = 2, NV_SHADOW = 4 };
enum { NV_MAT_MASK = (1 << 20) - 1, NV_K_SHIFT = 20, NV_FLAG_SHIFT = 26 };

// Per-iteration queue sizes and accumulated counters (device memory).
struct DevCounters {
  int cam_count[2];
  int nee_count;
  int shadow_count;  // NEE vertices with a shadow ray (length of the light-grouped order)
  int rh_count;
  int ph_count[2];
  int merge_count;
  int lit_count;
  int shadow_count_b;  // shadow rays left for the second walk (no blocker near the origin)
  uint32_t status;
  unsigned long long camera_rays, nee_vertices, shadow_rays, photons, photon_hits;
  unsigned long long merge_tests, merges, random_hits, octree_inserts, octree_queries;
  unsigned long long node_visits, prim_tests;
  unsigned long long visits_by[3], ptests_by[3];  // camera, shadow, photon traversal
  int fetch[4];                                   // dynamic-fetch counters of the traversal kernels
  int mh_count;                                   // photon hits staged for the per-cell merge
  int mh_tiles;                                   // full tiles of staged hits (of one bucket)
  int mh_small;                                   // partial tiles (the rest of a bucket)
  int mh_next, mh_next_small;                     // dynamic fetch of the tiles
  int oct_deferred;                               // octree inserts deferred past an exhausted pool
  unsigned long long merge_hits_staged;           // hits merged through the per-cell merge
};

// Buffers that pass 1 of an iteration fills and passes 2 and 3 read.  There
// are two sets, used by odd and even iterations, so pass 1 of iteration i + 1
// can run on one stream while passes 2 and 3 of iteration i finish on another.
struct IterSlot {
  NeeStore nv{};
  RHEvent* rh = nullptr;
  int* slot_map = nullptr;   // deterministic octree mode: NEE id per (pixel, k)
  DevCounters* cnt = nullptr;
};

struct CameraParams {
  float3 eye, fwd, right, up;
  float tanh_, aspect;
};

struct IterParams {
  int W, H, D;
  int iteration;
  uint2 key;
  float r, r2, kernel;  // merge radius, r^2, 1/(pi r^2)
  uint32_t mask;
  int n_lp;             // conventional light photons this iteration (0 unless mask bit 3)
  int keep_split;
  int cap_cam, cap_nee, cap_rh, cap_ph;
  float3 gmin;          // hashed grid origin
  float cell_inv;       // 1 / (2 r)
  uint32_t table_mask;  // hash table size - 1
  const uint32_t* cell_bits;  // occupancy bits of the grid's cells
  uint32_t cell_bits_mask;    // number of bits - 1
  int cap_mh;           // staged photon hits per iteration (0: every hit merges on its own)
  int stage_min;        // a hit is staged when more view vertices than this lie in its cells
};

enum { STAGE_REARM = 0, STAGE_CAMERA, STAGE_TRACE_CAM, STAGE_EXTEND, STAGE_SHADOW, STAGE_INSERT, STAGE_DENSITY,
       STAGE_NEE, STAGE_GRID, STAGE_EMISSION, STAGE_TRACE_PHOTON, STAGE_PHOTON, STAGE_GROUP, STAGE_MERGE,
       STAGE_COUNT };
// timed stage intervals per iteration: 5 D + 5 for max depth D (up to D = 64)
constexpr int kMaxStageRecords = 5 * kMaxDepth + 8;

struct Scratch {
  int* data = nullptr;
  size_t n = 0;
};

}  // namespace neb

struct neb_ctx {
  neb_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int W = 0, H = 0, D = 0, P = 0;

  // scene
  int nt = 0, ns = 0, nm = 0, nl = 0;
  float bmin[3]{}, bmax[3]{};
  float4 *tv0 = nullptr, *tv1 = nullptr, *tv2 = nullptr, *sph = nullptr, *mats = nullptr;
  int* sph_mat = nullptr;
  int *prim_light = nullptr, *light_prim = nullptr, *alias_idx = nullptr;
  float *light_psel = nullptr, *light_inv_area = nullptr, *alias_prob = nullptr;
  neb::NeeLight* nee_lights = nullptr;  // per light, in light-list order
  int2* alias_slots = nullptr;          // per alias slot: (probability bits, alias)
  neb::CameraParams cam{};
  bool scene_ready = false;

  // BVH (4-wide)
  neb::BVH4Node* nodes = nullptr;
  int* prim_start = nullptr;   // per primitive: the node kShadowLift levels above its leaf's node
  int n_nodes4 = 0;
  bool bvh_ready = false;

  // density octree
  int* oct_nodes = nullptr;
  neb::OctreeState* oct_state = nullptr;
  neb::OctreeParams oct{};
  int oct_cap = 0;

  // per-iteration buffers
  neb::CamRay* camq[2] = {nullptr, nullptr};
  neb::CamRay* camq_grouped = nullptr;  // bounce rays regrouped before tracing
  neb::PhotonRay* phq_grouped = nullptr;  // photon rays regrouped before tracing (FP32 records only)
  int* ph_group_counters = nullptr;       // their grouping counters (passes 2-3 run beside pass 1's grouping)
  neb::IterSlot slots[2];
  neb::PhotonRay* phq[2] = {nullptr, nullptr};
  int2* hits = nullptr;     // closest hits of the camera ray queue (pass 1)
  int2* hits_ph = nullptr;  // closest hits of the photon ray queue (pass 3)
  neb::ShadowRay* shadow_rays = nullptr;  // shadow rays grouped by light
  int* shadow_start = nullptr;            // per shadow ray: the subtree walked first (near its origin)
  neb::ShadowRay* shadow_rays_b = nullptr;  // rays the first walk did not settle, for the second
  int* shadow_start_b = nullptr;
  int* group_counters = nullptr;  // ray grouping of pass 1: group counts, then cursors
  neb_tuning tune{1, 3, 2, 2, 8, 1};  // launch settings (neb_set_tuning / neb_autotune)
  neb::MergeRec* mrec = nullptr;
  int* vert_bucket = nullptr;
  int* bucket_count = nullptr;
  int* bucket_start = nullptr;
  uint32_t* cell_bits = nullptr;  // occupancy bits of the grid's cells, 32 per bucket
  int cap_cam = 0, cap_nee = 0, cap_rh = 0, cap_ph = 0;
  uint32_t table_size = 0;
  // per-cell merge: staged photon hits, their order by bucket of the photon
  // table, the tiles, and the photon table's counts and starts
  neb::MergeHit* mh = nullptr;
  int* mh_sorted = nullptr;
  int2* mh_tile = nullptr;
  int* pb_count = nullptr;
  int* pb_start = nullptr;
  int cap_mh = 0;
  uint32_t ptable_size = 0;
  neb::Scratch scan_scratch;
  double* accum = nullptr;  // FP64 sums: [2][P][3], even iterations then odd iterations
  float* frame = nullptr;             // resolved image staged for neb_iterate_read
  cudaEvent_t ev_frame = nullptr;     // after the last frame copy of neb_iterate_read
  double* split = nullptr;
  neb::DevCounters* counters = nullptr;  // two sets, one per slot
  // passes 2-3 run on stream_b, overlapped with the next iteration's pass 1
  // on `stream`; ev_pass1[s] / ev_pass23[s] mark the end of each half for slot s
  cudaStream_t stream_b = nullptr;
  cudaStream_t stream_hi = nullptr;   // pass 1 of the overlapped schedule, at the device's highest priority
  cudaEvent_t ev_caller = nullptr;    // work the caller enqueued before an iteration
  cudaEvent_t ev_pass1[2] = {nullptr, nullptr}, ev_pass23[2] = {nullptr, nullptr};
  // overlapped iterations launch each half as a CUDA graph, recorded on
  // stream_cap every iteration and applied to the slot's executable graph
  bool use_graphs = true;
  cudaStream_t stream_cap = nullptr;
  cudaGraphExec_t graph_pass1[2] = {nullptr, nullptr}, graph_pass23[2] = {nullptr, nullptr};
  int iteration = 0;  // iterations completed (enqueued)
  long long launches = 0;  // kernels enqueued by neb_iterate

  // profiling
  bool profiling = false;
  cudaEvent_t ev[2 * neb::kMaxStageRecords] = {};
  double stage_ms[neb::STAGE_COUNT] = {};
  long long stage_launches[neb::STAGE_COUNT] = {};
};

namespace neb {

// Grid of a grid-stride kernel over at most `cap` items: enough blocks to give
// every item a thread, never more than max_blocks (small images launch small
// grids).
inline int capped_blocks(long long cap, int threads, int max_blocks) {
  long long b = (cap + threads - 1) / threads;
  return b < 1 ? 1 : (b > max_blocks ? max_blocks : (int)b);
}

// ---- launchers implemented in the .cu files -----------------------------------
SceneView scene_view(const neb_ctx* c);

// neb_bvh.cu
cudaError_t build_bvh(neb_ctx* c);
// 4-wide BVH over the n primitives of view s (triangles, then spheres; a
// sphere of radius 0 is a point) into a new device array *nodes_out;
// builder 0 PLOC, 1 Karras.  Synchronises st.
// Shadow walks start in the subtree this many levels above the node that
// holds the origin's primitive (then walk the rest of the tree if needed).
constexpr int kShadowLift = 3;
// parent_out / owner_out (or nullptr): the parent of every 4-wide node (-1 at
// the root) and the node holding each primitive as a leaf child, allocated here
// surface-area sums of the context's 4-wide tree: inner child boxes, leaf boxes, root box
cudaError_t bvh_area_sums(const neb_ctx* c, double out[3]);
cudaError_t build_bvh4(const SceneView& s, int n, int builder, cudaStream_t st, BVH4Node** nodes_out, int* n4_out,
                       int** parent_out = nullptr, int** owner_out = nullptr);
cudaError_t launch_trace_debug(const SceneView& s, const float* d_rays, int n, int* d_prim, float* d_t,
                               uint32_t* d_status, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* d_ctr, int n, uint2 key, uint32_t* d_out, cudaStream_t st);
cudaError_t launch_area(const float* d_boxes, const float* d_pos, const float* d_nrm, int n, double* d_out,
                        cudaStream_t st);

// neb_grid.cu
size_t scan_scratch_ints(size_t n);
size_t group_counter_ints();
int scan_launch_count(size_t n);
cudaError_t scan_exclusive(const int* d_in, int* d_out, size_t n, Scratch& scratch, cudaStream_t st);
cudaError_t grid_build(neb_ctx* c, const IterParams& ip, const IterSlot& sl, cudaStream_t st);
cudaError_t count_neighbours_device(const float* d_pts, int n, const float* d_q, int m, float r, int* d_out,
                                    cudaStream_t st);
// Hashed grid over n points [n][3] with cubic cells of side `cell` from gmin
// and `table` buckets (a power of two): counts (zero on entry, consumed back
// to zero), exclusive-scanned starts (table + 1) and the points in bucket
// order.
cudaError_t build_point_grid(const float* d_pts, int n, float cell, float3 gmin, uint32_t table, int* bucket_count,
                             int* bucket_start, int* vert_bucket, float4* sorted, Scratch& sc, cudaStream_t st);

// neb_merge.cu
// Per-cell merge of the photon hits staged during the photon walks: orders
// them by cell, then merges every cell's hits with the view vertices around
// it.  Returns the number of kernels enqueued through *launches.
cudaError_t merge_staged(neb_ctx* c, const IterParams& ip, const IterSlot& sl, double* accum, double* split,
                         cudaStream_t st, long long* launches);

// neb_octree.cu
OctreeParams octree_params(const float smin[3], const float smax[3], int capacity, int split_factor);
void octree_set_iteration_params(OctreeParams& P, int split_factor, int iter);
cudaError_t launch_oct_rearm(int* nodes, const OctreeState* st, const OctreeParams& P, cudaStream_t s);
cudaError_t launch_oct_insert_points(int* nodes, OctreeState* st, const OctreeParams& P, const float* d_pos, int n,
                                     int mode, cudaStream_t s);
cudaError_t launch_oct_density_points(const int* nodes, const OctreeState* st, const OctreeParams& P,
                                      const float* d_pos, const float* d_nrm, int n, int robust, float* d_out,
                                      cudaStream_t s);
cudaError_t launch_oct_insert_nee(neb_ctx* c, const IterSlot& sl, cudaStream_t st);
cudaError_t launch_oct_density_nee(neb_ctx* c, const IterSlot& sl, cudaStream_t st);

// neb_trace.cu
// packed: recs are PackedPhoton records (direction in octahedral form)
cudaError_t launch_trace_closest(neb_ctx* c, const float4* recs, const int* count_ptr, int cap, int2* hits,
                                 int which, DevCounters* cnt, cudaStream_t st, int packed = 0);
// groups the slot's shadow rays into c->shadow_rays, then walks them
cudaError_t launch_group_shadow(neb_ctx* c, const IterSlot& sl, cudaStream_t st);
cudaError_t launch_trace_shadow(neb_ctx* c, const IterSlot& sl, cudaStream_t st);
int shadow_walk_launches(const neb_ctx* c);  // kernels launch_trace_shadow enqueues
// regroups the camera queue q (count at count_ptr) into out (same count)
cudaError_t launch_group_camera(neb_ctx* c, const CamRay* q, const int* count_ptr, CamRay* out, cudaStream_t st);
// the same for a queue of FP32 photon records, with the photon grouping counters
cudaError_t launch_group_photons(neb_ctx* c, const PhotonRay* q, const int* count_ptr, PhotonRay* out,
                                 cudaStream_t st);

// neb_pass.cu
// overlap: passes 2-3 go to stream_b (ordered by the slot events), else all on c->stream
cudaError_t run_iteration(neb_ctx* c, int iteration, bool overlap);
cudaError_t launch_resolve(const double* accum, int P, int iterations, float* out, cudaStream_t st);
cudaError_t launch_sum_halves(const double* accum, int P, double* out, cudaStream_t st);
cudaError_t launch_error_sums(const double* accum, int P, int n_even, int n_odd, double* out, cudaStream_t st);
cudaError_t launch_read_rho(neb_ctx* c, float* d_out);

}  // namespace neb
