/*
 * neb.h -- C ABI of the GB300 (sm_103a) Next Event Backtracking library,
 * libneb.so.  Jendersie, "Next Event Backtracking" (arXiv 1909.00573).
 *
 * One iteration (neb_iterate) runs the three passes of the method's outline
 * (Sec. 3, Fig. 2) entirely in CUDA kernels on one GPU:
 *   pass 1  view paths; every view vertex where NEE is attempted is stored
 *           and counted in the density octree (Sec. 3.1, Sec. 5.1);
 *   pass 2  density rho at each NEE vertex (Eq. octdensity), NEE
 *           contributions (Sec. 3.2), photons Phi = dE / rho (Eq. flux)
 *           walked from the NEE vertices and merged at view vertices (Sec. 3.2);
 *   pass 3  self emission of stored random hits (Sec. 3.3),
 * weighted by the balance heuristic over all strategies (Sec. 4, Eq. misw).
 *
 * Conventions for every entry point:
 *  - Return value: NEB_OK (0) or a negative NEB_ERR_* code; the message of the
 *    last failure on a context is returned by neb_last_error().
 *  - Host pointers are borrowed for the duration of the call only (data is
 *    copied); the library never keeps or frees caller memory.
 *  - A context owns all of its device memory and its work runs in order on
 *    the CUDA stream given to neb_create (the caller's stream, e.g. the
 *    current PyTorch stream, or NULL for a stream the library creates).
 *    Entry points that return host data synchronise that stream.
 *  - Contexts are not thread-safe; use one context per host thread.
 *  - Layouts of scene arrays are those of paper_1909_00573_gb300/scenes.py:
 *    tri [nt][3][3] float, tri_mat [nt] uint32, sph [ns][4] float (centre,
 *    radius), sph_mat [ns] uint32, mats [nm][12] float (type, albedo rgb,
 *    emission rgb, ior, alpha, pad), cam [10] float (eye, target, up, vfov).
 */
#ifndef NEB_H
#define NEB_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  NEB_OK = 0,
  NEB_ERR_ARG = -1,            /* invalid argument or call order */
  NEB_ERR_OOM = -2,            /* device allocation failed */
  NEB_ERR_CUDA = -3,           /* a CUDA runtime call failed */
  NEB_ERR_DEVICE_TIMEOUT = -4, /* a bounded device spin-wait expired (octree split) */
  NEB_ERR_QUEUE_OVERFLOW = -5, /* a device work queue or stack overflowed */
  NEB_ERR_NO_DEVICE = -6       /* no CUDA device */
};

/* device status word bits, reported by neb_get_stats() */
enum {
  NEB_STATUS_SPIN_TIMEOUT = 1u,   /* an octree insert gave up waiting for a child pointer */
  NEB_STATUS_QUEUE_OVERFLOW = 2u, /* an append found its queue full */
  NEB_STATUS_STACK_OVERFLOW = 4u, /* a BVH traversal stack overflowed */
  NEB_STATUS_OCTREE_FULL = 8u     /* octree allocation overflow (not an error: Appendix B) */
};

typedef struct {
  int width, height;     /* image size; one camera path per pixel per iteration */
  int max_depth;         /* D: maximum path length in segments, 1 <= D <= 64 */
  float merge_radius;    /* r of the uniform kernel 1/(pi r^2) (Sec. 3.2) */
  int octree_capacity;   /* words of the density octree's pool; rounded up to 8m + 1 (the root and groups of eight children, Sec. 5.5) */
  int split_factor;      /* split factor of the density octree, >= 2: a cell splits at split_factor * iteration vertices (paper: 4, Sec. 5.5) */
  uint64_t seed;         /* Philox4x32-10 key */
  int octree_mode;       /* 0 concurrent lock-free inserts, 1 sequential in (pixel, k) order */
  int density_mode;      /* 0 robust: median of five queries (the centre and four displaced along the tangents), 1 single query */
  uint32_t strategy_mask;/* bit 0 random hit (e), bit 1 NEE (E), bit 2 NEB photon merge (P),
                            bit 3 conventional light-photon merge (LP, with lp_photons > 0) */
  int keep_split;        /* nonzero: keep the last iteration's contributions split by strategy */
  int bvh_builder;       /* 0 PLOC clustering over the Morton order (default), 1 Karras LBVH */
  int photon_records;    /* photon queue records: 0 FP32 (64 bytes), 1 packed (48 bytes: FP32
                            origin and MIS factors, RGB flux as three FP16 mantissas of a shared
                            power-of-two scale, direction octahedral with 16 bits per coordinate) */
  int lp_photons;        /* conventional light photons per iteration (n_LP, Sec. 6.1), used when
                            strategy_mask has bit 8; each is emitted from a light and merged at
                            view vertices like the NEB photons, under the same balance heuristic */
  int density_all;       /* 0: rho is evaluated only where a result uses it (NEE vertices whose
                            shadow ray reached the light, for w_E and Phi = dE / rho, and the vertex
                            before each random light hit, for w_e); 1: at every NEE vertex.  The
                            image is the same either way; 1 only fills neb_read_nee_rho */
  int merge_mode;        /* how photon hits are merged with the view vertices within r (Sec. 3.2).
                            Per hit: the hit searches the grid of view vertices as it is made.
                            Per cell: the photon walks stage their hits, and after the last walk
                            the staged hits of each grid cell are merged together, their points in
                            shared memory, each view vertex summing its merges before one FP64
                            addition.  0 (default): hits with more than 16 view vertices in their
                            cells per cell, the others per hit; 1: every hit per hit; 2: every hit
                            per cell.  Hits that find the staging list full merge per hit.  All
                            modes find the same pairs with the same terms; the sums differ only in
                            rounding (per cell, a vertex's merges of one cell add in FP32 first) */
  int merge_hits;        /* staging capacity of modes 0 and 2 in hits per iteration; 0: 2 W H (D - 1) */
} neb_config;

typedef struct {
  int64_t iterations;
  int64_t camera_rays, nee_vertices, shadow_rays, photons, photon_hits;
  int64_t merge_tests, merges, random_hits;
  int64_t octree_inserts, octree_queries;  /* queries count each of the five robust lookups */
  int64_t bvh_node_visits, prim_tests;
  int64_t kernel_launches;                 /* kernels enqueued by neb_iterate */
  int64_t stage_node_visits[3];            /* BVH node visits of the extend, shadow and photon kernels */
  int64_t stage_prim_tests[3];             /* primitive tests of the same kernels */
  int32_t octree_nodes, octree_depth;
  uint32_t status;                         /* NEB_STATUS_* bits, sticky */
  int32_t pad;
  int64_t merge_hits_staged;               /* photon hits merged per cell (merge_mode 0 and 2) */
} neb_stats;

typedef struct neb_ctx neb_ctx;

/* Creates a context bound to `cuda_stream` (cudaStream_t or NULL) and sizes
 * its per-iteration device buffers for cfg (all allocations happen here and
 * in neb_scene_upload / neb_build_bvh, never in neb_iterate). */
int neb_create(const neb_config* cfg, void* cuda_stream, neb_ctx** out);
void neb_destroy(neb_ctx* ctx);
const char* neb_last_error(const neb_ctx* ctx);

/* Copies the scene to the device (SoA triangles as float4 v0, v1, v2; spheres;
 * materials), builds the light list (emissive triangles in index order, then
 * spheres) with power-proportional selection through an alias table (Vose
 * 1991), and derives the octree box from the scene bounds (grown by 0.2 %
 * about their centre, as the paper's implementation does).  Resets the
 * accumulation. */
int neb_scene_upload(neb_ctx* ctx, const float* tri, const uint32_t* tri_mat, int nt,
                     const float* sph, const uint32_t* sph_mat, int ns,
                     const float* mats, int nm, const float* cam);

/* Builds the BVH on the device: Morton codes of primitive centroids on a 2^21
 * grid per axis (one scale for all axes), ordered by their top 62 bits with
 * two stable 4-bit LSD radix sorts (low key, then high key), then either PLOC
 * (Meister and Bittner 2018: rounds of mutual nearest-neighbour merges by
 * union surface area within +-16 positions of the Morton order; default) or
 * the Karras (HPG 2012) hierarchy with bottom-up bounds; the binary tree is
 * then collapsed into a 4-wide tree (128-byte nodes, largest-area child
 * opened first) that all walks use.  Leaves hold one primitive. */
int neb_build_bvh(neb_ctx* ctx);

/* Quality of the built tree by the surface area heuristic (MacDonald and
 * Booth): out[0] = expected 4-wide node visits (root included) and out[1] =
 * expected primitive tests of a ray through the scene box, for rays uniform
 * in space and direction, with no early exit.  Synchronises the context
 * stream.  NEB_ERR_ARG before neb_build_bvh. */
int neb_bvh_cost(neb_ctx* ctx, double* out);

/* Enqueues n_iterations NEB iterations (asynchronous).  Iteration indices
 * continue from the previous call (1-based).  The iterations run on two
 * streams owned by the context, after the work already enqueued on the
 * context stream: pass 1 on a high-priority stream, passes 2-3 of an
 * iteration on a second one, overlapping pass 1 of the next iteration; before
 * the call returns, the context stream is made to wait for the last
 * iteration, so work enqueued on it afterwards sees every result. */
int neb_iterate(neb_ctx* ctx, int n_iterations);

/* Progressive display: enqueues n_iterations iterations like neb_iterate and,
 * after each, the image of all iterations so far (as neb_resolve) copied into
 * rgb_host [H][W][3] float, each copy overwriting the previous one.  The
 * copies follow each iteration's passes 2-3 on the context's second stream,
 * so they do not hold back the next iteration's pass 1 (reading the image
 * through neb_resolve after every neb_iterate call would).  Asynchronous:
 * rgb_host must stay valid and unread until the context stream has been
 * synchronised (it waits for the last copy before the call returns); pinned
 * host memory keeps the copies asynchronous, pageable memory makes each copy
 * wait.  NEB_ERR_ARG for a null buffer or a context without scene and BVH. */
int neb_iterate_read(neb_ctx* ctx, int n_iterations, float* rgb_host);

/* Batched jobs: n_iterations iterations of each of the n contexts, enqueued
 * round-robin (iteration t of every job before iteration t + 1 of any) so
 * the jobs' kernels overlap on the GPU.  The contexts must be distinct and on
 * distinct streams (a NULL stream at neb_create gives each its own); each
 * job's results are exactly those of neb_iterate on it alone.  Returns after
 * enqueueing; each context stream waits for its own last iteration.
 * NEB_ERR_ARG for a null or repeated context, a shared stream, or a context
 * without its scene and BVH. */
int neb_iterate_batch(neb_ctx* const* ctxs, int n, int n_iterations);

/* Device bytes a context keeps between iterations for configuration cfg and
 * a scene of n_tri triangles, n_sph spheres, n_mat materials and n_lights
 * emissive primitives: the buffers of neb_create, neb_scene_upload and
 * neb_build_bvh, computed without allocating (the build needs transient
 * scratch on top).  For admitting many jobs to one GPU.  NEB_ERR_ARG on an
 * invalid cfg or counts. */
int neb_job_device_bytes(const neb_config* cfg, int n_tri, int n_sph, int n_mat, int n_lights, uint64_t* out);

/* Launch settings of a context; none of them changes any result.  Rays are
 * regrouped before they are traced by the cell of their origin in the scene
 * box and the cell of their direction (camera rays after the first bounce)
 * or of their light point (shadow rays), with 2^bits cells per axis;
 * 3 (origin_bits + other_bits) <= 12 for each.  shade_blocks_per_sm sizes the
 * grid of the shading kernels.  Defaults {1, 3, 2, 2, 8}. */
typedef struct {
  int cam_origin_bits, cam_dir_bits;         /* each in [0, 4] */
  int shadow_origin_bits, shadow_light_bits; /* each in [0, 4] */
  int shade_blocks_per_sm;                   /* [1, 32] */
  int photon_grouping;                       /* 0 or 1: regroup photon rays before each photon walk (only
                                                where the context holds a queue for it: FP32 photon
                                                records and a photon queue of at least 2^20 rays) */
} neb_tuning;
int neb_get_tuning(const neb_ctx* ctx, neb_tuning* out);
/* NEB_ERR_ARG for values out of range; applies from the next iteration. */
int neb_set_tuning(neb_ctx* ctx, const neb_tuning* t);
/* Autotuner: coordinate descent over candidate camera groupings, then
 * shadow groupings, then shading grid sizes, each candidate timed (CUDA
 * events on the context stream) over iterations_per_candidate iterations.
 * These are real iterations: they add to the image like any other.  Keeps
 * the fastest settings, writes them to *chosen (may be NULL) and returns
 * after the last candidate has finished. */
int neb_autotune(neb_ctx* ctx, int iterations_per_candidate, neb_tuning* chosen);

/* Progressive result: FP64 per-pixel sums divided by the iteration count,
 * written as [H][W][3] float.  out_is_device: nonzero if rgb_out is device
 * memory (written on the context stream), zero for host memory (synchronises). */
int neb_resolve(neb_ctx* ctx, float* rgb_out, int out_is_device);

/* Waits until everything enqueued on the context so far (iterations,
 * resolves, copies) has finished; other contexts' work is not waited for.
 * NEB_ERR_CUDA on a device error. */
int neb_synchronize(neb_ctx* ctx);

/* Raw FP64 sums [H][W][3] (host memory; synchronises). */
int neb_read_accum(neb_ctx* ctx, double* out);

/* Relative RMSE of the progressive image, estimated from its own samples:
 * contributions of even and odd iterations are summed apart, and with m_e,
 * m_o their per-pixel means (luminance, the sum of the channels) over the
 * n_e, n_o iterations of each parity, the variance of the mean of all n
 * iterations is Var(m_e - m_o) n_e n_o / n^2.  *rel_rmse = sqrt(sum over
 * pixels of that variance / sum of the squared mean).  It measures the
 * noise, not the bias of the consistent estimator (Sec. 3.2, Sec. 5).
 * Needs at least two iterations (else NEB_ERR_ARG); synchronises the context
 * stream. */
int neb_error_estimate(neb_ctx* ctx, double* rel_rmse);

/* Last iteration's contributions split by strategy [4][H][W][3] (0 random hit,
 * 1 NEE, 2 NEB photon merge, 3 light-photon merge); requires cfg.keep_split.
 * Host memory. */
int neb_read_split(neb_ctx* ctx, double* out);

/* Density rho at every NEE vertex of the last iteration, [H*W][D-1] indexed
 * pixel*(D-1) + (k-1); -1 where the path has no NEE vertex k, -2 where rho
 * was not evaluated (cfg.density_all = 0 and no result uses it).  Host memory. */
int neb_read_nee_rho(neb_ctx* ctx, float* out);
/* The NEE vertices of the last iteration in store order: positions and
 * geometric normals [cap][3] (host), *count = their number (at most
 * W*H*(D-1); only the first min(count, cap) are written). */
int neb_read_nee_vertices(neb_ctx* ctx, float* pos, float* nrm, int cap, int* count);

/* Counters accumulated since the scene upload, plus the device status word.
 * Synchronises.  Returns NEB_ERR_DEVICE_TIMEOUT / NEB_ERR_QUEUE_OVERFLOW if the
 * corresponding status bit is set (the stats are filled in either case). */
int neb_get_stats(neb_ctx* ctx, neb_stats* out);

/* Per-stage device times in milliseconds, accumulated over iterations since
 * profiling was enabled (CUDA events on the context stream around each
 * stage).  names receives up to max_stages NUL-terminated names of <= 31
 * chars (32 bytes each); returns the number of stages. */
int neb_set_profiling(neb_ctx* ctx, int enable);
int neb_get_stage_times(neb_ctx* ctx, double* ms, int64_t* launches, char* names, int max_stages);

/* ---------------- component entry points (tests and tools) --------------- */

/* Closest hit of n rays [n][6] (origin, unit direction) through the BVH:
 * prim index (-1 on a miss; triangles first, then spheres) and distance. */
int neb_trace_closest(neb_ctx* ctx, const float* rays, int n, int32_t* out_prim, float* out_t);

/* Philox4x32-10 on the device: n counters [n][4] under one key -> [n][4]. */
int neb_philox(const uint32_t* ctr, int n, const uint32_t key[2], uint32_t* out);

/* Area of the plane through a point with a unit normal inside an
 * axis-aligned box (Eq. area, Sec. 5.3 and Appendix A), evaluated in FP64
 * on the device for n cases, as the density query evaluates it: boxes [n][6]
 * (min, max), points [n][3], normals [n][3] (host arrays, copied); out [n]
 * (host).  A normal component within 1e-3 of +-1 gives the face area across
 * that axis; otherwise a component below 1e-4 is taken as zero (the
 * thresholds of the paper's implementation).  NEB_ERR_ARG for n < 0 or a
 * missing array, NEB_ERR_NO_DEVICE / NEB_ERR_OOM / NEB_ERR_CUDA. */
int neb_plane_box_area(const float* boxes, const float* pos, const float* nrm, int n, double* out);

/* Stand-alone density octree (Sec. 5) on the device: one int32 word per
 * cell, siblings in consecutive words, a word >= 0 a count and < 0 the
 * negated index of the cell's first child (Sec. 5.5); word 0 is the root.
 * The octree box is the scene box grown by 0.2 % about its centre; the word
 * pool holds `capacity` rounded up to 8m + 1 words.  split_factor >= 2. */
typedef struct neb_octree neb_octree;
int neb_octree_create(const float scene_min[3], const float scene_max[3], int capacity,
                      int split_factor, void* cuda_stream, neb_octree** out);
void neb_octree_destroy(neb_octree* o);
/* Starts iteration iter >= 1 (Sec. 5.4): split threshold split_factor *
 * min(iter, 1000), densities divided by min(iter, 1000), every free word
 * set to the count a new cell starts with, ceil(split_factor * iter / 4);
 * after iteration 1000 inserts are ignored. */
int neb_octree_set_iteration(neb_octree* o, int iter);
/* Counts n positions [n][3] (Sec. 5.1-5.2): each adds one to the leaf cell
 * holding it, and the position that brings a cell to the threshold splits
 * it (eight new cells from the pool; no room: the pool is marked exhausted
 * and cells keep counting).  mode 0: concurrent, one thread per position,
 * compare-and-swap counts, positions that count past the threshold while the
 * split is published wait for it (bounded) and count again in the child;
 * mode 1: one device thread in array order (deterministic).  Positions
 * outside the octree box are ignored. */
int neb_octree_insert(neb_octree* o, const float* pos, int n, int mode);
/* Density (Eq. octdensity) at n positions with geometric normals [n][3]:
 * robust = 0 one query, count / (iterations * max(floor, A)) with A the
 * plane's area in the leaf cell (FP64) and floor 0.01 of the squared cell
 * diagonal; robust = 1 the median of that query (floor 0.1) and four more
 * displaced by 1.1 cell diagonals along the tangents of the Duff et al.
 * basis, the upper of the middle two for an even count.  0 for an empty
 * cell or a position outside the box. */
int neb_octree_density(neb_octree* o, const float* pos, const float* nrm, int n, int robust, float* out);
/* Copies the node array (capacity entries) and meta = {alloc, depth, capacity, status}. */
int neb_octree_read(neb_octree* o, int32_t* nodes, int n_nodes, int32_t meta[4]);
/* Restores a node array and its allocation state, e.g. one read back by
 * neb_octree_read, to resume a density estimate (the octree integrates over
 * iterations, Sec. 5.4).  nodes: n_nodes host entries, 1 <= n_nodes <=
 * capacity, copied before return; entries past n_nodes become 0.  alloc:
 * the words in use, 1 + 8m <= capacity, or capacity + 1 when the pool was
 * exhausted; depth in [0, 30]; the status word is cleared.  NEB_ERR_ARG for
 * values out of range.
 * Node values are taken as given: a non-negative counter above the split
 * threshold with no child (a state inserts never leave) makes concurrent
 * inserts through it wait out their bounded spin, drop the position and
 * return NEB_ERR_DEVICE_TIMEOUT. */
int neb_octree_load(neb_octree* o, const int32_t* nodes, int n_nodes, int alloc, int depth);

/* The density estimators of Sec. 5 side by side, for n points [n][3] with
 * geometric normals [n][3] (host) taken as the NEE vertices of one
 * iteration; every estimate is made at each of the points and written to
 * rho[3][n]: (0) the density octree as the pass uses it (concurrent insert,
 * the robust median-of-five query; scene box, capacity and split factor as
 * in neb_octree_create); (1) the naive estimator: points within `radius` of
 * the point, itself included, / (pi radius^2), through a hashed grid;
 * (2) the k-nearest-neighbour estimator (k - 1) / (pi d_k^2), d_k the
 * distance to the k-th nearest other point (2 <= k <= 16; 0 with fewer than k
 * other points), through a 4-wide tree built over the points.  ms[3] (may be
 * NULL) receives each estimator's device time in milliseconds, structure
 * build plus queries, CUDA events on its stream.  NEB_ERR_ARG for bad sizes. */
int neb_density_estimators(const float* pos, const float* nrm, int n, const float scene_min[3],
                           const float scene_max[3], int octree_capacity, int split_factor, float radius, int k,
                           float* rho, double* ms);

/* Merge candidate search through the device hashed grid (cell size 2r, the
 * structure used by the photon merge): for each query, the number of points
 * with |p - q|^2 <= r^2 evaluated in FP32.  Grid cells are held within
 * +-2^30 per axis; far points share the boundary cell and counts stay exact
 * (slower when many points lie beyond it). */
int neb_count_neighbours(const float* pts, int n, const float* queries, int m, float r, int32_t* out);

/* The same neighbour count for callers that cannot allocate device memory:
 * for example a host application whose device memory is entirely reserved by
 * its own pooling allocator, or a latency-critical loop that must not hit the
 * device-wide synchronisation cudaMalloc and cudaFree can cause.  The paper
 * has no counterpart; this is a library service.
 *
 * d_pts [n][3], d_queries [m][3] and d_out [m] are DEVICE pointers owned by
 * the caller; cuda_stream is a cudaStream_t of the current device (NULL: the
 * default stream; a stream of another device returns NEB_ERR_ARG).  The
 * call only enqueues work (memset + kernels) on that stream and returns;
 * synchronise before reading d_out.  It allocates nothing: its scratch is a
 * fixed ~9 MiB array inside the library image (held by every GPU that loads
 * the library until the process exits), so n may not exceed
 * NEB_NOALLOC_MAX_POINTS (larger n returns NEB_ERR_ARG; m is unlimited).
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * The library keeps that address for the rest of the process: after a
 * cudaDeviceReset of the device it is stale, so do not call this entry point
 * on a device that has been reset.
 * Every call on a device shares the one array: calls whose work overlaps on
 * the GPU (other streams, other host threads) race and corrupt each other's
 * results; serialise them.  Results equal those of neb_count_neighbours. */
#define NEB_NOALLOC_MAX_POINTS (1 << 18)
int neb_count_neighbours_noalloc(const float* d_pts, int n, const float* d_queries, int m, float r,
                                 int32_t* d_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
