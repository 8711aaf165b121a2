/*
 * neb_oracle.h -- plain, single-threaded CPU oracle of the Next Event
 * Backtracking (NEB) iteration (Jendersie, "Next Event Backtracking").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: it has its own BVH, its own intersection routines, its
 * own octree and computes every MIS weight explicitly from the full vertex
 * list of the path (Eq. misweight .. Eq. misw), where the GPU uses a
 * recursive form.
 *
 * Precision: ray/primitive tests, hit points, the plane/box area and the
 * density quotient are FP64; vertex positions, directions and sampling
 * decisions are FP32, and so are the decisions the paper takes in FP32
 * (the octree cell a position falls in, the displaced points of the robust
 * density query, the case of the area formula); all radiometric quantities,
 * MIS products and the accumulation are FP64.  Build with
 * -ffp-contract=off so the FP32 parts round the same way on every host.
 */
#ifndef NEB_ORACLE_H
#define NEB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Scene arrays; layouts are documented in paper_1909_00573_gb300/scenes.py. */
typedef struct {
  const float* tri;       /* [nt][3][3] */
  const uint32_t* tri_mat;/* [nt] */
  int nt;
  const float* sph;       /* [ns][4] centre, radius */
  const uint32_t* sph_mat;/* [ns] */
  int ns;
  const float* mats;      /* [nm][12] */
  int nm;
  const float* cam;       /* [10] */
} orc_scene;

typedef struct {
  int width, height, max_depth;
  float merge_radius;
  int octree_capacity, split_factor;
  uint64_t seed;
  int density_mode;        /* 0 robust (median of 5), 1 single query */
  uint32_t strategy_mask;  /* 1 random hit, 2 NEE, 4 NEB photon merge, 8 conventional light photon merge */
  int first_iteration;     /* 1-based index of the first iteration rendered */
  int pixel_begin, pixel_end; /* camera paths traced: [begin, end) (row-major), end<=0: all */
  double* iter_seconds;       /* optional [n_iter]: wall time of each iteration (BVH build excluded) */
  int lp_photons;             /* conventional light photons per iteration (n_LP, Sec. 6.1; strategy bit 8) */
  double* iter_images;        /* optional [n_iter][H*W*3]: each iteration's own contributions */
} orc_config;

/* stats[] slots filled by orc_render (summed over iterations) */
enum {
  ORC_ST_CAMERA_RAYS = 0, ORC_ST_NEE_VERTICES, ORC_ST_SHADOW_RAYS, ORC_ST_PHOTONS,
  ORC_ST_PHOTON_HITS, ORC_ST_MERGES, ORC_ST_RANDOM_HITS, ORC_ST_OCTREE_NODES,
  ORC_ST_OCTREE_DEPTH, ORC_ST_COUNT
};

/* Render n_iter iterations.  accum: [H*W*3] FP64 sums over the iterations
 * (not divided).  last_split (may be NULL): [3][H*W*3] contributions of the
 * last iteration split by event type (0 random hit, 1 NEE, 2 photon merge).
 * nee_rho (may be NULL): [H*W*(D-1)] density at every NEE vertex of the last
 * iteration, indexed pixel*(D-1) + (k-1), -1 where no NEE vertex exists.
 * Returns 0 on success. */
int orc_render(const orc_scene* scene, const orc_config* cfg, int n_iter,
               double* accum, double* last_split, float* nee_rho, int64_t* stats);

/* ---- unit entry points used by the pin tests ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Eq. area (Sec. 5.3, Appendix A) for the plane through pos with unit normal
 * `normal` and the box [bmin, bmax], in FP64. */
double orc_intersection_area(const float bmin[3], const float bmax[3],
                             const float pos[3], const float normal[3]);

typedef struct orc_octree orc_octree;
orc_octree* orc_octree_new(const float scene_min[3], const float scene_max[3],
                           int capacity, int split_factor);
void orc_octree_free(orc_octree* o);
void orc_octree_set_iteration(orc_octree* o, int iter);
void orc_octree_increment(orc_octree* o, const float pos[3]);
float orc_octree_density(orc_octree* o, const float pos[3], const float normal[3], int robust);
/* The tree in the flat word layout of Sec. 5.5 (a leaf's word its count, a
 * split cell's word the negated index of its first child, words no cell has
 * taken the count a new cell would start with): copies min(n, capacity)
 * words; returns capacity.  meta: words used, depth, capacity. */
int orc_octree_dump(const orc_octree* o, int32_t* nodes, int n, int32_t meta[3]);
/* Replaces the tree by the one in the flat layout words[n] (word 0 the root);
 * words used and depth as given.  0, or -1 for a malformed layout. */
int orc_octree_load(orc_octree* o, const int32_t* words, int n, int words_used, int depth);

/* Tangent t and bitangent b of unit normal n (Duff et al. 2017, the basis of
 * the robust density query). */
void orc_onb(const float n[3], float t[3], float b[3]);

/* Light selection as the renderer does it: Vose's alias table over `power`
 * (psel[i] = power[i] / sum), then n_samples choices with Philox words keyed
 * by seed (counter: sample k, stream 0, dims 0-1, iteration 1) counted in
 * counts[n].  0, or -1 for n < 1. */
int orc_light_selection(const double* power, int n, int n_samples, uint64_t seed, double* psel, int64_t* counts);

/* BVH parity helpers: closest hit for n rays ([n][6] origin, direction);
 * out_prim -1 on miss, out_t the hit distance.  brute != 0 tests every
 * primitive instead of walking the BVH. */
int orc_trace(const orc_scene* scene, const float* rays, int n, int brute,
              int32_t* out_prim, float* out_t);

/* Merge candidate enumeration helper: for every query point, the number of
 * points within radius r (d^2 <= r^2 in FP32).  brute != 0 uses the O(N*M)
 * scan, otherwise the sorted-window search used by orc_render. */
void orc_count_neighbours(const float* pts, int n, const float* queries, int m,
                          float r, int brute, int32_t* out_count);

/* The two density estimators the paper tried before its octree (Sec. 5),
 * by brute force, each evaluated at every one of the n points [n][3]:
 * naive: the points within `radius` of the point, itself included, divided
 * by pi radius^2; k nearest (Loftsgaarden and Quesenberry 1965):
 * (k - 1) / (pi d_k^2), d_k^2 the k-th smallest squared distance to the other
 * points (0 when there are fewer than k).  Squared distances in FP32
 * (other - point, x + y + z order), the quotient in FP64 rounded to FP32. */
void orc_density_naive(const float* pts, int n, float radius, float* out);
void orc_density_knn(const float* pts, int n, int k, float* out);

/* Balance-heuristic weights of every strategy for one explicit path (used by
 * the MIS pin tests).  See the definition of orc_path in the source. */
int orc_mis_weights(const float* verts, int n_verts, const float* light,
                    float merge_radius, double rho, uint32_t mask, double* w_out);
/* The same with conventional light photons (Sec. 6.1): light = pos, normal,
 * p_l (NEE area pdf of the light point), p_l^LP (its pdf under light-photon
 * emission); n_lp light photons per iteration; mask bit 8 enables them.
 * w_out: [l + 1 + (l - 1)] = w_e, w_E, w_P1 .. w_P(l-2), w_LP1 .. w_LP(l-1). */
int orc_mis_weights_lp(const float* verts, int n_verts, const float* light, float merge_radius, double rho,
                       uint32_t mask, double n_lp, double* w_out);

/* BSDF probes for the pin tests (material row in the scenes layout). */
int orc_bsdf_probe(const float* mrow, const float* n, const float* wo, const float* u, int camera, float* wi,
                   double* weight, double* pdf_out, double* f_out);
void orc_bsdf_eval_probe(const float* mrow, const float* n, const float* wo, const float* wi, double* f_out,
                         double* pdf_out);

#ifdef __cplusplus
}
#endif
#endif
