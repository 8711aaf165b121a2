// neb_merge.cu -- the per-cell photon merge (Sec. 3.2: every photon hit x is
// merged with the view vertices x_k within r of it, kernel 1 / (pi r^2)).
//
// The photon walks stage the hits they would merge (MergeHit records); after
// the last walk the hits are ordered by bucket of a hashed grid of the view
// vertices' cells (side 2r) and cut into tiles of at most kMergeTile hits of
// one bucket.  A tile's hits are staged in shared memory and split by cell
// (distinct cells can share a bucket); for each cell the view vertices of the
// grid cells within r of its hits are walked.  A vertex farther than r from
// the box of the cell's hits is dropped after one test; the others are taken
// 32 at a time, one per lane, and tested against every hit of the cell from
// shared memory.  Accepted pairs queue up in shared memory and are evaluated
// 32 at a time, one per lane, and each vertex sums its merges in shared
// memory before one FP64 addition per channel to its pixel.  Each warp takes
// one tile at a time, full tiles (dense cells) first; a warp never waits for
// another, and a dense cell is spread over as many warps as it has tiles.
//
// The pairs found are exactly those of the per-hit search (the same FP32
// distance test, and the box test never rejects a vertex the distance test
// would accept: FP32 subtraction, squaring and addition are monotone), and
// each pair's term is computed as there; only the order and precision of the
// per-vertex partial sums differ (FP32 sums of one tile's merges, then FP64).
#include <cuda_runtime.h>

#include <cfloat>

#include "neb_accum.cuh"
#include "neb_device.cuh"
#include "neb_internal.h"

namespace neb {

constexpr int kMergeTile = 64;  // staged hits of one bucket merged together (at most)
// Staged hits are ordered by cells of side 2r / kHitCellSplit: smaller cells
// give each tile a smaller box, so fewer view vertices come within r of it.
constexpr float kHitCellSplit = 2.0f;
constexpr int kMergeWarps = 4;  // warps per block of the merge kernel
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNoGroup = 0xffffu;

// Cell of a staged hit (side 2r / kHitCellSplit; cell_inv is 1 / (2r)).
__device__ __forceinline__ int3 hit_cell(float4 k, float3 gmin, float cell_inv) {
  const float ci = cell_inv * kHitCellSplit;
  return make_int3(grid_cell_index((k.x - gmin.x) * ci), grid_cell_index((k.y - gmin.y) * ci),
                   grid_cell_index((k.z - gmin.z) * ci));
}

__device__ __forceinline__ bool same_cell(int3 a, int3 b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

// Warp-aggregated reservation of slots in a list of capacity cap (all lanes
// call it together): the lane's slot, or -1 when pred is false or the list
// is full.  The counter keeps counting past cap.
__device__ __forceinline__ int warp_reserve(int* counter, bool pred, int cap) {
  const unsigned mask = __ballot_sync(kFull, pred);
  if (mask == 0) return -1;
  const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(kFull, base, leader);
  if (!pred) return -1;
  const int slot = base + __popc(mask & ((1u << lane) - 1u));
  return slot < cap ? slot : -1;
}

// ---- ordering of the staged hits by cell -------------------------------------

__global__ void k_mh_count(const MergeHit* __restrict__ mh, const DevCounters* cnt, int cap, float3 gmin,
                           float cell_inv, uint32_t pmask, int* __restrict__ pb_count) {
  const int n = min(cnt->mh_count, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int3 c = hit_cell(__ldg(&mh[i].key), gmin, cell_inv);
    atomicAdd(pb_count + grid_hash(c.x, c.y, c.z, pmask), 1);
  }
}

// Writes each hit's index into its bucket range (the counts are consumed back
// to zero) and emits a tile at every kMergeTile-th position of a bucket: full
// tiles from the front of the tile list, the last, partial tile of each
// bucket from its back.
__global__ void k_mh_scatter(const MergeHit* __restrict__ mh, DevCounters* cnt, int cap, float3 gmin,
                             float cell_inv, uint32_t pmask, const int* __restrict__ pb_start, int* pb_count,
                             int* __restrict__ sorted, int2* __restrict__ tiles) {
  const int n = min(cnt->mh_count, cap);
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const int i = base + threadIdx.x;
    bool first = false;
    int2 t = make_int2(0, 0);
    if (i < n) {
      const int3 c = hit_cell(__ldg(&mh[i].key), gmin, cell_inv);
      const uint32_t b = grid_hash(c.x, c.y, c.z, pmask);
      const int b0 = pb_start[b];
      const int slot = b0 + atomicSub(pb_count + b, 1) - 1;
      sorted[slot] = i;
      if ((slot - b0) % kMergeTile == 0) {
        first = true;
        t = make_int2(slot, min(kMergeTile, pb_start[b + 1] - slot));
      }
    }
    const bool full = t.y == kMergeTile;
    const int tb = warp_reserve(&cnt->mh_tiles, first && full, cap);
    const int ts = warp_reserve(&cnt->mh_small, first && !full, cap);
    if (tb >= 0) tiles[tb] = t;
    if (ts >= 0) tiles[cap - 1 - ts] = t;
  }
}

// ---- the merge -------------------------------------------------------------------

struct MergeWarp {
  float4 key[kMergeTile];  // staged hit points; w: kmax | channel bit << 8 | group << 16
  float4 dir[kMergeTile];  // -photon direction, w: c1'
  float4 phi[kMergeTile];  // flux / c0, w: c2'
  int sv[64];              // grid entries of the view vertices kept for the next round
  int q[96];               // accepted pairs: hit << 6 | channel bit << 5 | lane of the vertex
  float4 vb[4][32];        // the round's vertices by lane: (n, cos_o = n.wo); (tau f, pdf of wo) for a
                           // diffuse vertex, (tau, -alpha) for a rough conductor; (wo, Cfac); (albedo, ior)
  float acc[2][32][3];     // per-lane vertex sums: NEB photons, light photons
};

struct MergeArgs {
  const MergeHit* mh;
  const int* sorted;
  const int2* tiles;
  const MergeRec* mrec;
  const int* bucket_start;  // the view-vertex grid
  NeeStore nv;
  const float4* mats;
  double* accum;
  double* split;
  DevCounters* cnt;
  int cap;
};

// Evaluates the first n queued pairs, one per lane, adding each term to the
// sum of its vertex.  The terms are those of the per-hit merge: a diffuse
// vertex's f, its pdf towards wo and tau f are taken from the round's
// vertex fields, computed there as the per-hit merge computes them.
__device__ __forceinline__ void merge_pairs(const IterParams& ip, MergeWarp& w, int n, uint32_t& merges) {
  const int lane = threadIdx.x & 31;
  if (lane >= n) return;
  const int ent = w.q[lane];
  const int g = ent >> 6, ch = (ent >> 5) & 1, vl = ent & 31;
  const float4 f0 = w.vb[0][vl], f1 = w.vb[1][vl];
  const float4 d4 = w.dir[g];
  const float3 nrm = xyz(f0), md = xyz(d4);
  float3 T;
  float pdfF, pdfC;
  if (f1.w >= 0.0f) {
    // diffuse: f = albedo / pi wherever cos_o cos_i > 0
    const float ci = dot(nrm, md);
    if (!(f0.w * ci > 0.0f)) return;
    pdfF = fabsf(ci) * kInvPi;
    pdfC = f1.w;
    T = xyz(f1);
  } else {
    const float4 v2 = w.vb[2][vl], v3 = w.vb[3][vl];
    Mat cm;
    cm.type = MAT_GGX;
    cm.albedo = xyz(v3);
    cm.emission = f3(0, 0, 0);
    cm.ior = v3.w;
    cm.alpha = -f1.w;
    const float3 cwo = xyz(v2);
    const float3 f = bsdf_eval(cm, nrm, cwo, md);
    if (!(maxc(f) > 0.0f)) return;
    pdfF = bsdf_pdf(cm, nrm, cwo, md);
    pdfC = bsdf_pdf(cm, nrm, md, cwo);
    T = cmul(xyz(f1), f);
  }
  const float4 p4 = w.phi[g];
  const float inv_w = 1.0f + d4.w * pdfF + p4.w * pdfC * w.vb[2][vl].w;
  const float3 L3 = mul(cmul(T, xyz(p4)), ip.kernel / inv_w);
  float* s = w.acc[ch][vl];
  atomicAdd(s, L3.x);
  atomicAdd(s + 1, L3.y);
  atomicAdd(s + 2, L3.z);
  ++merges;
}

// Appends the lanes that accept hit g (key bits kb) to the pair queue (all
// lanes call it).
__device__ __forceinline__ void queue_pairs(MergeWarp& w, bool ok, int g, int kb, int& qn) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(kFull, ok);
  if (ok) w.q[qn + __popc(m & ((1u << lane) - 1u))] = (g << 6) | (((kb >> 8) & 1) << 5) | lane;
  qn += __popc(m);
}

// Evaluates full batches of 32 queued pairs while there are any.
__device__ __forceinline__ void drain_pairs(const IterParams& ip, MergeWarp& w, int& qn, uint32_t& merges) {
  const int lane = threadIdx.x & 31;
  while (qn >= 32) {
    __syncwarp();
    merge_pairs(ip, w, 32, merges);
    __syncwarp();
    // each lane reads its own entries before writing them one batch lower
    for (int i = lane; i < qn - 32; i += 32) w.q[i] = w.q[i + 32];
    qn -= 32;
    __syncwarp();
  }
}

// One round: up to 32 view vertices (grid entries w.sv[0..nsv)), one per
// lane, against every staged hit of group grp.
__device__ __forceinline__ void merge_round(const MergeArgs& a, const IterParams& ip, MergeWarp& w, int n, int nsv,
                                            uint32_t grp, bool one_group, uint32_t& tests, uint32_t& merges) {
  const int lane = threadIdx.x & 31;
  bool valid = lane < nsv;
  float3 vp = f3(0, 0, 0);
  int kk = 64, pixel = 0;
  if (valid) {
    const float4 mp = __ldg(&a.mrec[w.sv[lane]].pos);
    const int id = __float_as_int(mp.w);
    const float4 nr = __ldg(&a.nv.nrm[id]), wo = __ldg(&a.nv.wo[id]);
    const float cfac = __ldg(&a.nv.pos[id].w);
    const float4 tau = __ldg(&a.nv.tau[id]);
    const int bits = __float_as_int(nr.w);
    const Mat cm = load_mat(a.mats, bits & NV_MAT_MASK);
    vp = xyz(mp);
    kk = (bits >> NV_K_SHIFT) & 63;
    pixel = __float_as_int(wo.w);
    const float co = dot(xyz(nr), xyz(wo));
    w.vb[0][lane] = make_float4(nr.x, nr.y, nr.z, co);
    w.vb[2][lane] = make_float4(wo.x, wo.y, wo.z, cfac);
    if (cm.type == MAT_DIFFUSE) {
      const float3 f = mul(cm.albedo, kInvPi);
      valid = maxc(f) > 0.0f;  // a black vertex merges nothing
      const float3 T = cmul(xyz(tau), f);
      w.vb[1][lane] = make_float4(T.x, T.y, T.z, fabsf(co) * kInvPi);
    } else {
      w.vb[1][lane] = make_float4(tau.x, tau.y, tau.z, -cm.alpha);
      w.vb[3][lane] = make_float4(cm.albedo.x, cm.albedo.y, cm.albedo.z, cm.ior);
    }
  }
  __syncwarp();
  int qn = 0;
  for (int g = 0; g < n; g += 2) {
    // two hits per step (the second may be past the end)
    const bool has1 = g + 1 < n;
    const float4 k0 = w.key[g], k1 = w.key[has1 ? g + 1 : g];
    const int b0 = __float_as_int(k0.w), b1 = __float_as_int(k1.w);
    const bool in0 = one_group || ((uint32_t)b0 >> 16) == grp;
    const bool in1 = has1 && (one_group || ((uint32_t)b1 >> 16) == grp);
    const float dx0 = vp.x - k0.x, dy0 = vp.y - k0.y, dz0 = vp.z - k0.z;
    const float dx1 = vp.x - k1.x, dy1 = vp.y - k1.y, dz1 = vp.z - k1.z;
    const float d20 = dx0 * dx0 + dy0 * dy0 + dz0 * dz0;
    const float d21 = dx1 * dx1 + dy1 * dy1 + dz1 * dz1;
    tests += valid ? (uint32_t)in0 + (uint32_t)in1 : 0u;
    queue_pairs(w, valid && in0 && d20 <= ip.r2 && kk <= (b0 & 0xff), g, b0, qn);
    queue_pairs(w, valid && in1 && d21 <= ip.r2 && kk <= (b1 & 0xff), g + 1, b1, qn);
    drain_pairs(ip, w, qn, merges);
  }
  __syncwarp();
  if (qn > 0) merge_pairs(ip, w, qn, merges);
  __syncwarp();
  if (lane < nsv) {
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
      float* s = w.acc[ch][lane];
      const float3 L = f3(s[0], s[1], s[2]);
      if (L.x != 0.0f || L.y != 0.0f || L.z != 0.0f) add_pixel(a.accum, a.split, 2 + ch, pixel, L, ip.W * ip.H);
      s[0] = s[1] = s[2] = 0.0f;
    }
  }
  __syncwarp();
}

// The n staged hits' group grp (one cell) against the view vertices around
// them.
__device__ __forceinline__ void merge_group(const MergeArgs& a, const IterParams& ip, MergeWarp& w, int n,
                                            uint32_t grp, bool one_group, uint32_t& tests, uint32_t& merges) {
  const int lane = threadIdx.x & 31;
  // box of the group's hits
  float3 lo = f3(FLT_MAX, FLT_MAX, FLT_MAX), hi = f3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
  for (int g = lane; g < n; g += 32) {
    const float4 k = w.key[g];
    if (!one_group && ((uint32_t)__float_as_int(k.w) >> 16) != grp) continue;
    lo = f3(fminf(lo.x, k.x), fminf(lo.y, k.y), fminf(lo.z, k.z));
    hi = f3(fmaxf(hi.x, k.x), fmaxf(hi.y, k.y), fmaxf(hi.z, k.z));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = f3(fminf(lo.x, __shfl_xor_sync(kFull, lo.x, o)), fminf(lo.y, __shfl_xor_sync(kFull, lo.y, o)),
            fminf(lo.z, __shfl_xor_sync(kFull, lo.z, o)));
    hi = f3(fmaxf(hi.x, __shfl_xor_sync(kFull, hi.x, o)), fmaxf(hi.y, __shfl_xor_sync(kFull, hi.y, o)),
            fmaxf(hi.z, __shfl_xor_sync(kFull, hi.z, o)));
  }
  // grid cells (side 2r) within r of the box (a margin of r / 100 covers the
  // rounding of the cell indices); the hits share one cell of side at most
  // 2r, so at most three per axis
  const float pad = 1.01f * ip.r;
  int c0[3], nc[3];
  {
    const float l3[3] = {lo.x, lo.y, lo.z}, h3[3] = {hi.x, hi.y, hi.z}, g3[3] = {ip.gmin.x, ip.gmin.y, ip.gmin.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      c0[ax] = grid_cell_index((l3[ax] - pad - g3[ax]) * ip.cell_inv);
      const int c1 = grid_cell_index((h3[ax] + pad - g3[ax]) * ip.cell_inv);
      nc[ax] = min(max(c1 - c0[ax] + 1, 1), 3);
    }
  }
  const int ncell = nc[0] * nc[1] * nc[2];
  // lanes without an occupied cell hold distinct dummies
  uint32_t b = 0x80000000u | (uint32_t)lane;
  bool occ = false;
  if (lane < ncell) {
    const int ix = lane % nc[0], iy = (lane / nc[0]) % nc[1], iz = lane / (nc[0] * nc[1]);
    occ = cell_occupied(ip.cell_bits, ip.cell_bits_mask, c0[0] + ix, c0[1] + iy, c0[2] + iz);
    if (occ) b = grid_hash(c0[0] + ix, c0[1] + iy, c0[2] + iz, ip.table_mask);
  }
  // a bucket reached from two cells is walked once
  const unsigned same = __match_any_sync(kFull, b);
  const bool own = occ && __ffs(same) - 1 == lane;
  int start = 0, len = 0;
  if (own) {
    start = __ldg(a.bucket_start + b);
    len = __ldg(a.bucket_start + b + 1) - start;
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  int nsv = 0;
  const unsigned lt = (1u << lane) - 1u;
  for (int q0 = 0; q0 < total; q0 += 32) {
    const int q = q0 + lane;
    // owner lane of entry q: the number of lanes whose inclusive count is <= q
    int L = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) {
      const int v = __shfl_sync(kFull, incl, L + st - 1);
      if (v <= q) L += st;
    }
    L = min(L, 31);
    const int e = __shfl_sync(kFull, start, L) + q - (__shfl_sync(kFull, incl, L) - __shfl_sync(kFull, len, L));
    bool keep = false;
    if (q < total) {
      const float4 mp = __ldg(&a.mrec[e].pos);
      const float bx = mp.x < lo.x ? lo.x - mp.x : (mp.x > hi.x ? mp.x - hi.x : 0.0f);
      const float by = mp.y < lo.y ? lo.y - mp.y : (mp.y > hi.y ? mp.y - hi.y : 0.0f);
      const float bz = mp.z < lo.z ? lo.z - mp.z : (mp.z > hi.z ? mp.z - hi.z : 0.0f);
      keep = bx * bx + by * by + bz * bz <= ip.r2;
    }
    const unsigned m = __ballot_sync(kFull, keep);
    if (keep) w.sv[nsv + __popc(m & lt)] = e;
    nsv += __popc(m);
    if (nsv >= 32) {
      __syncwarp();
      merge_round(a, ip, w, n, 32, grp, one_group, tests, merges);
      if (lane < nsv - 32) w.sv[lane] = w.sv[32 + lane];
      nsv -= 32;
      __syncwarp();
    }
  }
  __syncwarp();
  if (nsv > 0) merge_round(a, ip, w, n, nsv, grp, one_group, tests, merges);
}

// Splits the n staged hits by cell: group j holds the hits in the cell of the
// j-th hit, in staging order, that no earlier group took.  The group is
// written into bits 16.. of key.w; returns the number of groups.
__device__ __forceinline__ uint32_t assign_groups(const IterParams& ip, MergeWarp& w, int n) {
  const int lane = threadIdx.x & 31;
  uint32_t ngroups = 0;
  while (true) {
    int first = -1;
    for (int g0 = 0; g0 < n && first < 0; g0 += 32) {
      const int g = g0 + lane;
      const bool un = g < n && ((uint32_t)__float_as_int(w.key[g].w) >> 16) == kNoGroup;
      const unsigned m = __ballot_sync(kFull, un);
      if (m) first = g0 + __ffs(m) - 1;
    }
    if (first < 0) break;
    const int3 lc = hit_cell(w.key[first], ip.gmin, ip.cell_inv);
    __syncwarp();
    for (int g = lane; g < n; g += 32) {
      const int kb = __float_as_int(w.key[g].w);
      if (((uint32_t)kb >> 16) != kNoGroup) continue;
      if (same_cell(hit_cell(w.key[g], ip.gmin, ip.cell_inv), lc))
        w.key[g].w = __int_as_float((kb & 0xffff) | (int)(ngroups << 16));
    }
    __syncwarp();
    ++ngroups;
  }
  return ngroups;
}

__global__ void __launch_bounds__(32 * kMergeWarps) k_merge_cells(MergeArgs a, IterParams ip) {
  __shared__ MergeWarp smem[kMergeWarps];
  MergeWarp& w = smem[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < 2 * 32 * 3; i += 32) (&w.acc[0][0][0])[i] = 0.0f;
  uint32_t tests = 0, merges = 0, staged = 0;
  const int nfull = min(a.cnt->mh_tiles, a.cap), npart = min(a.cnt->mh_small, a.cap);
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&a.cnt->mh_next, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= nfull + npart) break;
    const int2 tl = a.tiles[t < nfull ? t : a.cap - 1 - (t - nfull)];
    const int n = tl.y;
    // stage the tile's hits; are they all in the cell of its first hit?
    const int3 c0 = hit_cell(__ldg(&a.mh[__ldg(a.sorted + tl.x)].key), ip.gmin, ip.cell_inv);
    bool same = true;
    for (int g = lane; g < n; g += 32) {
      const int rec = __ldg(a.sorted + tl.x + g);
      float4 k = __ldg(&a.mh[rec].key);
      same = same && same_cell(hit_cell(k, ip.gmin, ip.cell_inv), c0);
      k.w = __int_as_float((__float_as_int(k.w) & 0xffff) | (int)(kNoGroup << 16));
      w.key[g] = k;
      w.dir[g] = __ldg(&a.mh[rec].dir);
      w.phi[g] = __ldg(&a.mh[rec].phi);
    }
    const bool one = __all_sync(kFull, same);
    __syncwarp();
    const uint32_t ng = one ? 1u : assign_groups(ip, w, n);
    for (uint32_t grp = 0; grp < ng; ++grp) merge_group(a, ip, w, n, grp, one, tests, merges);
    staged += lane == 0 ? (uint32_t)n : 0u;
    __syncwarp();
  }
  warp_count(&a.cnt->merge_tests, tests);
  warp_count(&a.cnt->merges, merges);
  warp_count(&a.cnt->merge_hits_staged, staged);
}

static int merge_blocks() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge_cells, 32 * kMergeWarps, 0);
    blocks = (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
  }
  return blocks;
}

cudaError_t merge_staged(neb_ctx* c, const IterParams& ip, const IterSlot& sl, double* accum, double* split,
                         cudaStream_t st, long long* launches) {
  const uint32_t pmask = c->ptable_size - 1;
  const int B = capped_blocks(c->cap_mh, 256, 152 * 8);
  k_mh_count<<<B, 256, 0, st>>>(c->mh, sl.cnt, c->cap_mh, ip.gmin, ip.cell_inv, pmask, c->pb_count);
  cudaError_t e = scan_exclusive(c->pb_count, c->pb_start, (size_t)c->ptable_size + 1, c->scan_scratch, st);
  if (e != cudaSuccess) return e;
  k_mh_scatter<<<B, 256, 0, st>>>(c->mh, sl.cnt, c->cap_mh, ip.gmin, ip.cell_inv, pmask, c->pb_start, c->pb_count,
                                  c->mh_sorted, c->mh_tile);
  MergeArgs a;
  a.mh = c->mh;
  a.sorted = c->mh_sorted;
  a.tiles = c->mh_tile;
  a.mrec = c->mrec;
  a.bucket_start = c->bucket_start;
  a.nv = sl.nv;
  a.mats = c->mats;
  a.accum = accum;
  a.split = split;
  a.cnt = sl.cnt;
  a.cap = c->cap_mh;
  k_merge_cells<<<merge_blocks(), 32 * kMergeWarps, 0, st>>>(a, ip);
  *launches += 3 + scan_launch_count((size_t)c->ptable_size + 1);
  return cudaGetLastError();
}

}  // namespace neb
