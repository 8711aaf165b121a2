// neb_octree.cuh -- device side of the density octree (Sec. 5): the area of
// a plane inside a cell (Eq. area), counting a vertex with splits of full
// cells (lock-free, or in insertion order on one thread for the deterministic
// mode), and the density query (Eq. octdensity) with its robust
// median-of-five form.
//
// Memory layout (Sec. 5.5): one int32 word per cell, the eight children of a
// cell in consecutive words; a word >= 0 is a count, a word < 0 is the
// negated index of the cell's first child.  Word 0 is the root.
//
// Addressing: a position is turned once into its cell on the finest grid the
// tree can reach (2^30 cells per axis of the octree box); the child taken at
// level L is then read from bit 30 - L of each of the three coordinates.  On
// a grid of 2^L cells the cell index of unit coordinate u is floor(u 2^L),
// and scaling by a power of two is exact in FP32, so this is the same cell
// for every level as computing floor(u 2^L) level by level.
#pragma once
#include <climits>

#include "neb_device.cuh"

namespace neb {

constexpr int kOctKeyBits = kOctMaxDepth;  // 30: levels 1..30 below the root

// ---- Eq. area ----------------------------------------------------------------
// Area of the plane through p with unit normal n inside the box [lo, hi]
// (Eq. area, Sec. 5.3; Appendix A obtains it as the derivative of the box
// volume below the plane).  FP64, in a frame where every axis is mirrored so
// that the normal component m_i = |n_i| is non-negative: the corner lowest
// along the normal becomes the origin of the alternating corner sum, with
// a_i = m_i (p_i - that corner's coordinate) and w_i = m_i (hi_i - lo_i), and
// the corner whose upper-bound set is c contributes
// (-1)^|c| max(0, sum_i (a_i - [i in c] w_i))^(d-1), the sum being divided by
// (d-1)! prod m_i.  Mirroring changes the sign of both the corner parity and
// the product of the components, so the quotient is unchanged.  The number of
// axes d follows the FP32 normal as the paper's implementation decides it: a
// component within 1e-3 of +-1 leaves the face across that axis (d = 1), else
// the first component below 1e-4 is dropped and its extent multiplies the
// length found in the other two (d = 2), else d = 3.
__device__ __forceinline__ double plane_box_area64(const double lo[3], const double hi[3], const double p[3],
                                                   const float n[3]) {
  const float m[3] = {fabsf(n[0]), fabsf(n[1]), fabsf(n[2])};
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (fabsf(m[i] - 1.0f) < 1e-3f) {
      const int j = i == 2 ? 0 : i + 1, k = j == 2 ? 0 : j + 1;
      return (hi[j] - lo[j]) * (hi[k] - lo[k]);
    }
  const int drop = m[0] < 1e-4f ? 0 : (m[1] < 1e-4f ? 1 : (m[2] < 1e-4f ? 2 : -1));
  double a[3] = {0.0, 0.0, 0.0}, w[3] = {0.0, 0.0, 0.0}, mprod = 1.0;
  int d = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i == drop) continue;
    const double mi = (double)m[i];
    a[d] = mi * (n[i] >= 0.0f ? p[i] - lo[i] : hi[i] - p[i]);
    w[d] = mi * (hi[i] - lo[i]);
    mprod *= mi;
    ++d;
  }
  const double top = a[0] + a[1] + a[2];
  double sum = 0.0;
  if (d == 3) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double x = top - ((c & 1) ? w[0] : 0.0) - ((c & 2) ? w[1] : 0.0) - ((c & 4) ? w[2] : 0.0);
      const double g = x > 0.0 ? x * x : 0.0;
      sum += (__popc(c) & 1) ? -g : g;
    }
    return fabs(sum) / (2.0 * mprod);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double x = top - ((c & 1) ? w[0] : 0.0) - ((c & 2) ? w[1] : 0.0);
    const double g = x > 0.0 ? x : 0.0;
    sum += (__popc(c) & 1) ? -g : g;
  }
  return (hi[drop] - lo[drop]) * fabs(sum) / mprod;
}

// ---- addressing --------------------------------------------------------------
struct OctKey {
  unsigned x, y, z;  // cell on the 2^30 grid of the octree box
};

// Key of a position; false outside the box.  The box-relative position is
// computed in FP32 (no contraction), as the paper computes it, so that every
// cell decision matches an FP32 evaluation of its formula.
__device__ __forceinline__ bool oct_key(const OctreeParams& P, float px, float py, float pz, OctKey& k) {
  const float u0 = __fmul_rn(__fsub_rn(px, P.minb[0]), P.size_inv[0]);
  const float u1 = __fmul_rn(__fsub_rn(py, P.minb[1]), P.size_inv[1]);
  const float u2 = __fmul_rn(__fsub_rn(pz, P.minb[2]), P.size_inv[2]);
  if (!(u0 >= 0.0f && u0 < 1.0f && u1 >= 0.0f && u1 < 1.0f && u2 >= 0.0f && u2 < 1.0f)) return false;
  const float g = (float)(1u << kOctKeyBits);
  k.x = (unsigned)__fmul_rn(u0, g);
  k.y = (unsigned)__fmul_rn(u1, g);
  k.z = (unsigned)__fmul_rn(u2, g);
  return true;
}

// Child slot (0..7, x + 2y + 4z) taken at level L >= 1 on the way to key k.
__device__ __forceinline__ int oct_octant(const OctKey& k, int L) {
  const int s = kOctKeyBits - L;
  return (int)(((k.x >> s) & 1u) | (((k.y >> s) & 1u) << 1) | (((k.z >> s) & 1u) << 2));
}

// First level at which the paths to keys a and b part (kOctKeyBits + 1 when
// they end in the same finest cell).
__device__ __forceinline__ int oct_parting_level(const OctKey& a, const OctKey& b) {
  const unsigned diff = (a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z);
  return diff ? kOctKeyBits - (31 - __clz(diff)) : kOctKeyBits + 1;
}

// Leaf on the path of key k, found read-only from word `word` (value v) at
// `level`: returns the leaf's word; level and v are updated to the leaf's.
__device__ __forceinline__ int oct_descend(const int* __restrict__ nodes, const OctKey& k, int word, int& level,
                                           int& v) {
  while (v < 0) {
    ++level;
    word = -v + oct_octant(k, level);
    v = __ldg(nodes + word);
  }
  return word;
}

// ---- counting ------------------------------------------------------------------
// A vertex that counted past the threshold of a cell waits for the vertex
// that reached the threshold to publish the cell's child link.  The wait is
// bounded: when it runs out the status bit is set and the vertex stays
// counted in the cell.  Returns the link (< 0), or 0 when no link will come
// (the word pool is exhausted) or the wait ran out.
__device__ __forceinline__ int oct_wait_for_link(const int* word, OctreeState* st, const OctreeParams& P,
                                                 int spin_limit) {
  for (int i = 0; i < spin_limit; ++i) {
    const int v = *((const volatile int*)word);
    if (v < 0) return v;
    if (*((const volatile int*)&st->alloc) > P.capacity) return 0;
    __nanosleep(64);
  }
  atomicOr(&st->status, NEB_STATUS_SPIN_TIMEOUT);
  return 0;
}

// The vertex that brought the cell in `word` (at `level`) to the split
// threshold gives it eight children (Sec. 5.2): it takes the next eight words
// of the pool, which already hold the count a new cell starts with (the
// re-arm kernel writes it into every free word), and publishes the negated
// index of the first in place of the count; it stays counted in the cell it
// split.  With no eight words left the pool is marked exhausted (alloc >
// capacity, status bit) and the cell keeps counting.
template <bool kSequential>
__device__ __forceinline__ void oct_split(int* nodes, OctreeState* st, const OctreeParams& P, int word, int level) {
  if (!kSequential) {
    // Once the pool is used up no cell can split: the many cells that still
    // reach their threshold then take no atomic on the two pool words (one
    // marks the pool exhausted, so vertices waiting for a link stop waiting).
    const int a = *((const volatile int*)&st->alloc);
    if (a + 8 > P.capacity) {
      if (a <= P.capacity) atomicMax(&st->alloc, P.capacity + 1);
      if (!(*((const volatile uint32_t*)&st->status) & NEB_STATUS_OCTREE_FULL))
        atomicOr(&st->status, NEB_STATUS_OCTREE_FULL);
      return;
    }
  }
  const int first = kSequential ? st->alloc : atomicAdd(&st->alloc, 8);
  if (first + 8 > P.capacity) {
    if (kSequential) {
      st->alloc = P.capacity + 1;
      st->status |= NEB_STATUS_OCTREE_FULL;
    } else {
      atomicExch(&st->alloc, P.capacity + 1);
      atomicOr(&st->status, NEB_STATUS_OCTREE_FULL);
    }
    return;
  }
  if (kSequential) {
    st->alloc = first + 8;
    nodes[word] = -first;
    if (level + 1 > st->depth) st->depth = level + 1;
  } else {
    atomicExch(nodes + word, -first);
    atomicMax(&st->depth, level + 1);
  }
}

// Counts one vertex with key k (Sec. 5.1) on one thread, in insertion order
// (the deterministic mode): the count of the leaf cell on its path goes up by
// one; reaching the threshold splits the cell.  Splits stop at level 30.
__device__ __forceinline__ void oct_count_seq(int* nodes, OctreeState* st, const OctreeParams& P, const OctKey& k) {
  int word = 0, level = 0;
  int v = nodes[0];
  while (v < 0) {
    ++level;
    word = -v + oct_octant(k, level);
    v = nodes[word];
  }
  nodes[word] = v + 1;
  if (v + 1 == P.split_count && level < kOctMaxDepth) oct_split<true>(nodes, st, P, word, level);
}

// The same, concurrently (one thread per vertex).  Lanes of a warp that reach
// the same cell together add their vertices with one compare-and-swap by the
// lowest of them, taking no more than the cell still holds below the split
// threshold; the lane whose vertex lands on the threshold splits the cell.
// A vertex that finds a cell at or past the threshold is not counted there
// (that count would be overwritten by the link): it waits for the link and
// counts in the child.  When no link comes (the pool is exhausted, or the
// bounded wait ran out, which sets the status bit) it counts in the cell
// past the threshold.  Each vertex is counted exactly once; a cell that splits
// holds exactly the threshold when its link replaces the count.  Plain reads
// are enough on the way down: a link never changes once published, and a
// stale count only makes the compare-and-swap fail and return the word's
// current value.
//
// kDefer: a vertex that finds the pool exhausted before it is counted returns
// false instead, and the caller counts it after the launch, when every link
// of the launch is published and the tree can no longer change (a read-only
// descent and an add): once the pool runs out, most vertices meet full cells
// and would otherwise all count past the threshold through contended
// compare-and-swaps.  Returns true when the vertex was counted.
template <bool kDefer>
__device__ __forceinline__ bool oct_count(int* nodes, OctreeState* st, const OctreeParams& P, const OctKey& k,
                                          int spin_limit) {
  if (kDefer && *((const volatile int*)&st->alloc) > P.capacity) return false;
  const int lane = threadIdx.x & 31;
  int word = 0, level = 0;
  bool past = false;  // counting past the threshold of this cell is allowed
  int v = nodes[0];
  while (true) {
    if (v < 0) {
      ++level;
      word = -v + oct_octant(k, level);
      v = nodes[word];
      past = false;
      continue;
    }
    const int limit = (past || level >= kOctMaxDepth) ? INT_MAX : P.split_count;
    if (v >= limit) {
      v = oct_wait_for_link(nodes + word, st, P, spin_limit);
      if (v >= 0) {
        if (kDefer && *((const volatile int*)&st->alloc) > P.capacity) return false;
        past = true;
        v = nodes[word];
      }
      continue;
    }
    // one compare-and-swap per group of lanes at the same cell
    const unsigned grp = __match_any_sync(__activemask(), word);
    const int leader = __ffs(grp) - 1;
    const int n = __popc(grp), rank = __popc(grp & ((1u << lane) - 1u));
    int base = 0, got = 0;
    if (lane == leader) {
      int cur = v;
      while (true) {
        if (cur < 0 || cur >= limit) {  // now a link, or full: nobody counts here
          base = cur;
          break;
        }
        const int take = min(n, limit - cur);
        const int seen = atomicCAS(nodes + word, cur, cur + take);
        if (seen == cur) {
          base = cur;
          got = take;
          break;
        }
        cur = seen;
      }
    }
    base = __shfl_sync(grp, base, leader);
    got = __shfl_sync(grp, got, leader);
    if (rank < got) {
      if (limit == P.split_count && base + rank + 1 == limit) oct_split<false>(nodes, st, P, word, level);
      return true;
    }
    v = got > 0 ? base + got : base;  // the word as the group left it
  }
}

// Concurrent insert of one vertex; false when it was deferred (kDefer).
template <bool kDefer>
__device__ __forceinline__ bool oct_insert(int* nodes, OctreeState* st, const OctreeParams& P, const float pos[3],
                                           int spin_limit) {
  if (P.stop_filling) return true;
  OctKey k;
  if (oct_key(P, pos[0], pos[1], pos[2], k)) return oct_count<kDefer>(nodes, st, P, k, spin_limit);
  return true;
}

__device__ __forceinline__ void oct_insert_seq(int* nodes, OctreeState* st, const OctreeParams& P,
                                               const float pos[3]) {
  if (P.stop_filling) return;
  OctKey k;
  if (oct_key(P, pos[0], pos[1], pos[2], k)) oct_count_seq(nodes, st, P, k);
}

// Leaf word of a position once no cell can split any more (the pool was
// exhausted before this launch): a read-only descent; -1 outside the box.
__device__ __forceinline__ int oct_frozen_leaf(const int* nodes, const OctreeParams& P, const float pos[3]) {
  if (P.stop_filling) return -1;
  OctKey k;
  if (!oct_key(P, pos[0], pos[1], pos[2], k)) return -1;
  int level = 0, v = nodes[0];
  int word = 0;
  while (v < 0) {
    ++level;
    word = -v + oct_octant(k, level);
    v = nodes[word];
  }
  return word;
}

// ---- density -------------------------------------------------------------------
// Density of a leaf with count c > 0 at `level` on the path of key k, for the
// plane through pos with normal n (Eq. octdensity): c over the number of
// iterations and over the plane's area in the cell, the area held above a
// fraction of the squared cell diagonal (0.1 of it for the centre query of
// the robust estimate, 0.01 otherwise).  The cell box and the point are
// taken relative to the octree box's lower corner, in FP64, and the quotient
// is rounded to FP32.
__device__ __forceinline__ float oct_leaf_density(const OctreeParams& P, int c, int level, const OctKey& k,
                                                  const float pos[3], const float n[3], bool centre) {
  const int s = kOctKeyBits - level;
  const unsigned cell[3] = {k.x >> s, k.y >> s, k.z >> s};
  double lo[3], hi[3], p[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double extent = ldexp(P.box_extent[a], -level);
    lo[a] = (double)cell[a] * extent;
    hi[a] = lo[a] + extent;
    p[a] = (double)pos[a] - (double)P.minb[a];
  }
  const double area = plane_box_area64(lo, hi, p, n);
  const double diag = ldexp((double)P.scene_scale, -level);
  const double floor_area = diag * diag * (centre ? 0.1 : 0.01);
  return (float)((double)c / ((double)P.iter_clamp * (area > floor_area ? area : floor_area)));
}

// Single density query; 0 for an empty cell or a point outside the box.
__device__ __forceinline__ float oct_density(const int* __restrict__ nodes, const OctreeParams& P, const float pos[3],
                                             const float n[3]) {
  OctKey k;
  if (!oct_key(P, pos[0], pos[1], pos[2], k)) return 0.0f;
  int level = 0, v = __ldg(nodes);
  oct_descend(nodes, k, 0, level, v);
  return v > 0 ? oct_leaf_density(P, v, level, k, pos, n, false) : 0.0f;
}

// Robust density: the centre query and four queries at 1.1 cell diagonals
// from the point along the two tangents of the Duff et al. basis of the
// geometric normal; the result is the median of the positive ones, the upper
// of the middle two for an even number, 0 when none is positive.  The step
// and the displaced points are FP32 (no contraction), as the paper computes
// them; the step is 1.1e-3 when the centre cell is empty.  A displaced query
// runs through the same words as the centre query down to the level where
// their paths part, so it resumes from the centre's path there.
__device__ __forceinline__ float oct_density_robust(const int* __restrict__ nodes, const OctreeParams& P,
                                                    const float pos[3], const float n[3], int* queries) {
  float found[5];
  int nfound = 0;
  float step = 1e-3f;
  // centre query, remembering the word value at every level of its path
  int path[kOctMaxDepth + 1];
  OctKey kc;
  int centre_level = -1;
  if (oct_key(P, pos[0], pos[1], pos[2], kc)) {
    int level = 0, v = __ldg(nodes);
    path[0] = v;
    while (v < 0) {
      ++level;
      v = __ldg(nodes + (-v + oct_octant(kc, level)));
      path[level] = v;
    }
    centre_level = level;
    if (v > 0) {
      found[nfound++] = oct_leaf_density(P, v, level, kc, pos, n, true);
      step = ldexpf(P.scene_scale, -level);
    }
  }
  step = __fmul_rn(step, 1.1f);
  float3 t, b;
  onb(f3(n[0], n[1], n[2]), t, b);
  const float dx[4] = {t.x, -t.x, b.x, -b.x}, dy[4] = {t.y, -t.y, b.y, -b.y}, dz[4] = {t.z, -t.z, b.z, -b.z};
  // the four displaced walks step down together: each step issues up to four
  // independent loads instead of one chain at a time
  float q[4][3];
  OctKey kq[4];
  int vq[4], lq[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    q[i][0] = __fadd_rn(pos[0], __fmul_rn(dx[i], step));
    q[i][1] = __fadd_rn(pos[1], __fmul_rn(dy[i], step));
    q[i][2] = __fadd_rn(pos[2], __fmul_rn(dz[i], step));
    vq[i] = 0;  // outside the box: no walk, nothing found
    lq[i] = 0;
    if (oct_key(P, q[i][0], q[i][1], q[i][2], kq[i])) {
      if (centre_level >= 0) {
        const int part = oct_parting_level(kc, kq[i]);
        lq[i] = part - 1 < centre_level ? part - 1 : centre_level;
        vq[i] = path[lq[i]];
      } else {
        vq[i] = __ldg(nodes);
      }
    }
  }
  while (vq[0] < 0 || vq[1] < 0 || vq[2] < 0 || vq[3] < 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (vq[i] < 0) {
        ++lq[i];
        vq[i] = __ldg(nodes + (-vq[i] + oct_octant(kq[i], lq[i])));
      }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (vq[i] > 0) {
      const float r = oct_leaf_density(P, vq[i], lq[i], kq[i], q[i], n, false);
      if (r > 0.0f) found[nfound++] = r;
    }
  *queries += 5;
  if (nfound == 0) return 0.0f;
  // insertion sort of at most five values, then the upper median
  for (int i = 1; i < nfound; ++i) {
    const float x = found[i];
    int j = i - 1;
    while (j >= 0 && found[j] > x) {
      found[j + 1] = found[j];
      --j;
    }
    found[j + 1] = x;
  }
  return found[nfound / 2];
}

}  // namespace neb
