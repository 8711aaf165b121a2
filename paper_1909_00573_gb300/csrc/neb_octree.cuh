// neb_octree.cuh -- device side of the density octree (Sec. 5 and the
// listing of Appendix B): plane/box area (Eq. area), count-and-split insert
// (lock-free, and sequential for the deterministic mode), and the density
// query with its robust median-of-five variant.
#pragma once
#include "neb_device.cuh"

namespace neb {

// Eq. area with the listing's 1D (|n_d| within 1e-3 of 1) and 2D (|n_d| <
// 1e-4) cases; corners enter the alternating sum in the listing's order.
__host__ __device__ __forceinline__ float intersection_area(const float bmin[3], const float bmax[3],
                                                            const float pos[3], const float n[3]) {
  float cs[3] = {bmax[0] - bmin[0], bmax[1] - bmin[1], bmax[2] - bmin[2]};
  float an[3] = {fabsf(n[0]), fabsf(n[1]), fabsf(n[2])};
  if (fabsf(an[0] - 1.0f) < 1e-3f) return cs[1] * cs[2];
  if (fabsf(an[1] - 1.0f) < 1e-3f) return cs[0] * cs[2];
  if (fabsf(an[2] - 1.0f) < 1e-3f) return cs[0] * cs[1];
  for (int d = 0; d < 3; ++d) {
    if (an[d] < 1e-4f) {
      int x = d == 2 ? 0 : d + 1;
      int y = x == 2 ? 0 : x + 1;
      float h = n[x] * pos[x] + n[y] * pos[y];
      float s = 0.0f;
      s += fmaxf(0.0f, h - (n[x] * bmin[x] + n[y] * bmin[y]));
      s -= fmaxf(0.0f, h - (n[x] * bmin[x] + n[y] * bmax[y]));
      s -= fmaxf(0.0f, h - (n[x] * bmax[x] + n[y] * bmin[y]));
      s += fmaxf(0.0f, h - (n[x] * bmax[x] + n[y] * bmax[y]));
      return cs[d] * fabsf(s / (n[x] * n[y]));
    }
  }
  float h = n[0] * pos[0] + n[1] * pos[1] + n[2] * pos[2];
  float s = 0.0f, t;
  t = fmaxf(0.0f, h - (n[0] * bmin[0] + n[1] * bmin[1] + n[2] * bmin[2])); s += t * t;
  t = fmaxf(0.0f, h - (n[0] * bmin[0] + n[1] * bmin[1] + n[2] * bmax[2])); s -= t * t;
  t = fmaxf(0.0f, h - (n[0] * bmin[0] + n[1] * bmax[1] + n[2] * bmax[2])); s += t * t;
  t = fmaxf(0.0f, h - (n[0] * bmin[0] + n[1] * bmax[1] + n[2] * bmin[2])); s -= t * t;
  t = fmaxf(0.0f, h - (n[0] * bmax[0] + n[1] * bmax[1] + n[2] * bmin[2])); s += t * t;
  t = fmaxf(0.0f, h - (n[0] * bmax[0] + n[1] * bmin[1] + n[2] * bmin[2])); s -= t * t;
  t = fmaxf(0.0f, h - (n[0] * bmax[0] + n[1] * bmin[1] + n[2] * bmax[2])); s += t * t;
  t = fmaxf(0.0f, h - (n[0] * bmax[0] + n[1] * bmax[1] + n[2] * bmax[2])); s -= t * t;
  return fabsf(s / (2.0f * n[0] * n[1] * n[2]));
}

__device__ __forceinline__ bool oct_norm_pos(const OctreeParams& P, const float pos[3], float np[3]) {
  for (int c = 0; c < 3; ++c) np[c] = (pos[c] - P.minb[c]) * P.size_inv[c];
  for (int c = 0; c < 3; ++c)
    if (!(np[c] >= 0.0f && np[c] < 1.0f)) return false;
  return true;
}

// ---- insert ---------------------------------------------------------------
// Sequential form (one device thread): identical to the listing run by one
// CPU thread.
__device__ __forceinline__ int oct_split_seq(int* nodes, OctreeState* st, const OctreeParams& P, int idx, int count,
                                             int depth) {
  if (count >= P.split_count) {
    if (depth + 1 > kOctMaxDepth) return 0;
    if (count == P.split_count) {
      int child = st->alloc;
      st->alloc += 8;
      if (child >= P.capacity) {
        st->alloc = P.capacity + 1;
        st->status |= NEB_STATUS_OCTREE_FULL;
        return 0;
      }
      nodes[idx] = -child;
      if (depth + 1 > st->depth) st->depth = depth + 1;
      return 0;
    }
    return nodes[idx] < 0 ? nodes[idx] : 0;
  }
  return count;
}

__device__ __forceinline__ void oct_insert_seq(int* nodes, OctreeState* st, const OctreeParams& P,
                                               const float pos[3]) {
  if (P.stop_filling) return;
  float np[3];
  if (!oct_norm_pos(P, pos, np)) return;
  int v = nodes[0];
  if (v >= 0) nodes[0] = ++v;
  v = oct_split_seq(nodes, st, P, 0, v, 0);
  int edge = 1, depth = 0;
  while (v < 0) {
    edge *= 2;
    ++depth;
    int ix = ((int)(np[0] * (float)edge)) & 1;
    int iy = ((int)(np[1] * (float)edge)) & 1;
    int iz = ((int)(np[2] * (float)edge)) & 1;
    int idx = ix + 2 * (iy + 2 * iz) - v;
    v = nodes[idx];
    if (v >= 0) nodes[idx] = ++v;
    v = oct_split_seq(nodes, st, P, idx, v, depth);
  }
}

// Lock-free form: CAS increment of a non-negative counter
// (increment_if_positive), one thread per split (the one that reaches the
// threshold exactly), the others wait for the child pointer with a bounded
// spin and then count in the child.  A spin that runs out sets
// NEB_STATUS_SPIN_TIMEOUT and drops the insert; it never traps.
__device__ __forceinline__ int oct_inc_atomic(int* nodes, int idx, bool frozen) {
  // A plain (cacheable) first read is enough: a child pointer never changes
  // once published, and a stale counter only makes the CAS below fail and
  // return the current value.
  int old = nodes[idx];
  // frozen: the allocation overflowed before this kernel started, so no
  // counter can turn into a child pointer any more and a plain atomic add is
  // the same increment without CAS retries on crowded leaves
  if (frozen && old >= 0) return atomicAdd(nodes + idx, 1) + 1;
  while (true) {
    if (old < 0) return old;
    int prev = atomicCAS(nodes + idx, old, old + 1);
    if (prev == old) return old + 1;
    old = prev;
  }
}

__device__ __forceinline__ int oct_split_atomic(int* nodes, OctreeState* st, const OctreeParams& P, int idx,
                                                int count, int depth, int spin_limit) {
  if (count >= P.split_count) {
    if (depth + 1 > kOctMaxDepth) return 0;
    if (count == P.split_count) {
      int child = atomicAdd(&st->alloc, 8);
      if (child >= P.capacity) {
        atomicExch(&st->alloc, P.capacity + 1);
        atomicOr(&st->status, NEB_STATUS_OCTREE_FULL);
        return 0;
      }
      atomicExch(nodes + idx, -child);
      atomicMax(&st->depth, depth + 1);
      return 0;
    }
    for (int it = 0; it < spin_limit; ++it) {
      int c = *((volatile int*)(nodes + idx));
      if (c < 0) return c;
      if (*((volatile int*)&st->alloc) > P.capacity) return 0;
      __nanosleep(64);
    }
    atomicOr(&st->status, NEB_STATUS_SPIN_TIMEOUT);
    return 0;
  }
  return count;
}

__device__ __forceinline__ void oct_insert_atomic(int* nodes, OctreeState* st, const OctreeParams& P,
                                                  const float pos[3], int spin_limit, bool frozen) {
  if (P.stop_filling) return;
  float np[3];
  if (!oct_norm_pos(P, pos, np)) return;
  int v = oct_inc_atomic(nodes, 0, frozen);
  v = oct_split_atomic(nodes, st, P, 0, v, 0, spin_limit);
  int edge = 1, depth = 0;
  while (v < 0) {
    edge *= 2;
    ++depth;
    int ix = ((int)(np[0] * (float)edge)) & 1;
    int iy = ((int)(np[1] * (float)edge)) & 1;
    int iz = ((int)(np[2] * (float)edge)) & 1;
    int idx = ix + 2 * (iy + 2 * iz) - v;
    v = oct_inc_atomic(nodes, idx, frozen);
    v = oct_split_atomic(nodes, st, P, idx, v, depth, spin_limit);
  }
}

// Leaf reached by a position once the octree can no longer split (allocation
// overflowed): a read-only descent; -1 for positions outside the box.
__device__ __forceinline__ int oct_frozen_leaf(const int* nodes, const OctreeParams& P, const float pos[3]) {
  if (P.stop_filling) return -1;
  float np[3];
  if (!oct_norm_pos(P, pos, np)) return -1;
  int idx = 0;
  int v = nodes[0];
  int edge = 1;
  while (v < 0) {
    edge *= 2;
    int ix = ((int)(np[0] * (float)edge)) & 1;
    int iy = ((int)(np[1] * (float)edge)) & 1;
    int iz = ((int)(np[2] * (float)edge)) & 1;
    idx = ix + 2 * (iy + 2 * iz) - v;
    v = nodes[idx];
  }
  return idx;
}

// ---- query -----------------------------------------------------------------
// get_density of the listing with the final normalisation in FP64:
// rho = c / (min(iter, 1000) * max(minArea, A)).  *size receives the cell
// diagonal when non-null (robust centre query: minArea uses 0.1 instead of 0.01).
__device__ __forceinline__ float oct_density(const int* __restrict__ nodes, const OctreeParams& P, int depth,
                                             const float pos[3], const float n[3], float* size) {
  float off[3], np[3];
  for (int c = 0; c < 3; ++c) {
    off[c] = pos[c] - P.minb[c];
    np[c] = off[c] * P.size_inv[c];
  }
  for (int c = 0; c < 3; ++c)
    if (!(np[c] >= 0.0f && np[c] < 1.0f)) return 0.0f;
  int grid = 1 << depth;
  int ip[3];
  for (int c = 0; c < 3; ++c) ip[c] = (int)(np[c] * (float)grid);
  int v = __ldg(nodes);
  int mask = grid;
  while (v < 0) {
    mask >>= 1;
    int idx = ((ip[0] & mask) ? 1 : 0) + ((ip[1] & mask) ? 2 : 0) + ((ip[2] & mask) ? 4 : 0);
    idx -= v;
    v = __ldg(nodes + idx);
  }
  if (v > 0) {
    int cur = grid / mask;
    float cmin[3], cmax[3];
    for (int c = 0; c < 3; ++c) {
      float csz = 1.0f / ((float)cur * P.size_inv[c]);
      int cp = ip[c] / mask;
      cmin[c] = (float)cp * csz;
      cmax[c] = cmin[c] + csz;
    }
    float area = intersection_area(cmin, cmax, off, n);
    float diag = P.scene_scale / (float)cur;
    float min_area = diag * diag;
    if (size) { *size = diag; min_area *= 0.1f; } else min_area *= 0.01f;
    double rho = (double)v / ((double)P.iter_clamp * (double)fmaxf(min_area, area));
    return (float)rho;
  }
  return 0.0f;
}

// Cell of the leaf (v, mask) reached by a query with integer position ip,
// offset position off and normal n: returns the count v (0 when empty) and
// the area denominator max(minArea, A) of get_density's quotient.
__device__ __forceinline__ int oct_leaf_terms(const OctreeParams& P, int grid, int mask, int v, const int ip[3],
                                              const float off[3], const float n[3], float* size, float& denom) {
  denom = 1.0f;
  if (v <= 0) return 0;
  int cur = grid / mask;
  float cmin[3], cmax[3];
  for (int c = 0; c < 3; ++c) {
    float csz = 1.0f / ((float)cur * P.size_inv[c]);
    int cp = ip[c] / mask;
    cmin[c] = (float)cp * csz;
    cmax[c] = cmin[c] + csz;
  }
  float area = intersection_area(cmin, cmax, off, n);
  float diag = P.scene_scale / (float)cur;
  float min_area = diag * diag;
  if (size) { *size = diag; min_area *= 0.1f; } else min_area *= 0.01f;
  denom = fmaxf(min_area, area);
  return v;
}

// The listing's quotient with its normalisation in FP64, rounded to FP32.
__device__ __forceinline__ float oct_rho(int v, int iter_clamp, float denom) {
  if (v <= 0) return 0.0f;
  return (float)((double)v / ((double)iter_clamp * (double)denom));
}

// get_density_robust of the listing: median of the centre query and four
// queries displaced by 1.1 cell diagonals along the tangents of the Duff et
// al. basis of the geometric normal; ties go to the greater value.  A
// displaced query walks the same nodes as the centre one down to the first
// level where its cell coordinates differ, so it resumes from the centre's
// recorded path there instead of at the root (same nodes, same result).
__device__ __forceinline__ float oct_density_robust(const int* __restrict__ nodes, const OctreeParams& P, int depth,
                                                    const float pos[3], const float n[3], int* queries) {
  int cv[5] = {0, 0, 0, 0, 0};     // leaf counts of the five queries
  float cd[5] = {1, 1, 1, 1, 1};   // their area denominators
  float diag = 1e-3f;
  const int grid = 1 << depth;
  // centre query with its path: vs[L] = node value at level L
  int vs[kOctMaxDepth + 2];
  int ipc[3];
  int Lc = -1;
  {
    float off[3], np[3];
    bool in = true;
    for (int c = 0; c < 3; ++c) {
      off[c] = pos[c] - P.minb[c];
      np[c] = off[c] * P.size_inv[c];
      in = in && (np[c] >= 0.0f && np[c] < 1.0f);
    }
    if (in) {
      for (int c = 0; c < 3; ++c) ipc[c] = (int)(np[c] * (float)grid);
      int v = __ldg(nodes);
      int mask = grid;
      int L = 0;
      vs[0] = v;
      while (v < 0) {
        mask >>= 1;
        int idx = ((ipc[0] & mask) ? 1 : 0) + ((ipc[1] & mask) ? 2 : 0) + ((ipc[2] & mask) ? 4 : 0);
        idx -= v;
        v = __ldg(nodes + idx);
        vs[++L] = v;
      }
      Lc = L;
      cv[0] = oct_leaf_terms(P, grid, mask, v, ipc, off, n, &diag, cd[0]);
    }
  }
  diag *= 1.1f;
  float3 t, b;
  onb(f3(n[0], n[1], n[2]), t, b);
  float3 p = f3(pos[0], pos[1], pos[2]);
  float3 q[4] = {add(p, mul(t, diag)), sub(p, mul(t, diag)), add(p, mul(b, diag)), sub(p, mul(b, diag))};
  // The four displaced walks are independent: they step down together, so
  // each step issues up to four loads at once instead of one chain at a time.
  int v4[4], m4[4], ip4[4][3];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float qq[3] = {q[i].x, q[i].y, q[i].z};
    bool in = true;
    for (int c = 0; c < 3; ++c) {
      float np = (qq[c] - P.minb[c]) * P.size_inv[c];
      in = in && (np >= 0.0f && np < 1.0f);
      ip4[i][c] = in ? (int)(np * (float)grid) : 0;
    }
    v4[i] = 0;  // outside the scene box: no walk, count 0
    m4[i] = grid;
    if (in) {
      if (Lc >= 0) {
        unsigned diff = (unsigned)((ip4[i][0] ^ ipc[0]) | (ip4[i][1] ^ ipc[1]) | (ip4[i][2] ^ ipc[2]));
        // first level whose octant differs: mask (grid >> L) equals the top differing bit
        int Ld = diff ? depth - (31 - __clz(diff)) : depth + 1;
        int L = Ld - 1 < Lc ? Ld - 1 : Lc;
        v4[i] = vs[L];
        m4[i] = grid >> L;
      } else {
        v4[i] = __ldg(nodes);
      }
    }
  }
  while (v4[0] < 0 || v4[1] < 0 || v4[2] < 0 || v4[3] < 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (v4[i] < 0) {
        m4[i] >>= 1;
        int mk = m4[i];
        int idx = ((ip4[i][0] & mk) ? 1 : 0) + ((ip4[i][1] & mk) ? 2 : 0) + ((ip4[i][2] & mk) ? 4 : 0);
        v4[i] = __ldg(nodes + (idx - v4[i]));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (v4[i] > 0) {
      float qq[3] = {q[i].x, q[i].y, q[i].z};
      float off[3];
      for (int c = 0; c < 3; ++c) off[c] = qq[c] - P.minb[c];
      cv[i + 1] = oct_leaf_terms(P, grid, m4[i], v4[i], ip4[i], off, n, nullptr, cd[i + 1]);
    }
  }
  *queries += 5;
  // Median of the positive results, ties to the greater: the listing's partial
  // selection sort over the FP64 quotients rounded to FP32.
  float d[5];
  int count = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
    if (cv[i] > 0) d[count++] = oct_rho(cv[i], P.iter_clamp, cd[i]);
  if (count == 0) return 0.0f;
  const int m = count / 2;
  for (int i = 0; i <= m; ++i)
    for (int j = i + 1; j < count; ++j)
      if (d[j] < d[i]) { float tmp = d[i]; d[i] = d[j]; d[j] = tmp; }
  return d[m];
}

}  // namespace neb
