// neb_density.cu -- the density estimators of Sec. 5 side by side on the
// device: the density octree the pass uses, the naive fixed-radius estimator
// (the paper's first approach, a hash grid) and the k-nearest-neighbour
// estimator (its second approach, a kd-tree; here a 4-wide tree over the
// points plays the kd-tree's role).  Each estimates, at every point of a
// set inserted as one iteration, the number of points per unit area.
#include <cfloat>
#include <cstring>
#include <vector>

#include "neb_device.cuh"
#include "neb_internal.h"

namespace neb {

constexpr int kMaxK = 16;
constexpr double kPiD = 3.14159265358979323846;

__global__ void k_pack_points(const float* __restrict__ pos, int n, float4* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], 0.0f);
}

// Naive estimator: the points within distance h of point i (i included),
// through the hashed grid of cell size 2h (8 cells cover the ball), divided
// by pi h^2 (FP64, rounded to FP32).
__global__ void k_naive_rho(const float4* __restrict__ sorted, const int* __restrict__ bucket_start,
                            const float* __restrict__ pos, int n, float h2, float3 gmin, float cell_inv,
                            uint32_t mask, double inv_area, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float3 p = f3(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]);
    float gx = (p.x - gmin.x) * cell_inv, gy = (p.y - gmin.y) * cell_inv, gz = (p.z - gmin.z) * cell_inv;
    int cx = grid_cell_index(gx), cy = grid_cell_index(gy), cz = grid_cell_index(gz);
    int ox = (gx - (float)cx >= 0.5f) ? 1 : -1, oy = (gy - (float)cy >= 0.5f) ? 1 : -1,
        oz = (gz - (float)cz >= 0.5f) ? 1 : -1;
    uint32_t bk[8];
    for (int c = 0; c < 8; ++c)
      bk[c] = grid_hash(cx + ((c & 1) ? ox : 0), cy + ((c & 2) ? oy : 0), cz + ((c & 4) ? oz : 0), mask);
    int cnt = 0;
    for (int c = 0; c < 8; ++c) {
      bool dup = false;
      for (int c2 = 0; c2 < c; ++c2) dup |= bk[c2] == bk[c];
      if (dup) continue;
      for (int e = __ldg(bucket_start + bk[c]); e < __ldg(bucket_start + bk[c] + 1); ++e) {
        float4 q = __ldg(sorted + e);
        float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
        if (dx * dx + dy * dy + dz * dz <= h2) ++cnt;
      }
    }
    out[i] = (float)((double)cnt * inv_area);
  }
}

// k-nearest-neighbour estimator (Loftsgaarden and Quesenberry 1965, in the
// plane of the surface): rho = (k - 1) / (pi d_k^2), d_k the distance from
// point i to its k-th nearest other point, found by a branch-and-bound walk of
// the 4-wide tree over the points (children nearer than the current k-th
// distance are visited near first; leaves are points).  0 when the set has
// fewer than k other points.
__device__ __forceinline__ float box_dist2(float3 p, float lx, float hx, float ly, float hy, float lz, float hz) {
  float dx = fmaxf(fmaxf(lx - p.x, p.x - hx), 0.0f);
  float dy = fmaxf(fmaxf(ly - p.y, p.y - hy), 0.0f);
  float dz = fmaxf(fmaxf(lz - p.z, p.z - hz), 0.0f);
  return dx * dx + dy * dy + dz * dz;
}

__global__ void k_knn_rho(const BVH4Node* __restrict__ nodes, const float4* __restrict__ pts, int n, int k,
                          float* __restrict__ out, uint32_t* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float3 p = xyz(__ldg(pts + i));
    float best[kMaxK];
    for (int j = 0; j < kMaxK; ++j) best[j] = FLT_MAX;
    // a 4-wide walk pushes up to 3 subtrees per level, and a tree over
    // clustered points is deep
    constexpr int kStack = 256;
    int stack[kStack];
    float sdist[kStack];
    int sp = 0, node = 0;
    while (true) {
      if (node >= 0) {
        const float4* np = reinterpret_cast<const float4*>(nodes + node);
        float4 lx = __ldg(np), hx = __ldg(np + 1), ly = __ldg(np + 2), hy = __ldg(np + 3), lz = __ldg(np + 4),
               hz = __ldg(np + 5);
        int4 ch = __ldg(reinterpret_cast<const int4*>(np + 6));
        int cr[4];
        float cd[4];
        int cnt = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          int ref = comp4i(ch, c);
          if (ref == kEmptyChild) continue;
          if (ref < 0) {
            int j = ~ref;
            if (j == i) continue;
            float4 q = __ldg(pts + j);
            float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
            float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < best[k - 1]) {  // insert into the sorted k best
              int at = k - 1;
              while (at > 0 && best[at - 1] > d2) {
                best[at] = best[at - 1];
                --at;
              }
              best[at] = d2;
            }
            continue;
          }
          float d2 = box_dist2(p, comp4(lx, c), comp4(hx, c), comp4(ly, c), comp4(hy, c), comp4(lz, c), comp4(hz, c));
          if (d2 >= best[k - 1]) continue;
          cr[cnt] = ref;
          cd[cnt] = d2;
          ++cnt;
        }
        // visit the nearest child next, push the others far to near
        for (int a = 1; a < cnt; ++a) {
          float tv = cd[a];
          int rv = cr[a];
          int b = a - 1;
          while (b >= 0 && cd[b] > tv) {
            cd[b + 1] = cd[b];
            cr[b + 1] = cr[b];
            --b;
          }
          cd[b + 1] = tv;
          cr[b + 1] = rv;
        }
        for (int a = cnt - 1; a >= 1; --a) {
          if (sp < kStack) {
            stack[sp] = cr[a];
            sdist[sp] = cd[a];
            ++sp;
          } else {
            atomicOr(status, NEB_STATUS_STACK_OVERFLOW);
          }
        }
        node = cnt > 0 ? cr[0] : -1;
        continue;
      }
      // pop the next subtree that can still hold a nearer point
      node = -1;
      while (sp > 0) {
        --sp;
        if (sdist[sp] < best[k - 1]) {
          node = stack[sp];
          break;
        }
      }
      if (node < 0) break;
    }
    float dk = best[k - 1];
    out[i] = dk < FLT_MAX ? (float)((double)(k - 1) / (kPiD * (double)dk)) : 0.0f;
  }
}

}  // namespace neb

using namespace neb;

extern "C" int neb_density_estimators(const float* pos, const float* nrm, int n, const float scene_min[3],
                                      const float scene_max[3], int octree_capacity, int split_factor, float radius,
                                      int k, float* rho, double* ms) {
  if (!pos || !nrm || !scene_min || !scene_max || !rho || n < 1 || octree_capacity < 1 || split_factor < 2 ||
      !(radius > 0.0f) || k < 2 || k > kMaxK)
    return NEB_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return NEB_ERR_NO_DEVICE;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return NEB_ERR_CUDA;
  const size_t bytes3 = sizeof(float) * 3 * (size_t)n;
  OctreeParams P = octree_params(scene_min, scene_max, octree_capacity, split_factor);
  octree_set_iteration_params(P, split_factor, 1);
  uint32_t table = 1024;
  while (table < (uint32_t)(2 * n)) table <<= 1;
  Scratch sc;
  sc.n = scan_scratch_ints((size_t)table + 1);
  float *d_pos = nullptr, *d_nrm = nullptr, *d_out = nullptr;
  float4 *d_pts4 = nullptr, *d_sorted = nullptr;
  int *d_nodes = nullptr, *bc = nullptr, *bs = nullptr, *vb = nullptr;
  OctreeState* d_st = nullptr;
  uint32_t* d_status = nullptr;
  BVH4Node* tree = nullptr;
  bool ok = cudaMalloc(&d_pos, bytes3) == cudaSuccess && cudaMalloc(&d_nrm, bytes3) == cudaSuccess &&
            cudaMalloc(&d_out, sizeof(float) * 3 * (size_t)n) == cudaSuccess &&
            cudaMalloc(&d_pts4, sizeof(float4) * (size_t)n) == cudaSuccess &&
            cudaMalloc(&d_sorted, sizeof(float4) * (size_t)n) == cudaSuccess &&
            cudaMalloc(&d_nodes, sizeof(int) * (size_t)P.capacity) == cudaSuccess &&
            cudaMalloc(&d_st, sizeof(OctreeState)) == cudaSuccess &&
            cudaMalloc(&bc, sizeof(int) * ((size_t)table + 1)) == cudaSuccess &&
            cudaMalloc(&bs, sizeof(int) * ((size_t)table + 1)) == cudaSuccess &&
            cudaMalloc(&vb, sizeof(int) * (size_t)n) == cudaSuccess &&
            cudaMalloc(&sc.data, sizeof(int) * sc.n) == cudaSuccess &&
            cudaMalloc(&d_status, sizeof(uint32_t)) == cudaSuccess;
  cudaEvent_t ev[6] = {};
  for (auto& e : ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  int rc = ok ? NEB_OK : NEB_ERR_OOM;
  if (ok) {
    cudaMemcpyAsync(d_pos, pos, bytes3, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_nrm, nrm, bytes3, cudaMemcpyHostToDevice, st);
    OctreeState s0{1, 0, 0u, 0};
    cudaMemsetAsync(d_nodes, 0, sizeof(int) * (size_t)P.capacity, st);
    cudaMemcpyAsync(d_st, &s0, sizeof(s0), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(bc, 0, sizeof(int) * ((size_t)table + 1), st);
    cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st);
    // (0) the density octree, as one iteration of the pass uses it
    cudaEventRecord(ev[0], st);
    launch_oct_rearm(d_nodes, d_st, P, st);
    launch_oct_insert_points(d_nodes, d_st, P, d_pos, n, 0, st);
    launch_oct_density_points(d_nodes, d_st, P, d_pos, d_nrm, n, 1, d_out, st);
    cudaEventRecord(ev[1], st);
    // (1) naive estimator through the hashed grid
    cudaEventRecord(ev[2], st);
    const float cs = 2.0f * radius;
    const float3 gmin = f3(scene_min[0], scene_min[1], scene_min[2]);
    const int nb = capped_blocks(n, 256, 152 * 8);
    build_point_grid(d_pos, n, cs, gmin, table, bc, bs, vb, d_sorted, sc, st);
    k_naive_rho<<<nb, 256, 0, st>>>(d_sorted, bs, d_pos, n, radius * radius, gmin, 1.0f / cs, table - 1,
                                    1.0 / (kPiD * (double)radius * (double)radius), d_out + n);
    cudaEventRecord(ev[3], st);
    // (2) k-nearest neighbours through a 4-wide tree over the points
    cudaEventRecord(ev[4], st);
    k_pack_points<<<nb, 256, 0, st>>>(d_pos, n, d_pts4);
    SceneView sv;
    memset(&sv, 0, sizeof(sv));
    sv.sph = d_pts4;
    sv.ns = n;
    int n4 = 0;
    cudaError_t e = build_bvh4(sv, n, 0, st, &tree, &n4);
    if (e == cudaSuccess) {
      k_knn_rho<<<nb, 256, 0, st>>>(tree, d_pts4, n, k, d_out + 2 * (size_t)n, d_status);
      cudaEventRecord(ev[5], st);
      cudaMemcpyAsync(rho, d_out, sizeof(float) * 3 * (size_t)n, cudaMemcpyDeviceToHost, st);
      e = cudaStreamSynchronize(st);
    }
    uint32_t status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, d_status, sizeof(status), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      rc = NEB_ERR_CUDA;
    } else if (status) {
      rc = NEB_ERR_QUEUE_OVERFLOW;
    } else if (ms) {
      for (int i = 0; i < 3; ++i) {
        float t = 0.0f;
        cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
        ms[i] = t;
      }
    }
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  cudaFree(d_pos); cudaFree(d_nrm); cudaFree(d_out); cudaFree(d_pts4); cudaFree(d_sorted); cudaFree(d_nodes);
  cudaFree(d_st); cudaFree(bc); cudaFree(bs); cudaFree(vb); cudaFree(sc.data); cudaFree(d_status); cudaFree(tree);
  cudaStreamDestroy(st);
  return rc;
}
