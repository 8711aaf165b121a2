// neb_octree.cu -- density octree kernels (Sec. 5) and the stand-alone
// octree entry points of the C ABI.
#include <cmath>
#include <cstring>
#include <new>

#include "neb_internal.h"
#include "neb_octree.cuh"

namespace neb {

// The octree box is the scene box grown by 0.2 % about its centre, so that
// points on the scene's bounds fall inside (Appendix B does the same); the
// pool holds the requested number of words rounded up to 8m + 1 (the root and
// m groups of eight children).
OctreeParams octree_params(const float smin[3], const float smax[3], int capacity, int split_factor) {
  OctreeParams P;
  float edge[3];
  for (int c = 0; c < 3; ++c) {
    edge[c] = (smax[c] - smin[c]) * 1.002f;
    P.size_inv[c] = 1.0f / edge[c];
    P.box_extent[c] = 1.0 / (double)P.size_inv[c];
    P.minb[c] = smin[c] - edge[c] * (0.001f / 1.002f);
  }
  P.scene_scale = sqrtf(edge[0] * edge[0] + edge[1] * edge[1] + edge[2] * edge[2]);
  P.capacity = 8 * ((capacity + 7) / 8) + 1;
  P.split_count = split_factor;
  P.iter_clamp = 1;
  P.stop_filling = 0;
  P.init_value = 0;
  return P;
}

// Counts are integrated over the iterations (Sec. 5.4): the split threshold
// grows with the iteration (up to 1000, after which counting stops) and
// densities are divided by it.  A new cell starts with a quarter of the
// split factor per iteration so far, since a surface crosses about four of a
// cell's eight children (Sec. 5.2).  The re-arm kernel below writes that
// count into every free word of the pool.
void octree_set_iteration_params(OctreeParams& P, int split_factor, int iter) {
  const int ic = iter < kFillIterations ? iter : kFillIterations;
  P.iter_clamp = ic;
  P.stop_filling = iter > kFillIterations;
  P.split_count = split_factor * ic;
  P.init_value = (split_factor * ic + 3) / 4;  // ceil(split_factor * iter / 4) while counting
}

// every free word [alloc, capacity) gets the count a new cell starts with
__global__ void k_oct_rearm(int* nodes, const OctreeState* st, OctreeParams P) {
  if (P.stop_filling) return;
  int a = *((const volatile int*)&st->alloc);
  for (long long i = a + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P.capacity;
       i += (long long)gridDim.x * blockDim.x)
    nodes[i] = P.init_value;
}

// Appends index i to a list when pred (warp-aggregated; all lanes call it).
__device__ __forceinline__ void warp_push(int* list, int* count, bool pred, int i) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m == 0) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = i;
}

// Counts one vertex per lane in its leaf once no cell can split any more:
// a read-only descent, and lanes of a warp that land in the same leaf add
// their count with one atomic (neighbouring paths share leaves; crowded
// leaves would otherwise serialise thousands of single increments).  All
// lanes call it; pos == nullptr for a lane without a vertex.
__device__ __forceinline__ void oct_count_frozen(int* nodes, const OctreeParams& P, const float* pos) {
  const int leaf = pos ? oct_frozen_leaf(nodes, P, pos) : -1;
  const unsigned same = __match_any_sync(0xffffffffu, leaf);
  if (leaf >= 0 && (int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(nodes + leaf, __popc(same));
}

// Concurrent inserts of n points; those that find the pool exhausted go to
// the deferred list, counted by k_oct_count_deferred_points after this launch.
__global__ void k_oct_insert_points(int* nodes, OctreeState* st, OctreeParams P, const float* __restrict__ pos, int n,
                                    int spin_limit, int* deferred, int* n_deferred) {
  const bool frozen = st->alloc > P.capacity;  // overflowed in an earlier launch
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    float p[3] = {0.0f, 0.0f, 0.0f};
    if (i < n) {
      p[0] = pos[3 * i];
      p[1] = pos[3 * i + 1];
      p[2] = pos[3 * i + 2];
    }
    if (frozen) {
      oct_count_frozen(nodes, P, i < n ? p : nullptr);
      continue;
    }
    const bool later = i < n && !oct_insert<true>(nodes, st, P, p, spin_limit);
    warp_push(deferred, n_deferred, later, i);
  }
}

__global__ void k_oct_count_deferred_points(int* nodes, OctreeParams P, const float* __restrict__ pos,
                                            const int* __restrict__ deferred, const int* n_deferred) {
  const int n = *n_deferred;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    float p[3] = {0.0f, 0.0f, 0.0f};
    if (i < n) {
      const int j = deferred[i];
      p[0] = pos[3 * j];
      p[1] = pos[3 * j + 1];
      p[2] = pos[3 * j + 2];
    }
    oct_count_frozen(nodes, P, i < n ? p : nullptr);
  }
}

__global__ void k_oct_insert_points_seq(int* nodes, OctreeState* st, OctreeParams P, const float* __restrict__ pos,
                                        int n) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int i = 0; i < n; ++i) {
    float p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    oct_insert_seq(nodes, st, P, p);
  }
}

__global__ void k_oct_density_points(const int* __restrict__ nodes, OctreeParams P, const float* __restrict__ pos,
                                     const float* __restrict__ nrm, int n, int robust, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    float q[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
    int nq = 0;
    out[i] = robust ? oct_density_robust(nodes, P, p, q, &nq) : oct_density(nodes, P, p, q);
  }
}

// NEB pass: inserts of this iteration's NEE vertices.  Once the pool is
// exhausted (in an earlier iteration, or during this launch for the vertices
// that meet it, which go to the deferred list) no cell can split any more and
// every insert only counts in its leaf.
__global__ void k_oct_insert_nee(int* nodes, OctreeState* st, OctreeParams P, const float4* __restrict__ vpos,
                                 DevCounters* cnt, int cap, int spin_limit, int* deferred) {
  int count = min(cnt->nee_count, cap);
  const bool frozen = st->alloc > P.capacity;  // overflowed in an earlier iteration
  uint32_t done = 0;
  for (int base = blockIdx.x * blockDim.x; base < count; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    float p[3] = {0.0f, 0.0f, 0.0f};
    if (i < count) {
      const float4 v = vpos[i];
      p[0] = v.x;
      p[1] = v.y;
      p[2] = v.z;
    }
    if (frozen) {
      oct_count_frozen(nodes, P, i < count ? p : nullptr);
      done += i < count;
      continue;
    }
    const bool later = i < count && !oct_insert<true>(nodes, st, P, p, spin_limit);
    done += i < count && !later;
    warp_push(deferred, &cnt->oct_deferred, later, i);
  }
  if (done) atomicAdd(&cnt->octree_inserts, (unsigned long long)done);
}

// The vertices that met the exhausted pool during k_oct_insert_nee, counted
// in their leaves now that every link of that launch is published.
__global__ void k_oct_count_deferred_nee(int* nodes, OctreeParams P, const float4* __restrict__ vpos,
                                         DevCounters* cnt, const int* __restrict__ deferred) {
  const int n = cnt->oct_deferred;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    float p[3] = {0.0f, 0.0f, 0.0f};
    if (i < n) {
      const float4 v = vpos[deferred[i]];
      p[0] = v.x;
      p[1] = v.y;
      p[2] = v.z;
    }
    oct_count_frozen(nodes, P, i < n ? p : nullptr);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && n) atomicAdd(&cnt->octree_inserts, (unsigned long long)n);
}

// deterministic mode: one thread inserts in (pixel, k) order
__global__ void k_oct_insert_nee_seq(int* nodes, OctreeState* st, OctreeParams P, const float4* __restrict__ vpos,
                                     const int* __restrict__ slot_map, int n_slots, DevCounters* cnt) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  unsigned long long done = 0;
  for (int s = 0; s < n_slots; ++s) {
    int id = slot_map[s];
    if (id < 0) continue;
    float4 v = vpos[id];
    float p[3] = {v.x, v.y, v.z};
    oct_insert_seq(nodes, st, P, p);
    ++done;
  }
  cnt->octree_inserts += done;
}

// rho at the NEE vertices.  Unless `all`, only at the vertices of the lit
// list (their shadow ray reached the light): there rho enters w_E and the
// photon flux; elsewhere no result reads it (the random-hit weight evaluates
// its own, k_emission), and the -2 stored at the vertex's creation stays.
__global__ void k_oct_density_nee(const int* __restrict__ nodes, const OctreeState* st, OctreeParams P,
                                  const float4* __restrict__ vpos, const float4* __restrict__ vnrm, float4* vldir,
                                  const int* __restrict__ lit, DevCounters* cnt, int cap, int robust, int all) {
  int count = min(all ? cnt->nee_count : cnt->lit_count, cap);
  int queries = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    const int i = all ? t : lit[t];
    float4 v = vpos[i], nn = vnrm[i];
    float p[3] = {v.x, v.y, v.z};
    float q[3] = {nn.x, nn.y, nn.z};
    float rho;
    if (robust) {
      rho = oct_density_robust(nodes, P, p, q, &queries);
    } else {
      rho = oct_density(nodes, P, p, q);
      ++queries;
    }
    vldir[i].w = rho;
  }
  if (queries) atomicAdd(&cnt->octree_queries, (unsigned long long)queries);
}

static int blocks_for(int n, int threads) {
  int b = (n + threads - 1) / threads;
  return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

cudaError_t launch_oct_rearm(int* nodes, const OctreeState* st, const OctreeParams& P, cudaStream_t s) {
  k_oct_rearm<<<blocks_for(P.capacity, 256), 256, 0, s>>>(nodes, st, P);
  return cudaGetLastError();
}

cudaError_t launch_oct_insert_points(int* nodes, OctreeState* st, const OctreeParams& P, const float* d_pos, int n,
                                     int mode, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (mode == 1) {
    k_oct_insert_points_seq<<<1, 1, 0, s>>>(nodes, st, P, d_pos, n);
    return cudaGetLastError();
  }
  int* deferred = nullptr;  // the deferred list, then its length
  cudaError_t e = cudaMallocAsync(&deferred, sizeof(int) * ((size_t)n + 1), s);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(deferred + n, 0, sizeof(int), s);
  k_oct_insert_points<<<blocks_for(n, 256), 256, 0, s>>>(nodes, st, P, d_pos, n, kSpinLimit, deferred, deferred + n);
  k_oct_count_deferred_points<<<blocks_for(n, 256), 256, 0, s>>>(nodes, P, d_pos, deferred, deferred + n);
  e = cudaGetLastError();
  cudaFreeAsync(deferred, s);
  return e;
}

cudaError_t launch_oct_density_points(const int* nodes, const OctreeState* st, const OctreeParams& P,
                                      const float* d_pos, const float* d_nrm, int n, int robust, float* d_out,
                                      cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  (void)st;
  k_oct_density_points<<<blocks_for(n, 256), 256, 0, s>>>(nodes, P, d_pos, d_nrm, n, robust, d_out);
  return cudaGetLastError();
}

cudaError_t launch_oct_insert_nee(neb_ctx* c, const IterSlot& sl, cudaStream_t st) {
  if (c->cfg.octree_mode == 1)
    k_oct_insert_nee_seq<<<1, 1, 0, st>>>(c->oct_nodes, c->oct_state, c->oct, sl.nv.pos, sl.slot_map,
                                          c->P * (c->D - 1), sl.cnt);
  else {
    // the deferred list borrows the grid's per-vertex bucket array, which the
    // grid build of this iteration writes afresh after the density pass
    const int B = capped_blocks(c->cap_nee, 256, 152 * 8);
    k_oct_insert_nee<<<B, 256, 0, st>>>(c->oct_nodes, c->oct_state, c->oct, sl.nv.pos, sl.cnt, c->cap_nee, kSpinLimit,
                                        c->vert_bucket);
    k_oct_count_deferred_nee<<<B, 256, 0, st>>>(c->oct_nodes, c->oct, sl.nv.pos, sl.cnt, c->vert_bucket);
  }
  return cudaGetLastError();
}

cudaError_t launch_oct_density_nee(neb_ctx* c, const IterSlot& sl, cudaStream_t st) {
  k_oct_density_nee<<<capped_blocks(c->cap_nee, 256, 152 * 8), 256, 0, st>>>(c->oct_nodes, c->oct_state, c->oct, sl.nv.pos, sl.nv.nrm, sl.nv.ldir,
                                             sl.nv.lit, sl.cnt, c->cap_nee, c->cfg.density_mode == 0,
                                             c->cfg.density_all);
  return cudaGetLastError();
}

}  // namespace neb

// ---------------------------------------------------------------------------
// stand-alone octree (C ABI)
// ---------------------------------------------------------------------------
struct neb_octree {
  neb::OctreeParams P{};
  int split_factor = 4;
  int* nodes = nullptr;
  neb::OctreeState* st = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
};

extern "C" int neb_octree_create(const float scene_min[3], const float scene_max[3], int capacity, int split_factor,
                                 void* cuda_stream, neb_octree** out) {
  if (!scene_min || !scene_max || !out || capacity < 1 || split_factor < 2) return NEB_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return NEB_ERR_NO_DEVICE;
  neb_octree* o = new (std::nothrow) neb_octree();
  if (!o) return NEB_ERR_OOM;
  o->P = neb::octree_params(scene_min, scene_max, capacity, split_factor);
  o->split_factor = split_factor;
  if (cuda_stream) {
    o->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&o->stream, cudaStreamNonBlocking) != cudaSuccess) { delete o; return NEB_ERR_CUDA; }
    o->own_stream = true;
  }
  if (cudaMalloc(&o->nodes, sizeof(int) * (size_t)o->P.capacity) != cudaSuccess ||
      cudaMalloc(&o->st, sizeof(neb::OctreeState)) != cudaSuccess) {
    neb_octree_destroy(o);
    return NEB_ERR_OOM;
  }
  neb::OctreeState s0{1, 0, 0, 0};
  cudaMemsetAsync(o->nodes, 0, sizeof(int) * (size_t)o->P.capacity, o->stream);
  cudaMemcpyAsync(o->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, o->stream);
  if (cudaStreamSynchronize(o->stream) != cudaSuccess) { neb_octree_destroy(o); return NEB_ERR_CUDA; }
  *out = o;
  return NEB_OK;
}

extern "C" void neb_octree_destroy(neb_octree* o) {
  if (!o) return;
  if (o->nodes) cudaFree(o->nodes);
  if (o->st) cudaFree(o->st);
  if (o->own_stream && o->stream) cudaStreamDestroy(o->stream);
  delete o;
}

extern "C" int neb_octree_set_iteration(neb_octree* o, int iter) {
  if (!o || iter < 1) return NEB_ERR_ARG;
  neb::octree_set_iteration_params(o->P, o->split_factor, iter);
  if (neb::launch_oct_rearm(o->nodes, o->st, o->P, o->stream) != cudaSuccess) return NEB_ERR_CUDA;
  return cudaStreamSynchronize(o->stream) == cudaSuccess ? NEB_OK : NEB_ERR_CUDA;
}

extern "C" int neb_octree_insert(neb_octree* o, const float* pos, int n, int mode) {
  if (!o || (n > 0 && !pos) || n < 0 || (mode != 0 && mode != 1)) return NEB_ERR_ARG;
  if (n == 0) return NEB_OK;
  float* d = nullptr;
  if (cudaMallocAsync(&d, sizeof(float) * 3 * (size_t)n, o->stream) != cudaSuccess) return NEB_ERR_OOM;
  cudaMemcpyAsync(d, pos, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, o->stream);
  cudaError_t e = neb::launch_oct_insert_points(o->nodes, o->st, o->P, d, n, mode, o->stream);
  cudaFreeAsync(d, o->stream);
  if (e != cudaSuccess || cudaStreamSynchronize(o->stream) != cudaSuccess) return NEB_ERR_CUDA;
  neb::OctreeState s;
  cudaMemcpy(&s, o->st, sizeof(s), cudaMemcpyDeviceToHost);
  if (s.status & NEB_STATUS_SPIN_TIMEOUT) return NEB_ERR_DEVICE_TIMEOUT;
  return NEB_OK;
}

extern "C" int neb_octree_density(neb_octree* o, const float* pos, const float* nrm, int n, int robust, float* out) {
  if (!o || n < 0 || (n > 0 && (!pos || !nrm || !out))) return NEB_ERR_ARG;
  if (n == 0) return NEB_OK;
  float* d = nullptr;
  size_t bytes = sizeof(float) * 3 * (size_t)n;
  if (cudaMallocAsync(&d, bytes * 2 + sizeof(float) * (size_t)n, o->stream) != cudaSuccess) return NEB_ERR_OOM;
  cudaMemcpyAsync(d, pos, bytes, cudaMemcpyHostToDevice, o->stream);
  cudaMemcpyAsync(d + 3 * (size_t)n, nrm, bytes, cudaMemcpyHostToDevice, o->stream);
  float* dout = d + 6 * (size_t)n;
  cudaError_t e = neb::launch_oct_density_points(o->nodes, o->st, o->P, d, d + 3 * (size_t)n, n, robust, dout,
                                                 o->stream);
  cudaMemcpyAsync(out, dout, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, o->stream);
  cudaFreeAsync(d, o->stream);
  if (e != cudaSuccess || cudaStreamSynchronize(o->stream) != cudaSuccess) return NEB_ERR_CUDA;
  return NEB_OK;
}

extern "C" int neb_octree_load(neb_octree* o, const int32_t* nodes, int n_nodes, int alloc, int depth) {
  // words in use are the root plus whole groups of eight, or capacity + 1
  // once the pool has been exhausted
  if (!o || !nodes || n_nodes < 1 || n_nodes > o->P.capacity || alloc < 1 || alloc > o->P.capacity + 1 ||
      ((alloc - 1) % 8 != 0 && alloc != o->P.capacity + 1) || depth < 0 || depth > neb::kOctMaxDepth)
    return NEB_ERR_ARG;
  neb::OctreeState s{alloc, depth, 0u, 0};
  cudaMemsetAsync(o->nodes, 0, sizeof(int) * (size_t)o->P.capacity, o->stream);
  cudaMemcpyAsync(o->nodes, nodes, sizeof(int) * (size_t)n_nodes, cudaMemcpyHostToDevice, o->stream);
  cudaMemcpyAsync(o->st, &s, sizeof(s), cudaMemcpyHostToDevice, o->stream);
  return cudaStreamSynchronize(o->stream) == cudaSuccess ? NEB_OK : NEB_ERR_CUDA;
}

extern "C" int neb_octree_read(neb_octree* o, int32_t* nodes, int n_nodes, int32_t meta[4]) {
  if (!o || !meta) return NEB_ERR_ARG;
  neb::OctreeState s;
  if (cudaMemcpyAsync(&s, o->st, sizeof(s), cudaMemcpyDeviceToHost, o->stream) != cudaSuccess) return NEB_ERR_CUDA;
  int m = n_nodes < o->P.capacity ? n_nodes : o->P.capacity;
  if (nodes && m > 0) cudaMemcpyAsync(nodes, o->nodes, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, o->stream);
  if (cudaStreamSynchronize(o->stream) != cudaSuccess) return NEB_ERR_CUDA;
  meta[0] = s.alloc;
  meta[1] = s.depth;
  meta[2] = o->P.capacity;
  meta[3] = (int32_t)s.status;
  return NEB_OK;
}
