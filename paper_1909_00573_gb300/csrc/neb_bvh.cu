// neb_bvh.cu -- BVH construction on the device (linear BVH: Morton codes,
// radix sort, Karras' parallel hierarchy, bottom-up bounds) and the small
// component kernels used by the tests (closest hit, Philox, plane/box area).
//
// Karras, "Maximizing Parallelism in the Construction of BVHs, Octrees, and
// k-d Trees", HPG 2012.
#include <cuda_runtime.h>

#include <cfloat>

#include "neb_device.cuh"
#include "neb_internal.h"
#include "neb_octree.cuh"

namespace neb {

__device__ __forceinline__ int float_to_ordered(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_to_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ void prim_bounds(const SceneView& s, int p, float3& lo, float3& hi) {
  if (p < s.nt) {
    float3 a = xyz(__ldg(s.tv0 + p)), b = xyz(__ldg(s.tv1 + p)), c = xyz(__ldg(s.tv2 + p));
    lo = f3(fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z)));
    hi = f3(fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z)));
  } else {
    float4 sp = __ldg(s.sph + (p - s.nt));
    lo = f3(sp.x - sp.w, sp.y - sp.w, sp.z - sp.w);
    hi = f3(sp.x + sp.w, sp.y + sp.w, sp.z + sp.w);
  }
}

// centroid bounds (ordered-int atomics)
__global__ void k_centroid_bounds(SceneView s, int n, int* cb) {
  float3 lo = f3(FLT_MAX, FLT_MAX, FLT_MAX), hi = f3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    float3 a, b;
    prim_bounds(s, p, a, b);
    float3 c = mul(add(a, b), 0.5f);
    lo = f3(fminf(lo.x, c.x), fminf(lo.y, c.y), fminf(lo.z, c.z));
    hi = f3(fmaxf(hi.x, c.x), fmaxf(hi.y, c.y), fmaxf(hi.z, c.z));
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
    lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
    lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(cb + 0, float_to_ordered(lo.x));
    atomicMin(cb + 1, float_to_ordered(lo.y));
    atomicMin(cb + 2, float_to_ordered(lo.z));
    atomicMax(cb + 3, float_to_ordered(hi.x));
    atomicMax(cb + 4, float_to_ordered(hi.y));
    atomicMax(cb + 5, float_to_ordered(hi.z));
  }
}

__device__ __forceinline__ uint32_t expand_bits(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

// Morton code of the centroid on a 2^21 grid per axis (63 bits), as two
// sort keys: hi = the top 30 bits (the code of the top 10 bits of each
// coordinate), lo = the next 32 bits.  Sorting by lo and then, stably, by hi
// orders by the 62-bit prefix: small, dense objects (a torus of 20,000
// triangles inside one 1/1024 cell of a city) keep a spatial order instead of
// the order of their primitive indices.
__device__ __forceinline__ uint32_t expand_bits11(uint32_t v) {  // 11 bits -> every third of 31
  return expand_bits(v & 1023u) | (((v >> 10) & 1u) << 30);
}

__global__ void k_morton(SceneView s, int n, const int* cb, uint32_t* keys_hi, uint32_t* keys_lo, int* vals) {
  float3 lo = f3(ordered_to_float(cb[0]), ordered_to_float(cb[1]), ordered_to_float(cb[2]));
  float3 hi = f3(ordered_to_float(cb[3]), ordered_to_float(cb[4]), ordered_to_float(cb[5]));
  // one scale for all axes: Morton cells stay cubes in world space, so flat
  // scenes (a city is 400 x 20 x 400) are not split along their short axis
  // as often as along the long ones
  float3 ext = sub(hi, lo);
  float e = fmaxf(ext.x, fmaxf(ext.y, ext.z));
  float inv = e > 0.0f ? 1.0f / e : 0.0f;
  const float g = 2097152.0f;  // 2^21
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    float3 a, b;
    prim_bounds(s, p, a, b);
    float3 c = mul(add(a, b), 0.5f);
    float x = (c.x - lo.x) * inv;
    float y = (c.y - lo.y) * inv;
    float z = (c.z - lo.z) * inv;
    uint32_t ix = (uint32_t)fminf(fmaxf(x * g, 0.0f), g - 1.0f);
    uint32_t iy = (uint32_t)fminf(fmaxf(y * g, 0.0f), g - 1.0f);
    uint32_t iz = (uint32_t)fminf(fmaxf(z * g, 0.0f), g - 1.0f);
    keys_hi[p] = (expand_bits(ix >> 11) << 2) | (expand_bits(iy >> 11) << 1) | expand_bits(iz >> 11);
    uint64_t m33 = ((uint64_t)expand_bits11(ix & 2047u) << 2) | ((uint64_t)expand_bits11(iy & 2047u) << 1) |
                   (uint64_t)expand_bits11(iz & 2047u);
    keys_lo[p] = (uint32_t)(m33 >> 1);
    vals[p] = p;
  }
}

__global__ void k_gather_keys(const uint32_t* __restrict__ keys, const int* __restrict__ order, int n,
                              uint32_t* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = keys[order[i]];
}

// ---- stable LSD radix sort, 4-bit digits, one element per thread ----------------
constexpr int kSortThreads = 256;

__global__ void k_digit_hist(const uint32_t* __restrict__ keys, int n, int shift, int nblocks, int* hist) {
  __shared__ int h[16];
  if (threadIdx.x < 16) h[threadIdx.x] = 0;
  __syncthreads();
  int i = blockIdx.x * kSortThreads + threadIdx.x;
  if (i < n) atomicAdd(&h[(keys[i] >> shift) & 15u], 1);
  __syncthreads();
  if (threadIdx.x < 16) hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_digit_scatter(const uint32_t* __restrict__ keys, const int* __restrict__ vals, int n, int shift,
                                int nblocks, const int* __restrict__ offs, uint32_t* __restrict__ okeys,
                                int* __restrict__ ovals) {
  __shared__ int wcount[kSortThreads / 32][16];
  __shared__ int wpre[kSortThreads / 32][16];
  int i = blockIdx.x * kSortThreads + threadIdx.x;
  bool valid = i < n;
  uint32_t key = valid ? keys[i] : 0u;
  int digit = valid ? (int)((key >> shift) & 15u) : 16;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int rank = 0, mycount = 0;
#pragma unroll
  for (int v = 0; v < 16; ++v) {
    unsigned b = __ballot_sync(0xffffffffu, digit == v);
    if (lane == v) mycount = __popc(b);
    if (digit == v) rank = __popc(b & ((1u << lane) - 1u));
  }
  if (lane < 16) wcount[warp][lane] = mycount;
  __syncthreads();
  if (threadIdx.x < 16) {
    int run = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) {
      wpre[w][threadIdx.x] = run;
      run += wcount[w][threadIdx.x];
    }
  }
  __syncthreads();
  if (valid) {
    int dst = offs[digit * nblocks + blockIdx.x] + wpre[warp][digit] + rank;
    okeys[dst] = key;
    ovals[dst] = vals[i];
  }
}

// ---- Karras hierarchy ------------------------------------------------------------
__device__ __forceinline__ int karras_delta(const uint32_t* keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint32_t a = keys[i], b = keys[j];
  if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
  return __clz(a ^ b);
}

// children: >= 0 internal node, < 0 ~(sorted leaf position)
__global__ void k_karras(const uint32_t* __restrict__ keys, int n, int2* child, int* parent_int, int* parent_leaf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x) {
    int dnext = karras_delta(keys, n, i, i + 1), dprev = karras_delta(keys, n, i, i - 1);
    int d = dnext > dprev ? 1 : -1;
    int dmin = karras_delta(keys, n, i, i - d);
    int lmax = 2;
    while (karras_delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
      if (karras_delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = karras_delta(keys, n, i, j);
    int s = 0, t = l;
    do {
      t = (t + 1) >> 1;
      if (karras_delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + (d < 0 ? -1 : 0);
    int lo = min(i, j), hi = max(i, j);
    int left = (lo == gamma) ? ~gamma : gamma;
    int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    child[i] = make_int2(left, right);
    if (left >= 0) parent_int[left] = i; else parent_leaf[~left] = i;
    if (right >= 0) parent_int[right] = i; else parent_leaf[~right] = i;
  }
}

struct Box6 {
  float lo[3], hi[3];
};

__device__ __forceinline__ void child_box(const SceneView& s, int c, const int* sorted_prim, const Box6* boxes,
                                          float3& lo, float3& hi) {
  if (c < 0) {
    prim_bounds(s, sorted_prim[~c], lo, hi);
  } else {
    const float* b = reinterpret_cast<const float*>(boxes + c);
    lo = f3(__ldcg(b + 0), __ldcg(b + 1), __ldcg(b + 2));
    hi = f3(__ldcg(b + 3), __ldcg(b + 4), __ldcg(b + 5));
  }
}

__global__ void k_bounds(SceneView s, int n, const int* __restrict__ sorted_prim, const int2* __restrict__ child,
                         const int* __restrict__ parent_int, const int* __restrict__ parent_leaf, int* flags,
                         Box6* boxes) {
  for (int leaf = blockIdx.x * blockDim.x + threadIdx.x; leaf < n; leaf += gridDim.x * blockDim.x) {
    int p = parent_leaf[leaf];
    while (p >= 0) {
      __threadfence();
      if (atomicAdd(flags + p, 1) == 0) break;  // the sibling finishes this node
      __threadfence();
      int2 ch = child[p];
      float3 a0, a1, b0, b1;
      child_box(s, ch.x, sorted_prim, boxes, a0, a1);
      child_box(s, ch.y, sorted_prim, boxes, b0, b1);
      float* out = reinterpret_cast<float*>(boxes + p);
      __stcg(out + 0, fminf(a0.x, b0.x));
      __stcg(out + 1, fminf(a0.y, b0.y));
      __stcg(out + 2, fminf(a0.z, b0.z));
      __stcg(out + 3, fmaxf(a1.x, b1.x));
      __stcg(out + 4, fmaxf(a1.y, b1.y));
      __stcg(out + 5, fmaxf(a1.z, b1.z));
      p = p == 0 ? -1 : parent_int[p];
    }
  }
}

__global__ void k_write_nodes(SceneView s, int n, const int* __restrict__ sorted_prim, const int2* __restrict__ child,
                              const Box6* boxes, BVHNode* nodes) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x) {
    int2 ch = child[i];
    float3 a0, a1, b0, b1;
    child_box(s, ch.x, sorted_prim, boxes, a0, a1);
    child_box(s, ch.y, sorted_prim, boxes, b0, b1);
    BVHNode nd;
    nd.a = make_float4(a0.x, a1.x, a0.y, a1.y);
    nd.b = make_float4(b0.x, b1.x, b0.y, b1.y);
    nd.c = make_float4(a0.z, a1.z, b0.z, b1.z);
    int l = ch.x < 0 ? ~sorted_prim[~ch.x] : ch.x;
    int r = ch.y < 0 ? ~sorted_prim[~ch.y] : ch.y;
    nd.ch = make_int4(l, r, 0, 0);
    nodes[i] = nd;
  }
}

__global__ void k_single_leaf(SceneView s, BVH4Node* nodes) {
  float3 lo, hi;
  prim_bounds(s, 0, lo, hi);
  BVH4Node nd;
  const float I = INFINITY;
  nd.lox = make_float4(lo.x, I, I, I);
  nd.hix = make_float4(hi.x, -I, -I, -I);
  nd.loy = make_float4(lo.y, I, I, I);
  nd.hiy = make_float4(hi.y, -I, -I, -I);
  nd.loz = make_float4(lo.z, I, I, I);
  nd.hiz = make_float4(hi.z, -I, -I, -I);
  nd.ch = make_int4(~0, kEmptyChild, kEmptyChild, kEmptyChild);
  nd.pad = make_float4(0, 0, 0, 0);
  nodes[0] = nd;
}

// ---- PLOC: parallel locally-ordered clustering over the Morton order -------------
// Meister and Bittner, "Parallel Locally-Ordered Clustering for Bounding Volume
// Hierarchy Construction", IEEE TVCG 2018.  Clusters start as the Morton-sorted
// primitives; every round each cluster finds the neighbour within +-R positions
// whose union box has the smallest surface area, mutual nearest neighbours merge
// into a new internal node, and the survivors are compacted in order.  Internal
// nodes are numbered from N-2 downwards so the final merge (the root) is node 0.
constexpr int kPlocR = 16;
constexpr int kPlocThreads = 256;

__device__ __forceinline__ float half_area(float3 lo, float3 hi) {
  float3 d = sub(hi, lo);
  return d.x * d.y + d.y * d.z + d.z * d.x;
}

__global__ void k_ploc_init(SceneView s, int n, const int* __restrict__ sorted_prim, int* cid, float4* blo,
                            float4* bhi) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int p = sorted_prim[i];
    float3 lo, hi;
    prim_bounds(s, p, lo, hi);
    cid[i] = ~p;
    blo[i] = make_float4(lo.x, lo.y, lo.z, 0.0f);
    bhi[i] = make_float4(hi.x, hi.y, hi.z, 0.0f);
  }
}

__global__ void __launch_bounds__(kPlocThreads) k_ploc_nn(int n, const float4* __restrict__ blo,
                                                          const float4* __restrict__ bhi, int* __restrict__ nn) {
  __shared__ float4 slo[kPlocThreads + 2 * kPlocR], shi[kPlocThreads + 2 * kPlocR];
  int b0 = blockIdx.x * kPlocThreads;
  for (int t = threadIdx.x; t < kPlocThreads + 2 * kPlocR; t += kPlocThreads) {
    int g = b0 - kPlocR + t;
    if (g >= 0 && g < n) {
      slo[t] = blo[g];
      shi[t] = bhi[g];
    }
  }
  __syncthreads();
  int i = b0 + threadIdx.x;
  if (i >= n) return;
  int me = threadIdx.x + kPlocR;
  float3 alo = xyz(slo[me]), ahi = xyz(shi[me]);
  float best = 3.402823466e+38f;
  int bj = -1;
  for (int d = -kPlocR; d <= kPlocR; ++d) {
    int j = i + d;
    if (d == 0 || j < 0 || j >= n) continue;
    float3 lo = xyz(slo[me + d]), hi = xyz(shi[me + d]);
    float a = half_area(f3(fminf(alo.x, lo.x), fminf(alo.y, lo.y), fminf(alo.z, lo.z)),
                        f3(fmaxf(ahi.x, hi.x), fmaxf(ahi.y, hi.y), fmaxf(ahi.z, hi.z)));
    if (a < best) {  // ascending j: ties keep the smaller index
      best = a;
      bj = j;
    }
  }
  nn[i] = bj;
}

__global__ void k_ploc_flags(int n, const int* __restrict__ nn, int* merge_flag, int* keep_flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int j = nn[i];
    bool mutual = j >= 0 && nn[j] == i;
    merge_flag[i] = (mutual && i < j) ? 1 : 0;
    keep_flag[i] = (!mutual || i < j) ? 1 : 0;
  }
}

__global__ void k_ploc_compact(int n, const int* __restrict__ nn, const int* __restrict__ cid,
                               const float4* __restrict__ blo, const float4* __restrict__ bhi,
                               const int* __restrict__ merge_rank, const int* __restrict__ keep_pos, int node_base,
                               BVHNode* nodes, int* cid2, float4* blo2, float4* bhi2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int j = nn[i];
    bool mutual = j >= 0 && nn[j] == i;
    if (mutual && i > j) continue;  // absorbed by its partner
    int pos = keep_pos[i];
    float4 lo = blo[i], hi = bhi[i];
    if (!mutual) {
      cid2[pos] = cid[i];
      blo2[pos] = lo;
      bhi2[pos] = hi;
      continue;
    }
    float4 lo2 = blo[j], hi2 = bhi[j];
    int node = node_base - merge_rank[i];
    BVHNode nd;
    nd.a = make_float4(lo.x, hi.x, lo.y, hi.y);
    nd.b = make_float4(lo2.x, hi2.x, lo2.y, hi2.y);
    nd.c = make_float4(lo.z, hi.z, lo2.z, hi2.z);
    nd.ch = make_int4(cid[i], cid[j], 0, 0);
    nodes[node] = nd;
    cid2[pos] = node;
    blo2[pos] = make_float4(fminf(lo.x, lo2.x), fminf(lo.y, lo2.y), fminf(lo.z, lo2.z), 0.0f);
    bhi2[pos] = make_float4(fmaxf(hi.x, hi2.x), fmaxf(hi.y, hi2.y), fmaxf(hi.z, hi2.z), 0.0f);
  }
}

// merges and survivors of a round: the last entries of the two exclusive scans plus their flags
__global__ void k_ploc_tail(const int* mrank, const int* mflag, const int* kpos, const int* kflag, int count,
                            int* out) {
  out[0] = mrank[count - 1] + mflag[count - 1];
  out[1] = kpos[count - 1] + kflag[count - 1];
}

// A build's temporaries are stream-ordered allocations on its stream (no
// device-wide synchronisation on free), and its per-round readbacks go to one
// pinned word pair per host thread, allocated once.
template <typename T>
static bool talloc(T** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, st) == cudaSuccess;
}
template <typename T>
static void tfree(T* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}
static int* readback_words() {
  thread_local int* h = nullptr;
  if (!h && cudaMallocHost(&h, 2 * sizeof(int)) != cudaSuccess) h = nullptr;
  return h;
}

static cudaError_t ploc_build(const SceneView& s, int n, const int* sorted_prim, BVHNode* nodes, Scratch& sc,
                              cudaStream_t st) {
  int *cid[2] = {nullptr, nullptr}, *nn = nullptr, *mflag = nullptr, *kflag = nullptr, *mrank = nullptr,
      *kpos = nullptr, *tail = nullptr;
  float4 *blo[2] = {nullptr, nullptr}, *bhi[2] = {nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  bool ok = talloc(&cid[0], 4ull * n, st) && talloc(&cid[1], 4ull * n, st) && talloc(&blo[0], 16ull * n, st) &&
            talloc(&blo[1], 16ull * n, st) && talloc(&bhi[0], 16ull * n, st) && talloc(&bhi[1], 16ull * n, st) &&
            talloc(&nn, 4ull * n, st) && talloc(&mflag, 4ull * n, st) && talloc(&kflag, 4ull * n, st) &&
            talloc(&mrank, 4ull * n, st) && talloc(&kpos, 4ull * n, st) && talloc(&tail, 16, st);
  int* h = readback_words();  // pinned: the per-round readback is one small asynchronous copy
  ok = ok && h;
  if (!ok) e = cudaErrorMemoryAllocation;
  if (ok) {
    int gb = (n + 255) / 256;
    if (gb > 152 * 16) gb = 152 * 16;
    k_ploc_init<<<gb, 256, 0, st>>>(s, n, sorted_prim, cid[0], blo[0], bhi[0]);
    int cur = 0, count = n, base = n - 2;
    int rounds = 0;
    while (count > 1 && e == cudaSuccess) {
      int nb = (count + kPlocThreads - 1) / kPlocThreads;
      k_ploc_nn<<<nb, kPlocThreads, 0, st>>>(count, blo[cur], bhi[cur], nn);
      int fb = nb > 152 * 16 ? 152 * 16 : nb;
      k_ploc_flags<<<fb, 256, 0, st>>>(count, nn, mflag, kflag);
      scan_exclusive(mflag, mrank, count, sc, st);
      scan_exclusive(kflag, kpos, count, sc, st);
      k_ploc_tail<<<1, 1, 0, st>>>(mrank, mflag, kpos, kflag, count, tail);
      cudaMemcpyAsync(h, tail, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
      k_ploc_compact<<<fb, 256, 0, st>>>(count, nn, cid[cur], blo[cur], bhi[cur], mrank, kpos, base, nodes,
                                         cid[1 - cur], blo[1 - cur], bhi[1 - cur]);
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) break;
      int merges = h[0], next = h[1];
      if (merges <= 0 || next >= count) { e = cudaErrorUnknown; break; }  // no progress: cannot happen
      base -= merges;
      count = next;
      cur = 1 - cur;
      ++rounds;
    }
    if (e == cudaSuccess && base != -1) e = cudaErrorUnknown;
  }
  tfree(cid[0], st); tfree(cid[1], st); tfree(blo[0], st); tfree(blo[1], st); tfree(bhi[0], st); tfree(bhi[1], st);
  tfree(nn, st); tfree(mflag, st); tfree(kflag, st); tfree(mrank, st); tfree(kpos, st); tfree(tail, st);
  return e;
}

// ---- collapse of the binary tree into a 4-wide BVH ----------------------------------
// Top down, one tree level of 4-wide nodes per launch: a node starts from the
// two children of its binary node and repeatedly opens the inner child with
// the largest surface area until it has four children or only leaves.  The
// children that stay inner become the next level's work; siblings get
// consecutive node indices.
// parent / owner (or nullptr): parent node of each new node, node holding each primitive leaf
__global__ void k_collapse4(const BVHNode* __restrict__ bin, const int2* __restrict__ work, int n_work,
                            BVH4Node* out, int2* next_work, int* counters, int* parent, int* owner) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < n_work; w += gridDim.x * blockDim.x) {
    int2 it = work[w];
    BVHNode b = bin[it.x];
    int ref[4];
    float3 lo[4], hi[4];
    ref[0] = b.ch.x;
    lo[0] = f3(b.a.x, b.a.z, b.c.x);
    hi[0] = f3(b.a.y, b.a.w, b.c.y);
    ref[1] = b.ch.y;
    lo[1] = f3(b.b.x, b.b.z, b.c.z);
    hi[1] = f3(b.b.y, b.b.w, b.c.w);
    int cnt = 2;
    while (cnt < 4) {
      int best = -1;
      float barea = -1.0f;
      for (int i = 0; i < cnt; ++i)
        if (ref[i] >= 0) {
          float a = half_area(lo[i], hi[i]);
          if (a > barea) { barea = a; best = i; }
        }
      if (best < 0) break;
      BVHNode cb = bin[ref[best]];
      ref[best] = cb.ch.x;
      lo[best] = f3(cb.a.x, cb.a.z, cb.c.x);
      hi[best] = f3(cb.a.y, cb.a.w, cb.c.y);
      ref[cnt] = cb.ch.y;
      lo[cnt] = f3(cb.b.x, cb.b.z, cb.c.z);
      hi[cnt] = f3(cb.b.y, cb.b.w, cb.c.w);
      ++cnt;
    }
    int k = 0;
    for (int i = 0; i < cnt; ++i) k += ref[i] >= 0;
    int base = k ? atomicAdd(&counters[0], k) : 0;
    int wb = k ? atomicAdd(&counters[1], k) : 0;
    float L[3][4], H[3][4];
    int R[4];
    int j = 0;
    for (int i = 0; i < 4; ++i) {
      if (i < cnt) {
        L[0][i] = lo[i].x; L[1][i] = lo[i].y; L[2][i] = lo[i].z;
        H[0][i] = hi[i].x; H[1][i] = hi[i].y; H[2][i] = hi[i].z;
        if (ref[i] >= 0) {
          R[i] = base + j;
          next_work[wb + j] = make_int2(ref[i], base + j);
          if (parent) parent[base + j] = it.y;
          ++j;
        } else {
          R[i] = ref[i];
          if (owner) owner[~ref[i]] = it.y;
        }
      } else {
        // an empty slot holds the inverted infinite box, which every slab
        // test misses (entry +inf, exit -inf whatever the ray's octant)
        L[0][i] = L[1][i] = L[2][i] = INFINITY;
        H[0][i] = H[1][i] = H[2][i] = -INFINITY;
        R[i] = kEmptyChild;
      }
    }
    BVH4Node o;
    o.lox = make_float4(L[0][0], L[0][1], L[0][2], L[0][3]);
    o.hix = make_float4(H[0][0], H[0][1], H[0][2], H[0][3]);
    o.loy = make_float4(L[1][0], L[1][1], L[1][2], L[1][3]);
    o.hiy = make_float4(H[1][0], H[1][1], H[1][2], H[1][3]);
    o.loz = make_float4(L[2][0], L[2][1], L[2][2], L[2][3]);
    o.hiz = make_float4(H[2][0], H[2][1], H[2][2], H[2][3]);
    o.ch = make_int4(R[0], R[1], R[2], R[3]);
    o.pad = make_float4(0, 0, 0, 0);
    out[it.y] = o;
  }
}

static cudaError_t collapse4(const BVHNode* bin, int n_bin, BVH4Node* out, cudaStream_t st, int* n_out, int* parent,
                             int* owner) {
  int2 *w0 = nullptr, *w1 = nullptr;
  int* cnt = nullptr;
  cudaError_t e = cudaSuccess;
  if (!talloc(&w0, 8ull * (n_bin + 1), st) || !talloc(&w1, 8ull * (n_bin + 1), st) || !talloc(&cnt, 8, st)) {
    tfree(w0, st); tfree(w1, st); tfree(cnt, st);
    return cudaErrorMemoryAllocation;
  }
  int2 root = make_int2(0, 0);
  int init[2] = {1, 0};
  cudaMemcpyAsync(w0, &root, 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(cnt, init, 8, cudaMemcpyHostToDevice, st);
  int n_work = 1;
  int* h = readback_words();  // pinned: one small asynchronous readback per level
  if (!h) {
    tfree(w0, st); tfree(w1, st); tfree(cnt, st);
    return cudaErrorMemoryAllocation;
  }
  h[0] = 1;
  h[1] = 0;
  while (n_work > 0) {
    int blocks = (n_work + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_collapse4<<<blocks, 256, 0, st>>>(bin, w0, n_work, out, w1, cnt, parent, owner);
    cudaMemcpyAsync(h, cnt, 8, cudaMemcpyDeviceToHost, st);
    cudaMemsetAsync(cnt + 1, 0, 4, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) break;
    n_work = h[1];
    int2* t = w0; w0 = w1; w1 = t;
  }
  *n_out = h[0];
  tfree(w0, st); tfree(w1, st); tfree(cnt, st);
  return e;
}

// Surface-area sums of a 4-wide tree: out[0] += area of every inner child box,
// out[1] += area of every leaf box, out[2] = area of the root's children's
// union (one thread).  Over the root area they are the expected node visits
// (besides the root) and primitive tests of a ray that meets the scene box,
// for rays uniform in space and direction (MacDonald and Booth's surface area
// heuristic).
__device__ __forceinline__ float box_area(float lx, float hx, float ly, float hy, float lz, float hz) {
  float dx = fmaxf(hx - lx, 0.0f), dy = fmaxf(hy - ly, 0.0f), dz = fmaxf(hz - lz, 0.0f);
  return 2.0f * (dx * dy + dy * dz + dz * dx);
}

__global__ void k_bvh4_area(const BVH4Node* __restrict__ nodes, int n4, double* out) {
  double inner = 0.0, leaf = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
    const BVH4Node nd = nodes[i];
    for (int c = 0; c < 4; ++c) {
      int ref = comp4i(nd.ch, c);
      if (ref == kEmptyChild) continue;
      double a = box_area(comp4(nd.lox, c), comp4(nd.hix, c), comp4(nd.loy, c), comp4(nd.hiy, c),
                          comp4(nd.loz, c), comp4(nd.hiz, c));
      if (ref >= 0) inner += a;
      else leaf += a;
    }
  }
  atomicAdd(out, inner);
  atomicAdd(out + 1, leaf);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const BVH4Node r = nodes[0];
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    for (int c = 0; c < 4; ++c) {
      if (comp4i(r.ch, c) == kEmptyChild) continue;
      lo[0] = fminf(lo[0], comp4(r.lox, c)); hi[0] = fmaxf(hi[0], comp4(r.hix, c));
      lo[1] = fminf(lo[1], comp4(r.loy, c)); hi[1] = fmaxf(hi[1], comp4(r.hiy, c));
      lo[2] = fminf(lo[2], comp4(r.loz, c)); hi[2] = fmaxf(hi[2], comp4(r.hiz, c));
    }
    out[2] = box_area(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]);
  }
}

cudaError_t bvh_area_sums(const neb_ctx* c, double out[3]) {
  double* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, 3 * sizeof(double), c->stream);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(d, 0, 3 * sizeof(double), c->stream);
  int blocks = (c->n_nodes4 + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_bvh4_area<<<blocks > 0 ? blocks : 1, 256, 0, c->stream>>>(c->nodes, c->n_nodes4, d);
  cudaMemcpyAsync(out, d, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d, c->stream);
  return cudaStreamSynchronize(c->stream);
}

__global__ void k_lift(int* node_of_prim, const int* __restrict__ parent, int n, int n_nodes, int lift) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    int nd = node_of_prim[p];
    for (int l = 0; l < lift && nd > 0 && nd < n_nodes; ++l) nd = parent[nd];
    node_of_prim[p] = nd > 0 && nd < n_nodes ? nd : 0;
  }
}

cudaError_t build_bvh(neb_ctx* c) {
  int n = c->nt + c->ns;
  if (c->nodes) { cudaFree(c->nodes); c->nodes = nullptr; }
  if (c->prim_start) { cudaFree(c->prim_start); c->prim_start = nullptr; }
  if (n == 0) return cudaSuccess;
  int* parent = nullptr;
  cudaError_t e = build_bvh4(scene_view(c), n, c->cfg.bvh_builder, c->stream, &c->nodes, &c->n_nodes4, &parent,
                             &c->prim_start);
  if (e == cudaSuccess) {
    // each primitive's leaf node, lifted in place to the subtree shadow walks start in
    int blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_lift<<<blocks, 256, 0, c->stream>>>(c->prim_start, parent, n, c->n_nodes4, kShadowLift);
    e = cudaStreamSynchronize(c->stream);
  }
  cudaFree(parent);
  return e;
}

cudaError_t build_bvh4(const SceneView& s, int n, int builder, cudaStream_t st, BVH4Node** nodes_out, int* n4_out,
                       int** parent_out, int** owner_out) {
  BVH4Node* nodes = nullptr;
  cudaError_t e = cudaMalloc(&nodes, sizeof(BVH4Node) * (size_t)(n > 1 ? n - 1 : 1));
  if (e != cudaSuccess) return e;
  *nodes_out = nodes;
  *n4_out = 1;
  int *parent = nullptr, *owner = nullptr;
  if (parent_out && owner_out) {
    e = cudaMalloc(&parent, sizeof(int) * (size_t)(n > 1 ? n - 1 : 1));
    if (e != cudaSuccess) return e;
    *parent_out = parent;
    e = cudaMalloc(&owner, sizeof(int) * (size_t)n);
    if (e != cudaSuccess) return e;
    *owner_out = owner;
    cudaMemsetAsync(parent, 0xff, sizeof(int), st);  // the root has no parent
  }
  if (n == 1) {
    k_single_leaf<<<1, 1, 0, st>>>(s, nodes);
    if (owner) cudaMemsetAsync(owner, 0, sizeof(int), st);
    return cudaGetLastError();
  }
  // the binary tree (LBVH or PLOC) is built first and collapsed into the 4-wide one
  BVHNode* bin = nullptr;
  if (!talloc(&bin, sizeof(BVHNode) * (size_t)(n - 1), st)) return cudaErrorMemoryAllocation;
  int nblocks = (n + kSortThreads - 1) / kSortThreads;
  size_t hist_n = (size_t)16 * nblocks;
  uint32_t *k0 = nullptr, *k1 = nullptr, *khi = nullptr;
  int *v0 = nullptr, *v1 = nullptr, *hist = nullptr, *offs = nullptr, *cb = nullptr;
  int2* child = nullptr;
  int *pint = nullptr, *pleaf = nullptr, *flags = nullptr;
  Box6* boxes = nullptr;
  Scratch sc;
  sc.n = scan_scratch_ints(hist_n);
  bool ok = talloc(&k0, 4ull * n, st) && talloc(&k1, 4ull * n, st) && talloc(&khi, 4ull * n, st) &&
            talloc(&v0, 4ull * n, st) && talloc(&v1, 4ull * n, st) && talloc(&hist, 4ull * hist_n, st) &&
            talloc(&offs, 4ull * hist_n, st) && talloc(&cb, 4ull * 6, st) && talloc(&child, 8ull * (n - 1), st) &&
            talloc(&pint, 4ull * (n - 1), st) && talloc(&pleaf, 4ull * n, st) && talloc(&flags, 4ull * (n - 1), st) &&
            talloc(&boxes, sizeof(Box6) * (size_t)(n - 1), st) && talloc(&sc.data, 4ull * sc.n, st);
  if (ok) {
    int init[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000, (int)0x80000000};
    cudaMemcpyAsync(cb, init, sizeof(init), cudaMemcpyHostToDevice, st);
    int gb = (n + 255) / 256;
    if (gb > 152 * 16) gb = 152 * 16;
    k_centroid_bounds<<<gb, 256, 0, st>>>(s, n, cb);
    k_morton<<<gb, 256, 0, st>>>(s, n, cb, khi, k0, v0);
    auto sort32 = [&](int bits) {  // stable LSD passes over (k0, v0); an even count leaves them in k0, v0
      for (int shift = 0; shift < bits; shift += 4) {
        k_digit_hist<<<nblocks, kSortThreads, 0, st>>>(k0, n, shift, nblocks, hist);
        scan_exclusive(hist, offs, hist_n, sc, st);
        k_digit_scatter<<<nblocks, kSortThreads, 0, st>>>(k0, v0, n, shift, nblocks, offs, k1, v1);
        uint32_t* tk = k0; k0 = k1; k1 = tk;
        int* tv = v0; v0 = v1; v1 = tv;
      }
    };
    sort32(32);                                              // by the low 32 bits
    k_gather_keys<<<gb, 256, 0, st>>>(khi, v0, n, k0);        // the high keys in that order
    sort32(30);                                              // stably by the high 30 bits
    if (builder == 1) {
      cudaMemsetAsync(pint, 0xff, 4ull * (n - 1), st);
      cudaMemsetAsync(flags, 0, 4ull * (n - 1), st);
      k_karras<<<gb, 256, 0, st>>>(k0, n, child, pint, pleaf);
      k_bounds<<<gb, 256, 0, st>>>(s, n, v0, child, pint, pleaf, flags, boxes);
      k_write_nodes<<<gb, 256, 0, st>>>(s, n, v0, child, boxes, bin);
      e = cudaStreamSynchronize(st);
    } else {
      Scratch sc2;
      sc2.n = scan_scratch_ints(n);
      e = talloc(&sc2.data, 4ull * sc2.n, st) ? cudaSuccess : cudaErrorMemoryAllocation;
      if (e == cudaSuccess) e = ploc_build(s, n, v0, bin, sc2, st);
      tfree(sc2.data, st);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    int n4 = 0;
    if (e == cudaSuccess) e = collapse4(bin, n - 1, nodes, st, &n4, parent, owner);
    *n4_out = n4;
  } else {
    e = cudaErrorMemoryAllocation;
  }
  tfree(k0, st); tfree(k1, st); tfree(khi, st); tfree(v0, st); tfree(v1, st); tfree(hist, st); tfree(offs, st);
  tfree(cb, st); tfree(child, st); tfree(pint, st); tfree(pleaf, st); tfree(flags, st); tfree(boxes, st);
  tfree(sc.data, st);
  tfree(bin, st);
  cudaStreamSynchronize(st);
  return e;
}

// ---- component kernels -------------------------------------------------------------
__global__ void k_trace_debug(SceneView s, const float* __restrict__ rays, int n, int* prim, float* tout,
                              uint32_t* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    RayPre r = make_ray(f3(rays[6 * i], rays[6 * i + 1], rays[6 * i + 2]),
                        f3(rays[6 * i + 3], rays[6 * i + 4], rays[6 * i + 5]));
    float t;
    uint32_t visits = 0, ptests = 0;
    int p = trace_closest(s, r, FLT_MAX, t, status, visits, ptests);
    prim[i] = p;
    tout[i] = p >= 0 ? t : __int_as_float(0x7f800000);
  }
}

cudaError_t launch_trace_debug(const SceneView& s, const float* d_rays, int n, int* d_prim, float* d_t,
                               uint32_t* d_status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_trace_debug<<<(n + 127) / 128, 128, 0, st>>>(s, d_rays, n, d_prim, d_t, d_status);
  return cudaGetLastError();
}

__global__ void k_philox(const uint4* __restrict__ ctr, int n, uint2 key, uint4* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = philox4x32_10(ctr[i], key);
}

cudaError_t launch_philox(const uint32_t* d_ctr, int n, uint2 key, uint32_t* d_out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_philox<<<(n + 255) / 256, 256, 0, st>>>(reinterpret_cast<const uint4*>(d_ctr), n, key,
                                            reinterpret_cast<uint4*>(d_out));
  return cudaGetLastError();
}

__global__ void k_area(const float* __restrict__ boxes, const float* __restrict__ pos, const float* __restrict__ nrm,
                       int n, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double lo[3] = {boxes[6 * i], boxes[6 * i + 1], boxes[6 * i + 2]};
    const double hi[3] = {boxes[6 * i + 3], boxes[6 * i + 4], boxes[6 * i + 5]};
    const double p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    const float q[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
    out[i] = plane_box_area64(lo, hi, p, q);
  }
}

cudaError_t launch_area(const float* d_boxes, const float* d_pos, const float* d_nrm, int n, double* d_out,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_area<<<(n + 255) / 256, 256, 0, st>>>(d_boxes, d_pos, d_nrm, n, d_out);
  return cudaGetLastError();
}

}  // namespace neb
