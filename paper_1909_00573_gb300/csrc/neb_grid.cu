// neb_grid.cu -- device-wide exclusive scan and the hashed grid over the
// mergeable view vertices (the spatial structure of the inverted merge
// search, Sec. 3.2): cell size 2r, counting sort of vertex records into
// buckets so that a photon's r-ball touches at most 8 cells.
#include <cuda_runtime.h>

#include "neb_accum.cuh"
#include "neb_device.cuh"
#include "neb_internal.h"

namespace neb {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 1024 elements per block

// Block-local exclusive scan of a 1024-element tile; block totals go to `sums`.
__global__ void k_scan_tiles(const int* __restrict__ in, int* __restrict__ out, size_t n, int* __restrict__ sums) {
  __shared__ int warp_tot[kScanThreads / 32];
  size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int run = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int x = (base + j < n) ? in[base + j] : 0;
    v[j] = run;
    run += x;
  }
  // warp inclusive scan of the per-thread totals
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive
    if (lane == kScanThreads / 32 - 1 && sums) sums[blockIdx.x] = wi;
  }
  __syncthreads();
  int off = warp_tot[warp] + incl - run;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j)
    if (base + j < n) out[base + j] = v[j] + off;
}

__global__ void k_scan_add(int* __restrict__ out, size_t n, const int* __restrict__ offs) {
  size_t base = (size_t)blockIdx.x * kScanTile;
  int o = offs[blockIdx.x];
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads)
    if (base + j < n) out[base + j] += o;
}

int scan_launch_count(size_t n) {
  size_t nb = (n + kScanTile - 1) / kScanTile;
  return nb <= 1 ? 1 : 2 + scan_launch_count(nb);
}

size_t scan_scratch_ints(size_t n) {
  size_t total = 0;
  while (n > (size_t)kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    total += 2 * n + 2;
  }
  return total + 16;
}

static cudaError_t scan_rec(const int* in, int* out, size_t n, int* scratch, cudaStream_t st) {
  size_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb <= 1) {
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
    return cudaGetLastError();
  }
  int* sums = scratch;
  int* sums_scan = scratch + nb;
  k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums);
  cudaError_t e = scan_rec(sums, sums_scan, nb, scratch + 2 * nb + 2, st);
  if (e != cudaSuccess) return e;
  k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, sums_scan);
  return cudaGetLastError();
}

cudaError_t scan_exclusive(const int* d_in, int* d_out, size_t n, Scratch& scratch, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (scratch.n < scan_scratch_ints(n)) return cudaErrorInvalidValue;
  return scan_rec(d_in, d_out, n, scratch.data, st);
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t point_bucket(float3 p, float3 gmin, float cell_inv, uint32_t mask) {
  int cx = grid_cell_index((p.x - gmin.x) * cell_inv);
  int cy = grid_cell_index((p.y - gmin.y) * cell_inv);
  int cz = grid_cell_index((p.z - gmin.z) * cell_inv);
  return grid_hash(cx, cy, cz, mask);
}

__global__ void k_grid_count(NeeStore nv, DevCounters* cnt, int cap, float3 gmin, float cell_inv, uint32_t mask,
                             int* __restrict__ bucket_count, int* __restrict__ vert_bucket, uint32_t* cell_bits,
                             uint32_t bits_mask) {
  int count = min(cnt->nee_count, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    int bits = __float_as_int(nv.nrm[i].w);
    int b = -1;
    if ((bits >> NV_FLAG_SHIFT) & NV_MERGEABLE) {
      const float3 p = xyz(nv.pos[i]);
      const int cx = grid_cell_index((p.x - gmin.x) * cell_inv), cy = grid_cell_index((p.y - gmin.y) * cell_inv),
                cz = grid_cell_index((p.z - gmin.z) * cell_inv);
      b = (int)grid_hash(cx, cy, cz, mask);
      atomicAdd(bucket_count + b, 1);
      const uint32_t h = cell_bit_index(cx, cy, cz, bits_mask);
      const uint32_t bit = 1u << (h & 31u);
      if (!(cell_bits[h >> 5] & bit)) atomicOr(cell_bits + (h >> 5), bit);
    }
    vert_bucket[i] = b;
  }
}

// Writes each record into its bucket range; the counts are consumed back to
// zero, leaving bucket_count ready for the next iteration.
__global__ void k_grid_scatter(NeeStore nv, DevCounters* cnt, int cap, const int* __restrict__ vert_bucket,
                               const int* __restrict__ bucket_start, int* bucket_count, MergeRec* __restrict__ out) {
  int count = min(cnt->nee_count, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    int b = vert_bucket[i];
    if (b < 0) continue;
    int slot = bucket_start[b] + atomicSub(bucket_count + b, 1) - 1;
    float4 p = nv.pos[i];
    out[slot].pos = make_float4(p.x, p.y, p.z, __int_as_float(i));
  }
}

cudaError_t grid_build(neb_ctx* c, const IterParams& ip, const IterSlot& sl, cudaStream_t st) {
  const int B = capped_blocks(c->cap_nee, 256, 152 * 8);
  cudaMemsetAsync(c->cell_bits, 0, sizeof(uint32_t) * (size_t)c->table_size, st);
  k_grid_count<<<B, 256, 0, st>>>(sl.nv, sl.cnt, c->cap_nee, ip.gmin, ip.cell_inv, ip.table_mask, c->bucket_count,
                                  c->vert_bucket, c->cell_bits, ip.cell_bits_mask);
  cudaError_t e = scan_exclusive(c->bucket_count, c->bucket_start, (size_t)c->table_size + 1, c->scan_scratch, st);
  if (e != cudaSuccess) return e;
  k_grid_scatter<<<B, 256, 0, st>>>(sl.nv, sl.cnt, c->cap_nee, c->vert_bucket, c->bucket_start, c->bucket_count,
                                    c->mrec);
  return cudaGetLastError();
}

// ---- stand-alone neighbour counting through the same grid -------------------
__global__ void k_pts_count(const float* __restrict__ pts, int n, float3 gmin, float cell_inv, uint32_t mask,
                            int* bucket_count, int* vb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t b = point_bucket(f3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]), gmin, cell_inv, mask);
    vb[i] = (int)b;
    atomicAdd(bucket_count + b, 1);
  }
}

__global__ void k_pts_scatter(const float* __restrict__ pts, int n, const int* vb, const int* bucket_start,
                              int* bucket_count, float4* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int b = vb[i];
    int slot = bucket_start[b] + atomicSub(bucket_count + b, 1) - 1;
    out[slot] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], 0.0f);
  }
}

__global__ void k_pts_query(const float4* __restrict__ sorted, const int* __restrict__ bucket_start,
                            const float* __restrict__ q, int m, float r2, float3 gmin, float cell_inv, uint32_t mask,
                            int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    float3 hp = f3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
    float gx = (hp.x - gmin.x) * cell_inv, gy = (hp.y - gmin.y) * cell_inv, gz = (hp.z - gmin.z) * cell_inv;
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
      for (int e = bucket_start[bk[c]]; e < bucket_start[bk[c] + 1]; ++e) {
        float4 p = sorted[e];
        float dx = p.x - hp.x, dy = p.y - hp.y, dz = p.z - hp.z;
        if (dx * dx + dy * dy + dz * dz <= r2) ++cnt;
      }
    }
    out[i] = cnt;
  }
}

cudaError_t build_point_grid(const float* d_pts, int n, float cell, float3 gmin, uint32_t table, int* bucket_count,
                             int* bucket_start, int* vert_bucket, float4* sorted, Scratch& sc, cudaStream_t st) {
  const int nb = capped_blocks(n, 256, 152 * 8);
  if (n > 0) k_pts_count<<<nb, 256, 0, st>>>(d_pts, n, gmin, 1.0f / cell, table - 1, bucket_count, vert_bucket);
  cudaError_t e = scan_exclusive(bucket_count, bucket_start, (size_t)table + 1, sc, st);
  if (e != cudaSuccess) return e;
  if (n > 0) k_pts_scatter<<<nb, 256, 0, st>>>(d_pts, n, vert_bucket, bucket_start, bucket_count, sorted);
  return cudaGetLastError();
}

cudaError_t count_neighbours_device(const float* d_pts, int n, const float* d_q, int m, float r, int* d_out,
                                    cudaStream_t st) {
  // grid origin: componentwise minimum of the points and queries, one cell below
  // (computed on the host by the caller-facing wrapper would cost a copy; the
  // hash makes any fixed origin work, so use the origin of the coordinates)
  uint32_t table = 1024;
  while (table < (uint32_t)(2 * (n > 0 ? n : 1))) table <<= 1;
  float cs = 2.0f * r;
  float3 gmin = f3(0.0f, 0.0f, 0.0f);
  int *bc = nullptr, *bs = nullptr, *vb = nullptr;
  float4* sorted = nullptr;
  Scratch sc;
  sc.n = scan_scratch_ints(table + 1);
  cudaError_t e = cudaSuccess;
  if ((e = cudaMallocAsync(&bc, sizeof(int) * (table + 1), st)) != cudaSuccess) return e;
  cudaMallocAsync(&bs, sizeof(int) * (table + 1), st);
  cudaMallocAsync(&vb, sizeof(int) * (size_t)(n > 0 ? n : 1), st);
  cudaMallocAsync(&sorted, sizeof(float4) * (size_t)(n > 0 ? n : 1), st);
  cudaMallocAsync(&sc.data, sizeof(int) * sc.n, st);
  cudaMemsetAsync(bc, 0, sizeof(int) * (table + 1), st);
  build_point_grid(d_pts, n, cs, gmin, table, bc, bs, vb, sorted, sc, st);
  if (m > 0)
    k_pts_query<<<(m + 255) / 256, 256, 0, st>>>(sorted, bs, d_q, m, r * r, gmin, 1.0f / cs, table - 1, d_out);
  e = cudaGetLastError();
  cudaFreeAsync(bc, st);
  cudaFreeAsync(bs, st);
  cudaFreeAsync(vb, st);
  cudaFreeAsync(sorted, st);
  cudaFreeAsync(sc.data, st);
  return e;
}

}  // namespace neb

// ---------------------------------------------------------------------------
// Neighbour counting without any device allocation.
//
// Same grid and kernels as count_neighbours_device, but every scratch buffer
// (bucket counts and starts, per-point buckets, the bucket-sorted points and
// the scan's block sums) lives in one file-scope __device__ array of fixed
// size.  The array is part of the module image, so every GPU that loads the
// library holds it until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {
constexpr uint32_t kNaTable = 1u << 19;                       // hash buckets
constexpr size_t kNaCountsOff = 0;                            // int[kNaTable + 1]
constexpr size_t kNaStartsOff = (2u << 20) + 256;             // int[kNaTable + 1]
constexpr size_t kNaBucketOff = (4u << 20) + 512;             // int[NEB_NOALLOC_MAX_POINTS]
constexpr size_t kNaSortedOff = (5u << 20) + 512;             // float4[NEB_NOALLOC_MAX_POINTS]
constexpr size_t kNaScanOff = (9u << 20) + 512;               // int[kNaScanInts]
constexpr size_t kNaScanInts = 4096;
constexpr size_t kNaBytes = kNaScanOff + kNaScanInts * sizeof(int);
static_assert((kNaTable + 1) * sizeof(int) <= kNaStartsOff - kNaCountsOff, "counts");
static_assert((kNaTable + 1) * sizeof(int) <= kNaBucketOff - kNaStartsOff, "starts");
static_assert(NEB_NOALLOC_MAX_POINTS * sizeof(int) <= kNaSortedOff - kNaBucketOff, "buckets");
static_assert(NEB_NOALLOC_MAX_POINTS * sizeof(float4) <= kNaScanOff - kNaSortedOff, "sorted points");
static_assert(kNaScanInts >= 2 * ((kNaTable + 1 + 1023) / 1024) + 2 + 16, "scan block sums");

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char* g_na_addr[kNaMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol's host-side name as a pointer).
static int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return NEB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NEB_ERR_CUDA;
    g_na_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_addr[dev];
  return NEB_OK;
}

extern "C" int neb_count_neighbours_noalloc(const float* d_pts, int n, const float* d_queries, int m, float r,
                                            int32_t* d_out, void* cuda_stream) {
  if (n < 0 || m < 0 || !(r > 0.0f) || (n > 0 && !d_pts) || (m > 0 && (!d_queries || !d_out)))
    return NEB_ERR_ARG;
  if (n > NEB_NOALLOC_MAX_POINTS) return NEB_ERR_ARG;
  if (m == 0) return NEB_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (st) {  // the scratch address is the current device's: the stream must be on it
    int dev = 0, sdev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess) return NEB_ERR_CUDA;
    if (sdev != dev) return NEB_ERR_ARG;
  }
  unsigned char* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != NEB_OK) return rc;
  int* counts = reinterpret_cast<int*>(base + kNaCountsOff);
  int* starts = reinterpret_cast<int*>(base + kNaStartsOff);
  int* vb = reinterpret_cast<int*>(base + kNaBucketOff);
  float4* sorted = reinterpret_cast<float4*>(base + kNaSortedOff);
  neb::Scratch sc;
  sc.data = reinterpret_cast<int*>(base + kNaScanOff);
  sc.n = kNaScanInts;
  const float cs = 2.0f * r;
  const float3 gmin = neb::f3(0.0f, 0.0f, 0.0f);
  // the previous call's bucket counts are consumed to zero by its scatter, but
  // a call that failed half-way could leave them dirty: clear them every time
  if (cudaMemsetAsync(counts, 0, sizeof(int) * (kNaTable + 1), st) != cudaSuccess) return NEB_ERR_CUDA;
  if (n > 0) neb::k_pts_count<<<(n + 255) / 256, 256, 0, st>>>(d_pts, n, gmin, 1.0f / cs, kNaTable - 1, counts, vb);
  if (neb::scan_exclusive(counts, starts, kNaTable + 1, sc, st) != cudaSuccess) return NEB_ERR_CUDA;
  if (n > 0) neb::k_pts_scatter<<<(n + 255) / 256, 256, 0, st>>>(d_pts, n, vb, starts, counts, sorted);
  neb::k_pts_query<<<(m + 255) / 256, 256, 0, st>>>(sorted, starts, d_queries, m, r * r, gmin, 1.0f / cs,
                                                    kNaTable - 1, d_out);
  return cudaGetLastError() == cudaSuccess ? NEB_OK : NEB_ERR_CUDA;
}
