// neb_accum.cuh -- device helpers shared by the contribution kernels: the
// FP64 per-pixel sums (the progressive accumulation) and warp-summed counters.
#pragma once
#include "neb_device.cuh"

namespace neb {

// Sum of v over the warp added to *dst by lane 0 (all lanes call it).
__device__ __forceinline__ void warp_count(unsigned long long* dst, uint32_t v) {
  uint32_t s = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}

// Adds L to the FP64 sums of `pixel` and, when kept, to its strategy channel.
__device__ __forceinline__ void add_pixel(double* accum, double* split, int which, int pixel, float3 L, int P) {
  double* a = accum + (size_t)pixel * 3;
  atomicAdd(a, (double)L.x);
  atomicAdd(a + 1, (double)L.y);
  atomicAdd(a + 2, (double)L.z);
  if (split) {
    double* sp = split + ((size_t)which * P + pixel) * 3;
    atomicAdd(sp, (double)L.x);
    atomicAdd(sp + 1, (double)L.y);
    atomicAdd(sp + 2, (double)L.z);
  }
}

// Occupancy of the merge grid's cells: one bit per value of a second hash of
// the cell (independent of the bucket hash), set for every cell that holds a
// mergeable view vertex.  A search skips a cell whose bit is clear: no vertex
// lies in it, whatever other cells share its bucket.
__device__ __forceinline__ uint32_t cell_bit_index(int x, int y, int z, uint32_t mask) {
  return (((uint32_t)x * 0x9E3779B1u) ^ ((uint32_t)y * 0x85EBCA77u) ^ ((uint32_t)z * 0xC2B2AE3Du)) & mask;
}
__device__ __forceinline__ bool cell_occupied(const uint32_t* __restrict__ bits, uint32_t mask, int x, int y, int z) {
  const uint32_t h = cell_bit_index(x, y, z, mask);
  return (__ldg(bits + (h >> 5)) >> (h & 31u)) & 1u;
}

}  // namespace neb
