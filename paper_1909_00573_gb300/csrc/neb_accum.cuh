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

}  // namespace neb
