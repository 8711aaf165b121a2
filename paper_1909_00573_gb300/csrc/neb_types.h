// neb_types.h -- plain data types shared by the host and device code of libneb.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/neb.h"

namespace neb {

enum { MAT_DIFFUSE = 0, MAT_DIELECTRIC = 1, MAT_GGX = 2 };

// BVH2 node, 64 bytes, read with four 128-bit loads:
//   [0] left  child box  (lo.x, hi.x, lo.y, hi.y)
//   [1] right child box  (lo.x, hi.x, lo.y, hi.y)
//   [2] (left lo.z, left hi.z, right lo.z, right hi.z)
//   [3] (left, right, -, -): >= 0 internal node index, < 0 ~primitive (leaf)
struct __align__(16) BVHNode {
  float4 a, b, c;
  int4 ch;
};

// BVH4 node, 128 bytes (eight 128-bit loads): per axis the low and high
// bounds of the four children, then the four child links (>= 0 node index,
// < 0 ~primitive, kEmptyChild for an unused slot).
struct __align__(16) BVH4Node {
  float4 lox, hix, loy, hiy, loz, hiz;
  int4 ch;
  float4 pad;
};
constexpr int kEmptyChild = (int)0x80000000;

// Octree globals of Appendix B (initialize / set_iteration), device resident.
struct OctreeParams {
  float minb[3], size_inv[3], scene_scale;
  int capacity;
  int split_count;   // SPLIT_FACTOR * min(iter, 1000)
  int iter_clamp;
  int stop_filling;
  int init_value;    // ceil(SPLIT_FACTOR / 4 * iter)
};

struct OctreeState {  // device memory
  int alloc;
  int depth;
  uint32_t status;
  int pad;
};

constexpr int kMaxDepth = 64;
constexpr int kOctMaxDepth = 30;
constexpr int kFillIterations = 1000;
constexpr int kSpinLimit = 1 << 20;

}  // namespace neb
