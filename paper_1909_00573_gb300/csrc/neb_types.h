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

// Density-octree parameters, passed to the kernels by value (Sec. 5): the
// octree box (the scene box grown by 0.2 %), the word pool's size, and the
// quantities that change with the iteration.
struct OctreeParams {
  float minb[3];        // lower corner of the octree box
  float size_inv[3];    // 1 / edge length of the box, per axis (FP32)
  double box_extent[3]; // 1 / size_inv, the edge lengths the cell boxes are cut from (FP64)
  float scene_scale;    // length of the box diagonal
  int capacity;         // words in the pool, 8m + 1
  int split_count;      // a cell splits when its count reaches split_factor * min(iter, 1000)
  int iter_clamp;       // min(iter, 1000): densities are divided by it
  int stop_filling;     // iter > 1000: counting stops
  int init_value;       // count of a new cell: ceil(split_factor * iter / 4)
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
