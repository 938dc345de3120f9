// Host-side records shared by the two BVH builders (host C++ and GPU).
#pragma once
#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

struct Box {
  float lo[3], hi[3];
  void reset() { for (int k = 0; k < 3; ++k) { lo[k] = FLT_MAX; hi[k] = -FLT_MAX; } }
  void grow(const Box& b) {
    for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], b.lo[k]); hi[k] = std::max(hi[k], b.hi[k]); }
  }
  void grow(const float* p) {
    for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], p[k]); hi[k] = std::max(hi[k], p[k]); }
  }
  double area() const {
    double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
    if (dx < 0 || dy < 0 || dz < 0) return 0.0;
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  }
};

// A node of the binary build tree: inner (count == 0, children left/right) or
// leaf (triangles perm[first .. first + count)).
struct BuildNode { Box box; int left, right, first, count; };

constexpr int kSahBins = 32;
constexpr int kLeafMax = 4;

// GPU binned-SAH build of n triangles (host array [n][9]): fills the node list
// (node 0 = root), the triangle permutation in leaf order and the tree depth.
int gpu_binned_sah(const float* tris, int64_t n, cudaStream_t stream, std::vector<BuildNode>& nodes,
                   std::vector<int>& perm, int& max_depth);
