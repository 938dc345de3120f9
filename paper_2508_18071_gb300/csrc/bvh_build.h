// Host-side records shared by the BVH builders (host C++ and GPU).
#pragma once
#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include "et_internal.cuh"

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

// Device buffer of the builders, grown on demand and freed with the builder.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;
  int ensure(size_t n) {
    if (n <= cap) return ET_OK;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    ET_CHECK_CUDA(cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)));
    cap = n;
    return ET_OK;
  }
  ~DevBuf() { cudaFree(p); }
};

// GPU full-sweep SAH build (the host sweep's algorithm and node order):
// node list (node 0 = root), the triangle permutation in leaf order and the
// tree depth.  ET_ERR_UNIMPLEMENTED if the tree is deeper than the traversal
// stack.
int gpu_sweep_sah(const float* tris, int64_t n, cudaStream_t stream, std::vector<BuildNode>& nodes,
                  std::vector<int>& perm, int& max_depth);

// GPU binned-SAH build of n triangles (host array [n][9]): fills the node list
// (node 0 = root), the triangle permutation in leaf order and the tree depth.
int gpu_binned_sah(const float* tris, int64_t n, cudaStream_t stream, std::vector<BuildNode>& nodes,
                   std::vector<int>& perm, int& max_depth);
