// Internal definitions shared by the translation units of libeventtracer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include "../../include/eventtracer.h"

#define ET_CHECK_CUDA(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) {                                  \
      et_set_last_cuda_error(_e);                             \
      return _e == cudaErrorMemoryAllocation ? ET_ERR_OOM : ET_ERR_CUDA; \
    }                                                         \
  } while (0)

// every kernel launch of the library is followed by this: counts it, checks it
#define ET_CHECK_LAUNCH()           \
  do {                              \
    et_count_launch();              \
    ET_CHECK_CUDA(cudaGetLastError()); \
  } while (0)

void et_count_launch();

void et_set_last_cuda_error(cudaError_t e);

// --------------------------------------------------------------- scene layout
// Triangles are stored in BVH leaf order as three float4: (v0, prim id bits),
// (v1, material bits), (v2, 0).  Light triangles carry material LIGHT_BIT | light.
#define ET_LIGHT_BIT 0x80000000u
constexpr int kMaxBvhDepth = 64;   // traversal stack entries (one pending subtree per level)

// BVH2 node: both children's boxes plus their references (64 bytes).
// child reference >= 0: inner node index; < 0: leaf, v = -ref - 1,
// first triangle = v >> 3, count = v & 7.
struct __align__(16) BvhNode {
  float4 a;   // c0.lo.x c0.lo.y c0.lo.z c0.hi.x
  float4 b;   // c0.hi.y c0.hi.z c1.lo.x c1.lo.y
  float4 c;   // c1.lo.z c1.hi.x c1.hi.y c1.hi.z
  int4 d;     // c0 ref, c1 ref, 0, 0
};

struct DevLight {
  float p0[3], e1[3], e2[3], n[3], L[3];
  float area, prob, cdf;
};

struct DevMaterial {
  float albedo[3];
  float roughness;
  int type;
  int pad[3];
};

struct et_scene_dev {
  const float4* tris;        // [n][3]
  const BvhNode* nodes;
  const DevMaterial* mats;
  const DevLight* lights;
  int n_lights;
  int root_ref;
  float env;
  int64_t n_tris;
};

// -------------------------------------------------------------- small vectors
struct f3 { float x, y, z; };
__host__ __device__ inline f3 mk(float x, float y, float z) { f3 r; r.x = x; r.y = y; r.z = z; return r; }
__host__ __device__ inline f3 operator+(f3 a, f3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ inline f3 operator-(f3 a, f3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ inline f3 operator*(f3 a, float s) { return mk(a.x * s, a.y * s, a.z * s); }
__host__ __device__ inline f3 operator*(f3 a, f3 b) { return mk(a.x * b.x, a.y * b.y, a.z * b.z); }
__host__ __device__ inline f3 operator-(f3 a) { return mk(-a.x, -a.y, -a.z); }
__host__ __device__ inline float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline f3 cross(f3 a, f3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline f3 normalize(f3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__host__ __device__ inline float comp(f3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ------------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64-bit
// products with multipliers 0xD2511F53 and 0xCD9E8D57; key bumped by the Weyl
// increments 0x9E3779B9 and 0xBB67AE85 between rounds.
struct u4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  u4 r; r.x = c0; r.y = c1; r.z = c2; r.w = c3;
  return r;
}

// 24 random bits -> float in [0, 1), exactly representable
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }
