// Moving geometry: new triangle positions for a built scene, with the
// hierarchy refitted (same topology, boxes recomputed bottom-up).
//
// The paper's scenes are mostly static with a moving camera; objects that move
// (rigidly or not) between frames need only new bounds, not a new tree, as
// long as the motion is small against the scene: the triangle records are
// rewritten in leaf order from the caller's input-order array, then the inner
// nodes are refitted one depth level at a time, deepest first, each node taking
// its children's boxes from its leaf triangles or from the child node's record.
// Boxes are float minima / maxima of the float vertices: exact, so the
// traversal's conservative culling and the closest-hit tie rule are unchanged.
#include <cfloat>
#include "et_internal.cuh"
#include "scene_internal.h"

namespace {

// slot s of the leaf-ordered records takes input triangle perm[s]'s vertices
// (light triangles, which follow the user triangles, stay)
__global__ void scatter_tris(const float* __restrict__ upd, const int32_t* __restrict__ perm,
                             int64_t n_slots, int64_t n_user, float4* __restrict__ tris) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  const int32_t t = perm[s];
  if (t >= n_user) return;
  const float* v = upd + 9 * (int64_t)t;
  float4* r = tris + 3 * s;
  const float4 a = r[0], b = r[1], c = r[2];
  r[0] = make_float4(v[0], v[1], v[2], a.w);
  r[1] = make_float4(v[3], v[4], v[5], b.w);
  r[2] = make_float4(v[6], v[7], v[8], c.w);
}

struct B6 { float lo[3], hi[3]; };

__device__ __forceinline__ B6 child_box(const BvhNode* nodes, const float4* tris, int ref) {
  B6 b;
  if (ref >= 0) {
    const BvhNode n = nodes[ref];
    b.lo[0] = fminf(n.a.x, n.b.z); b.lo[1] = fminf(n.a.y, n.b.w); b.lo[2] = fminf(n.a.z, n.c.x);
    b.hi[0] = fmaxf(n.a.w, n.c.y); b.hi[1] = fmaxf(n.b.x, n.c.z); b.hi[2] = fmaxf(n.b.y, n.c.w);
    return b;
  }
  const int v = -ref - 1;
  const int first = v >> 3, cnt = v & 7;
  for (int k = 0; k < 3; ++k) { b.lo[k] = FLT_MAX; b.hi[k] = -FLT_MAX; }
  for (int i = 0; i < cnt; ++i) {
    const float4* t = tris + 3 * (int64_t)(first + i);
    for (int j = 0; j < 3; ++j) {
      const float4 p = t[j];
      b.lo[0] = fminf(b.lo[0], p.x); b.lo[1] = fminf(b.lo[1], p.y); b.lo[2] = fminf(b.lo[2], p.z);
      b.hi[0] = fmaxf(b.hi[0], p.x); b.hi[1] = fmaxf(b.hi[1], p.y); b.hi[2] = fmaxf(b.hi[2], p.z);
    }
  }
  return b;
}

__global__ void refit_level(BvhNode* __restrict__ nodes, const float4* __restrict__ tris,
                            const int32_t* __restrict__ order, int begin, int end) {
  const int i = begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= end) return;
  BvhNode& n = nodes[order[i]];
  const int4 d = n.d;
  const B6 l = child_box(nodes, tris, d.x), r = child_box(nodes, tris, d.y);
  n.a = make_float4(l.lo[0], l.lo[1], l.lo[2], l.hi[0]);
  n.b = make_float4(l.hi[1], l.hi[2], r.lo[0], r.lo[1]);
  n.c = make_float4(r.lo[2], r.hi[0], r.hi[1], r.hi[2]);
}

}  // namespace

extern "C" int et_scene_update(et_scene* s, const float* tris, void* stream_) {
  if (!s || (!tris && s->n_user > 0)) return ET_ERR_ARG;
  if (s->n_user == 0) return ET_OK;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!s->d_upd) {
    const cudaError_t e = cudaMalloc((void**)&s->d_upd, sizeof(float) * 9 * (size_t)s->n_user);
    if (e != cudaSuccess) {
      et_set_last_cuda_error(e);
      s->d_upd = nullptr;
      return e == cudaErrorMemoryAllocation ? ET_ERR_OOM : ET_ERR_CUDA;
    }
  }
  ET_CHECK_CUDA(cudaMemcpyAsync(s->d_upd, tris, sizeof(float) * 9 * (size_t)s->n_user,
                                cudaMemcpyHostToDevice, stream));
  scatter_tris<<<(unsigned)((s->n_tris + 255) / 256), 256, 0, stream>>>(s->d_upd, s->d_perm, s->n_tris,
                                                                        s->n_user, s->d_tris);
  ET_CHECK_LAUNCH();
  for (size_t k = 0; k + 1 < s->refit_levels.size(); ++k) {
    const int b = s->refit_levels[k], e = s->refit_levels[k + 1];
    if (e <= b) continue;
    refit_level<<<(unsigned)((e - b + 127) / 128), 128, 0, stream>>>(s->d_nodes, s->d_tris, s->d_refit, b, e);
    ET_CHECK_LAUNCH();
  }
  return ET_OK;
}
