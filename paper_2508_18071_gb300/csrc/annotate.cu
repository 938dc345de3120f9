// Primary-hit annotations: the by-products of path tracing that come with the
// rendered events for free (depth, surface normal, segmentation ids and the
// screen-space motion of the visible point), from one ray through each pixel
// centre per frame.  One thread per (frame, pixel); the closest hit uses the
// same traversal and triangle test as the renderer.
#include <cmath>
#include "et_internal.cuh"
#include "pt_common.cuh"
#include "scene_internal.h"

namespace {

__global__ void __launch_bounds__(128)
annotate_kernel(et_scene_dev S, const et_camera* __restrict__ cams, int F, bool has_next, int W,
                int H, float* __restrict__ depth, float* __restrict__ normal,
                int32_t* __restrict__ prim, int32_t* __restrict__ material, float* __restrict__ flow) {
  const int64_t npix = (int64_t)W * H;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)F * npix) return;
  const int f = (int)(i / npix);
  const int x = (int)(i % W), y = (int)((i % npix) / W);
  const pt::Cam cam = pt::load_cam(cams[f]);
  const float px = (2.0f * ((float)x + 0.5f) / (float)W - 1.0f) * cam.th * ((float)W / (float)H);
  const float py = (1.0f - 2.0f * ((float)y + 0.5f) / (float)H) * cam.th;
  const f3 d = normalize(cam.c0 * px + cam.c1 * py - cam.c2);
  pt::Ray r;
  pt::ray_setup(r, cam.pos, d);
  const pt::Hit h = pt::traverse<false>(S, r, FLT_MAX);
  const float nan = __int_as_float(0x7FC00000);
  if (h.slot < 0) {
    if (depth) depth[i] = __int_as_float(0x7F800000);
    if (normal) { normal[3 * i] = normal[3 * i + 1] = normal[3 * i + 2] = 0.0f; }
    if (prim) prim[i] = -1;
    if (material) material[i] = -1;
    if (flow) { flow[2 * i] = nan; flow[2 * i + 1] = nan; }
    return;
  }
  const float4* tp = S.tris + 3 * (int64_t)h.slot;
  const float4 A = tp[0], B = tp[1], C = tp[2];
  if (depth) depth[i] = h.t * -dot(d, cam.c2);
  if (normal) {
    f3 n = normalize(cross(mk(B.x - A.x, B.y - A.y, B.z - A.z), mk(C.x - A.x, C.y - A.y, C.z - A.z)));
    if (dot(n, d) > 0.0f) n = n * -1.0f;
    normal[3 * i] = n.x; normal[3 * i + 1] = n.y; normal[3 * i + 2] = n.z;
  }
  if (prim) prim[i] = (int32_t)__float_as_uint(A.w);
  if (material) material[i] = (int32_t)__float_as_uint(B.w);
  if (flow) {
    float fx = nan, fy = nan;
    if (f + 1 < F || has_next) {
      const pt::Cam c2 = pt::load_cam(cams[f + 1]);
      const f3 p = cam.pos + d * h.t;
      const f3 q = p - c2.pos;
      const float a = dot(q, c2.c0), b = dot(q, c2.c1), c = dot(q, c2.c2);
      if (c < 0.0f) {
        const float qx = a / -c, qy = b / -c;
        fx = (qx / (c2.th * ((float)W / (float)H)) + 1.0f) * 0.5f * (float)W - ((float)x + 0.5f);
        fy = (1.0f - qy / c2.th) * 0.5f * (float)H - ((float)y + 0.5f);
      }
    }
    flow[2 * i] = fx;
    flow[2 * i + 1] = fy;
  }
}

}  // namespace

extern "C" int et_render_annotations(const et_scene* scene, const et_camera* cams, int32_t n_frames,
                                     const et_camera* next_cam, int32_t W, int32_t H, float* depth,
                                     float* normal, int32_t* prim, int32_t* material, float* flow,
                                     void* stream_) {
  if (!scene || (!cams && n_frames > 0) || n_frames < 0 || n_frames > 65535) return ET_ERR_ARG;
  if (W < 1 || H < 1 || W > 65535 || H > 65535) return ET_ERR_ARG;
  if (!depth && !normal && !prim && !material && !flow) return ET_ERR_ARG;
  if (n_frames == 0) return ET_OK;
  cudaStream_t stream = (cudaStream_t)stream_;
  et_scene* s = const_cast<et_scene*>(scene);
  const int need = n_frames + 1;
  if (need > s->cam_cap) {
    ET_CHECK_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->d_cams);
    s->d_cams = nullptr;
    s->cam_cap = 0;
    ET_CHECK_CUDA(cudaMalloc((void**)&s->d_cams, sizeof(et_camera) * (size_t)need));
    s->cam_cap = need;
  }
  ET_CHECK_CUDA(cudaMemcpyAsync(s->d_cams, cams, sizeof(et_camera) * (size_t)n_frames,
                                cudaMemcpyHostToDevice, stream));
  if (next_cam)
    ET_CHECK_CUDA(cudaMemcpyAsync(s->d_cams + n_frames, next_cam, sizeof(et_camera),
                                  cudaMemcpyHostToDevice, stream));
  const int64_t n = (int64_t)n_frames * W * H;
  annotate_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(
      s->dev, s->d_cams, n_frames, next_cam != nullptr, W, H, depth, normal, prim, material, flow);
  ET_CHECK_LAUNCH();
  return ET_OK;
}
