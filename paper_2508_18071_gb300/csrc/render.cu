// et_render_frames: path tracing of the 1 kHz frames (paper Sec. 3.2).
//
// Two schedules of the same per-path arithmetic (pt_common.cuh):
//  * ET_RENDER_WAVEFRONT (default, wavefront.cu): per-bounce ray queues and
//    persistent traversal warps that refill idle lanes;
//  * ET_RENDER_MEGAKERNEL (this file): one thread per pixel runs its whole
//    paths; needs no workspace.
// Both write the frame's mean radiance and the Eq. 1 log luminance from the
// same per-path sums in the same order, so their outputs are identical.
#include "et_internal.cuh"
#include "pt_common.cuh"
#include "scene_internal.h"
#include "render_internal.h"

namespace {

__device__ __forceinline__ f3 trace_sample(const et_scene_dev& S, const pt::Cam& cam, int W, int H,
                                           int x, int y, uint32_t smp, uint32_t frame,
                                           int max_depth, uint32_t k0, uint32_t k1, int32_t* rec) {
  const uint32_t pix = (uint32_t)(y * W + x);
  f3 o, d;
  pt::camera_ray(cam, W, H, x, y, smp, frame, k0, k1, o, d);
  f3 beta = mk(1.0f, 1.0f, 1.0f), L = mk(0.0f, 0.0f, 0.0f);
  float prev_pdf = 0.0f;
  for (int b = 1; b <= max_depth; ++b) {
    pt::Ray ray;
    pt::ray_setup(ray, o, d);
    const pt::Hit h = pt::traverse<false>(S, ray, FLT_MAX);
    if (rec) rec[2 * (b - 1)] = h.slot < 0 ? -1 : (int32_t)h.prim;
    pt::Vertex v;
    if (!pt::arrive(S, o, d, h, b, max_depth, prev_pdf, beta, L, v)) break;
    if (S.n_lights > 0) {
      f3 dir, contrib;
      float tmax;
      int light;
      int32_t nrec = -1;
      if (pt::nee(S, v, pix, smp, frame, b, k0, k1, beta, dir, tmax, contrib, light)) {
        pt::Ray sr;
        pt::ray_setup(sr, v.on, dir);
        const bool vis = pt::traverse<true>(S, sr, tmax).slot < 0;
        nrec = 2 * light + (vis ? 1 : 0);
        if (vis) L = L + contrib;
      }
      if (rec) rec[2 * (b - 1) + 1] = nrec;
    }
    float pdf;
    if (!pt::continue_path(v, pix, smp, frame, b, k0, k1, beta, d, pdf)) break;
    o = v.on;
    prev_pdf = pdf;
  }
  return L;
}

__global__ void __launch_bounds__(128)
render_kernel(et_scene_dev S, const et_camera* __restrict__ cams, int W, int H, int y0, int y1,
              int spp, int max_depth, uint32_t first_frame, uint32_t k0, uint32_t k1, float* rgb,
              float* logl, int log_mode, float log_param, int32_t* records) {
  const int tiles_x = (W + 15) / 16;
  const int tile = blockIdx.x;
  const int x = (tile % tiles_x) * 16 + (threadIdx.x & 15);
  const int yb = (tile / tiles_x) * 8 + (threadIdx.x >> 4);   // row within the band
  const int y = y0 + yb;
  const int f = blockIdx.y;
  if (x >= W || y >= y1) return;
  const pt::Cam cam = pt::load_cam(cams[f]);
  f3 acc = mk(0.0f, 0.0f, 0.0f);
  const int64_t pix = ((int64_t)f * (y1 - y0) + yb) * W + x;
  for (int s = 0; s < spp; ++s) {
    int32_t* rec = nullptr;
    if (records) {
      rec = records + (pix * spp + s) * max_depth * 2;
      for (int i = 0; i < 2 * max_depth; ++i) rec[i] = (i & 1) ? -1 : -2;
    }
    acc = acc + trace_sample(S, cam, W, H, x, y, (uint32_t)s, first_frame + (uint32_t)f, max_depth,
                             k0, k1, rec);
  }
  const f3 m = acc * (1.0f / (float)spp);
  if (rgb) { rgb[3 * pix] = m.x; rgb[3 * pix + 1] = m.y; rgb[3 * pix + 2] = m.z; }
  if (logl) logl[pix] = pt::log_luminance(m, log_mode, log_param);
}

}  // namespace

int et_render_megakernel(et_scene* s, int n_frames, int first_frame, int W, int H, int y0, int y1,
                         int spp, int max_depth, uint64_t seed, float* rgb, float* logl, int log_mode,
                         float log_param, int32_t* records, cudaStream_t stream) {
  const int tiles = ((W + 15) / 16) * ((y1 - y0 + 7) / 8);
  dim3 grid(tiles, n_frames);
  render_kernel<<<grid, 128, 0, stream>>>(s->dev, s->d_cams, W, H, y0, y1, spp, max_depth,
                                          (uint32_t)first_frame, (uint32_t)seed,
                                          (uint32_t)(seed >> 32), rgb, logl, log_mode, log_param,
                                          records);
  ET_CHECK_LAUNCH();
  return ET_OK;
}

extern "C" int et_render_frames(const et_scene* scene, const et_camera* cams, int32_t n_frames,
                                int32_t first_frame, int32_t W, int32_t H, int32_t spp,
                                int32_t max_depth, uint64_t seed, float* rgb, float* logl,
                                int32_t log_mode, float log_param, int32_t* records, void* stream_) {
  return et_render_rows(scene, cams, n_frames, first_frame, W, H, 0, H, spp, max_depth, seed, rgb,
                        logl, log_mode, log_param, records, stream_);
}

extern "C" int et_render_rows(const et_scene* scene, const et_camera* cams, int32_t n_frames,
                              int32_t first_frame, int32_t W, int32_t H, int32_t y0, int32_t y1,
                              int32_t spp, int32_t max_depth, uint64_t seed, float* rgb, float* logl,
                              int32_t log_mode, float log_param, int32_t* records, void* stream_) {
  if (!scene || (!cams && n_frames > 0) || n_frames < 0 || n_frames > 65535) return ET_ERR_ARG;
  if (W < 1 || H < 1 || W > 65535 || H > 65535 || spp < 1 || spp > 4096 || max_depth < 1 ||
      max_depth > 16 || first_frame < 0)
    return ET_ERR_ARG;
  if (y0 < 0 || y1 > H || y0 >= y1) return ET_ERR_ARG;
  if (!rgb && !logl) return ET_ERR_ARG;
  if (log_mode != ET_LOG_EPS && log_mode != ET_LOG_PAPER) return ET_ERR_ARG;
  if (logl && !(log_param > 0.0f)) return ET_ERR_ARG;
  if (n_frames == 0) return ET_OK;
  cudaStream_t stream = (cudaStream_t)stream_;
  et_scene* s = const_cast<et_scene*>(scene);
  if (n_frames > s->cam_cap) {
    ET_CHECK_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->d_cams);
    s->d_cams = nullptr;
    s->cam_cap = 0;
    ET_CHECK_CUDA(cudaMalloc((void**)&s->d_cams, sizeof(et_camera) * (size_t)n_frames));
    s->cam_cap = n_frames;
  }
  ET_CHECK_CUDA(cudaMemcpyAsync(s->d_cams, cams, sizeof(et_camera) * (size_t)n_frames,
                                cudaMemcpyHostToDevice, stream));
  if (s->render_mode == ET_RENDER_MEGAKERNEL)
    return et_render_megakernel(s, n_frames, first_frame, W, H, y0, y1, spp, max_depth, seed, rgb,
                                logl, log_mode, log_param, records, stream);
  return et_render_wavefront(s, n_frames, first_frame, W, H, y0, y1, spp, max_depth, seed, rgb, logl,
                             log_mode, log_param, records, stream);
}

// ------------------------------------------------------------ profiling
namespace {
int prof_event(RenderProf& P, size_t* idx) {
  if (P.used == P.pool.size()) {
    cudaEvent_t e;
    ET_CHECK_CUDA(cudaEventCreate(&e));
    P.pool.push_back(e);
  }
  *idx = P.used++;
  return ET_OK;
}
}  // namespace

int prof_begin(et_scene* s, int kind, cudaStream_t st, size_t* e0) {
  (void)kind;
  if (!s->prof.on) return ET_OK;
  int rc = prof_event(s->prof, e0);
  if (rc != ET_OK) return rc;
  ET_CHECK_CUDA(cudaEventRecord(s->prof.pool[*e0], st));
  return ET_OK;
}

int prof_end(et_scene* s, int kind, size_t e0, int64_t items, const uint32_t* dev_len, cudaStream_t st) {
  RenderProf& P = s->prof;
  if (!P.on) return ET_OK;
  size_t e1 = 0;
  int rc = prof_event(P, &e1);
  if (rc != ET_OK) return rc;
  ET_CHECK_CUDA(cudaEventRecord(P.pool[e1], st));
  int slot = -1;
  if (dev_len) {
    if (P.n_len < RenderProf::kSlots) {
      slot = P.n_len++;
      ET_CHECK_CUDA(cudaMemcpyAsync(P.h_len + slot, dev_len, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    } else {
      P.overflow = true;
    }
  }
  P.marks.push_back({kind, e0, e1, slot, items});
  return ET_OK;
}

extern "C" int et_render_profile(et_scene* scene, int32_t enable) {
  if (!scene) return ET_ERR_ARG;
  RenderProf& P = scene->prof;
  if (enable && !P.h_len) ET_CHECK_CUDA(cudaMallocHost((void**)&P.h_len, sizeof(uint32_t) * RenderProf::kSlots));
  P.on = enable != 0;
  return ET_OK;
}

extern "C" int et_render_profile_read(et_scene* scene, double* ms, int64_t* launches, int64_t* items) {
  if (!scene || !ms || !launches || !items) return ET_ERR_ARG;
  RenderProf& P = scene->prof;
  for (int k = 0; k < RenderProf::kKinds; ++k) { ms[k] = 0.0; launches[k] = 0; items[k] = 0; }
  if (!P.marks.empty()) ET_CHECK_CUDA(cudaEventSynchronize(P.pool[P.marks.back().e1]));
  for (const auto& m : P.marks) {
    float t = 0.0f;
    ET_CHECK_CUDA(cudaEventElapsedTime(&t, P.pool[m.e0], P.pool[m.e1]));
    ms[m.kind] += t;
    launches[m.kind] += 1;
    items[m.kind] += m.slot >= 0 ? (int64_t)P.h_len[m.slot] : m.items;
  }
  const bool over = P.overflow;
  P.marks.clear();
  P.used = 0;
  P.n_len = 0;
  P.overflow = false;
  return over ? ET_ERR_CAPACITY : ET_OK;
}

extern "C" int et_render_set_mode(et_scene* scene, int32_t mode) {
  if (!scene || (mode != ET_RENDER_WAVEFRONT && mode != ET_RENDER_MEGAKERNEL &&
                 mode != ET_RENDER_WAVEFRONT_TILES && mode != ET_RENDER_WAVEFRONT_SORTED))
    return ET_ERR_ARG;
  scene->render_mode = mode;
  return ET_OK;
}

// ------------------------------------------------------------------ Philox
namespace {

__global__ void philox_kernel(const uint4* ctr, const uint2* key, int64_t n, uint4* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = ctr[i];
  const uint2 k = key[i];
  const u4 r = philox10(c.x, c.y, c.z, c.w, k.x, k.y);
  out[i] = make_uint4(r.x, r.y, r.z, r.w);
}

}  // namespace

// The renderer's and the sensor model's counter-based generator, evaluated on
// caller counters (the bitwise pin of the device Philox4x32-10).
extern "C" int et_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                                void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return ET_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(ctr) & 15) || (reinterpret_cast<uintptr_t>(out) & 15) ||
      (reinterpret_cast<uintptr_t>(key) & 7))
    return ET_ERR_ARG;
  if (n == 0) return ET_OK;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const uint4*>(ctr), reinterpret_cast<const uint2*>(key), n, reinterpret_cast<uint4*>(out));
  ET_CHECK_LAUNCH();
  return ET_OK;
}
