// Host-side definition of the opaque et_scene handle.
#pragma once
#include <vector>
#include "et_internal.cuh"

// Per-kernel timing of the wavefront schedule (et_render_profile): events
// around each launch and the queue lengths each launch processed, copied to
// pinned host memory; summed by et_render_profile_read.
struct RenderProf {
  static constexpr int kKinds = 5;        // raygen, trace, shade, shadow, accumulate
  static constexpr int kSlots = 1 << 15;  // queue-length copies held between reads
  bool on = false;
  std::vector<cudaEvent_t> pool;          // events, reused across reads
  size_t used = 0;
  struct Mark { int kind; size_t e0, e1; int slot; int64_t items; };
  std::vector<Mark> marks;
  uint32_t* h_len = nullptr;              // pinned: queue lengths read by the device
  int n_len = 0;
  bool overflow = false;
};

struct et_scene {
  float4* d_tris = nullptr;
  BvhNode* d_nodes = nullptr;
  DevMaterial* d_mats = nullptr;
  DevLight* d_lights = nullptr;
  et_camera* d_cams = nullptr;   // camera staging for et_render_frames
  int64_t cam_cap = 0;
  int64_t n_tris = 0, n_nodes = 0;
  double sah = 0.0;
  et_scene_dev dev{};
  int render_mode = ET_RENDER_WAVEFRONT_TILES;
  int builder = ET_BVH_GPU;
  void* wf_mem = nullptr;        // wavefront queues and path state, grown on demand
  int64_t wf_cap = 0, wf_acc_cap = 0;
  void* wf_sort_mem = nullptr;   // sorted mode: keys, indices and radix-sort scratch
  int64_t wf_sort_cap = 0;
  size_t wf_sort_tmp = 0;
  float box_lo[3] = {0, 0, 0}, box_hi[3] = {0, 0, 0};   // the hierarchy's root box
  // moving geometry (et_scene_update): leaf slot -> input triangle, inner nodes
  // deepest level first with the level boundaries, upload staging
  int64_t n_user = 0;
  int32_t* d_perm = nullptr;
  int32_t* d_refit = nullptr;
  std::vector<int> refit_levels;
  float* d_upd = nullptr;
  RenderProf prof;
};
