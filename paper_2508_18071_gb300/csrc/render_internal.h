// The two schedules behind et_render_frames (cameras already staged on the device).
#pragma once
#include "scene_internal.h"

// Rows [y0, y1) of W x H frames: outputs are band-relative ([F][y1 - y0][W]),
// rays and random numbers those of the full image's rows.
int et_render_megakernel(et_scene* s, int n_frames, int first_frame, int W, int H, int y0, int y1,
                         int spp, int max_depth, uint64_t seed, float* rgb, float* logl, int log_mode,
                         float log_param, int32_t* records, cudaStream_t stream);
int et_render_wavefront(et_scene* s, int n_frames, int first_frame, int W, int H, int y0, int y1,
                        int spp, int max_depth, uint64_t seed, float* rgb, float* logl, int log_mode,
                        float log_param, int32_t* records, cudaStream_t stream);

// et_render_profile hooks used by the schedules (no-ops unless profiling is on):
// prof_begin records the start event of a launch of `kind`; prof_end records
// its end, with `items` processed, or with the length the device holds at
// `dev_len` (copied asynchronously) when dev_len is not null.
int prof_begin(et_scene* s, int kind, cudaStream_t st, size_t* e0);
int prof_end(et_scene* s, int kind, size_t e0, int64_t items, const uint32_t* dev_len, cudaStream_t st);
