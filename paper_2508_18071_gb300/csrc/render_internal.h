// The two schedules behind et_render_frames (cameras already staged on the device).
#pragma once
#include "scene_internal.h"

int et_render_megakernel(et_scene* s, int n_frames, int first_frame, int W, int H, int spp,
                         int max_depth, uint64_t seed, float* rgb, float* logl, int log_mode,
                         float log_param, int32_t* records, cudaStream_t stream);
int et_render_wavefront(et_scene* s, int n_frames, int first_frame, int W, int H, int spp,
                        int max_depth, uint64_t seed, float* rgb, float* logl, int log_mode,
                        float log_param, int32_t* records, cudaStream_t stream);
