// Declarations shared by the EvSNet translation units.
#pragma once
#include <cuda_runtime.h>
#include "../../include/eventtracer.h"

constexpr int kMaxLayers = 8;

int et_evsnet_forward_f32(const float* logl, int32_t F, const et_evsnet_weights* net,
                          et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                          int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream);
int et_evsnet_forward_tc(const float* logl, int32_t F, const et_evsnet_weights* net,
                         et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                         int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream);
int et_evsnet_forward_pix(const float* logl, int32_t F, const et_evsnet_weights* net,
                          et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                          int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream);
int et_evsnet_forward_f32s(const float* logl, int32_t F, const et_evsnet_weights* net,
                           et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                           int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream);
int et_evsnet_forward_tct(const float* logl, int32_t F, const et_evsnet_weights* net,
                          et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                          int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream);
// bound of the tensor-core kernels' MMA waits (et_set_wait_budget, else the default)
uint32_t et_tc_wait_iters();
