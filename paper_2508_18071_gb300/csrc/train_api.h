// Limits shared by the training translation unit and its callers.
#pragma once
#include "../../include/eventtracer.h"

constexpr int kMaxSeg = 32;   // longest BPTT segment (membrane checkpoint interval)

#include <cuda_runtime.h>

// The paper's pixel-wise temporal form (1x1 spatial extent, causal kernel kt,
// plain stack or residual blocks), trained with whole-clip activations
// (train_temporal.cu).
bool et_train_is_temporal(const et_evsnet_weights* net);
size_t et_train_temporal_bytes(const et_evsnet_weights* net, const et_train_shape* sh);
int et_train_temporal_forward(const float* logl, const et_train_shape* sh,
                              const et_evsnet_weights* net, int8_t* spikes, float* S_on,
                              float* S_off, float* V_ckpt, float* I_out, void* workspace,
                              cudaStream_t st);
int et_train_temporal_backward(const float* logl, const et_train_shape* sh,
                               const et_evsnet_weights* net, const float* V_ckpt,
                               const float* dS_on, const float* dS_off, float alpha,
                               float* grad_w, float* grad_b, void* workspace, cudaStream_t st);

// The spatial form's C -> C 3x3 layers on the tensor cores (BF16 operands, FP32
// accumulation; train_tc.cu), N images of C <= 16 plane-major channels:
// forward out = ReLU(conv(in) + b), with I = bp + wp . out when I is not NULL;
// or, with data_grad, out = conv^T(in) * 1(a_prev > 0).
int et_train_tc_conv(const float* in, int N, int C, int H, int W, const float* w, const float* b,
                     float* out, const float* wp, const float* bp, float* I, const float* a_prev,
                     bool data_grad, cudaStream_t stream);
// The weight and bias gradients of such a layer with BF16 operands on the
// tensor cores: grad w[co][ci][t] += sum dz[co][p] act[ci][p + off(t)],
// grad b[co] += sum dz[co][p] (FP32 accumulation; added to gw / gb).
int et_train_tc_wgrad(const float* dz, const float* act, int N, int C, int H, int W, float* gw,
                      float* gb, cudaStream_t stream);

// The temporal form's C -> C layers on the tensor cores (BF16 operands, FP32
// accumulation; train_tct.cu), activations [B][K][hw][C] with C <= 16 and
// kt <= 7: forward out = ReLU(conv(in) + b (+ extra)), with I = bp + wp . out
// when I is not NULL; or, with data_grad, out = (extra + conv^T(in)) *
// 1(mask > 0), in being dL/dz of the layer's output.
bool et_train_tct_supported(const et_evsnet_weights* net);
int et_train_tct_conv(const float* in, int B, int K, int64_t hw, int C, int kt, const float* w, const float* b,
                      const float* extra, const float* mask, float* out, const float* wp, const float* bp,
                      float* I, bool data_grad, cudaStream_t st);
// Its weight and bias gradients: grad w[co][ci][tau] += sum dz[k][co]
// in[k - (kt-1) + tau][ci], grad b[co] += sum dz[k][co] (added to gw / gb).
int et_train_tct_wgrad(const float* dz, const float* in, int B, int K, int64_t hw, int C, int kt, float* gw,
                       float* gb, cudaStream_t st);
