// et_evsnet_forward: argument checks and dispatch between the FP32 (CUDA core:
// pixel-wise form in evsnet_pix.cu, 3x3 stacks of up to 16 channels in
// evsnet_f32s.cu, other spatial forms in evsnet.cu) and BF16 / FP8 (tensor
// core: 3x3 stacks in evsnet_tc.cu, the pixel-wise temporal form with or
// without a spatial stem in evsnet_tct.cu) EvSNet kernels.
#include "et_internal.cuh"
#include "evsnet_common.h"

extern "C" int et_evsnet_forward(const float* logl, int32_t F, const et_evsnet_weights* net,
                                 et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                                 int64_t* n_events, float* I_out, int8_t* spikes, void* stream_) {
  if (!net || !st || !n_events || F < 0 || cap < 0 || (cap > 0 && !events)) return ET_ERR_ARG;
  if (F > 0 && !logl) return ET_ERR_ARG;
  if (!net->w || !net->b || !st->V || !st->last_l) return ET_ERR_ARG;
  if (st->H < 1 || st->W < 1 || st->H > 65535 || st->W > 65535) return ET_ERR_ARG;
  if (net->n_layers < 1 || net->n_layers > kMaxLayers || net->C < 1 || net->kt < 1 || net->ks < 1 ||
      (net->ks % 2) == 0)
    return ET_ERR_ARG;
  if (net->kind != ET_NET_STACK && net->kind != ET_NET_RESIDUAL) return ET_ERR_ARG;
  if (net->kind == ET_NET_RESIDUAL && (net->n_layers % 2) == 0) return ET_ERR_ARG;
  if (net->kt > 1 && !st->hist) return ET_ERR_ARG;
  if (net->ks0 < 0 || net->ks0 > 7 || (net->ks0 > 0 && net->ks0 % 2 == 0)) return ET_ERR_ARG;
  if (net->delay < 0 || net->delay > (1 << 24)) return ET_ERR_ARG;
  // a spatial stem is taken by the pixel-wise kernels (temporal layers after it)
  if (net->ks0 > 0 && net->ks != 1) return ET_ERR_UNIMPLEMENTED;
  if (net->C > 32 || net->ks > 7 || net->kt > 9) return ET_ERR_UNIMPLEMENTED;
  // a temporal history with a spatial halo would be read by neighbouring tiles
  // while it is rewritten: not supported by these kernels
  if (net->kt > 1 && net->ks > 1) return ET_ERR_UNIMPLEMENTED;
  cudaStream_t stream = (cudaStream_t)stream_;
  ET_CHECK_CUDA(cudaMemsetAsync(n_events, 0, sizeof(int64_t), stream));
  if (F == 0) return ET_OK;
  int rc;
  // the kernels label step f of the call t0 + f and emit nothing below 0: the
  // delay shifts every label by -delay
  t0 -= net->delay;
  if (net->dtype == ET_F32 && net->ks == 1)
    rc = et_evsnet_forward_pix(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
  else if (net->dtype == ET_F32) {
    // the 3x3 kernel declines (before launching anything) what it does not cover
    rc = et_evsnet_forward_f32s(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
    if (rc == ET_ERR_UNIMPLEMENTED)
      rc = et_evsnet_forward_f32(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
  }
  else if ((net->dtype == ET_BF16 || net->dtype == ET_FP8) && net->ks == 1)
    rc = et_evsnet_forward_tct(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
  else if ((net->dtype == ET_BF16 || net->dtype == ET_FP8) && net->ks0 == 0)
    rc = et_evsnet_forward_tc(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
  else
    rc = ET_ERR_UNIMPLEMENTED;
  if (rc != ET_OK) return rc;
  const int64_t npix = (int64_t)st->H * st->W;
  ET_CHECK_CUDA(cudaMemcpyAsync(st->last_l, logl + (int64_t)(F - 1) * npix, sizeof(float) * npix,
                                cudaMemcpyDeviceToDevice, stream));
  st->initialized = 1;
  return ET_OK;
}
