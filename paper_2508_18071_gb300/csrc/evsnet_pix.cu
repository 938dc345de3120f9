// EvSNet forward in FP32 for the pixel-wise form (1x1 spatial extent: the
// paper's temporal network, Eq. 5 with kernel kt along time, plain stack or
// residual blocks; Eq. 6 projection; BiLIF of Eq. 2-3).
//
// With no spatial coupling every pixel is an independent 1-D network over
// time, so one thread owns one pixel for the whole call: the current step's
// activations stay in registers (16 or 32 channels), the weights sit in shared
// memory laid out [layer][tap][input channel][output channel] so that the
// whole warp reads the same four weights per 16-byte load, and the causal
// history of each layer's input (the caller's state, [layer][kt-1][C][H][W])
// is read and written in place, coalesced across the warp's pixels.  Within a
// call the history is a ring (the slot of the oldest input takes the newest);
// at the end each thread rotates its pixel's slots back to oldest-first order,
// the layout the state promises between calls.
//
// With a spatial stem (ks0 > 0) layer 0 is a one-step ks0 x ks0 convolution of
// X: each thread reads its neighbours' X for the current step from the log
// frames (and the state's previous frame, which this kernel only reads) and
// layer 0 keeps no history; the temporal layers after it are per pixel.
#include "et_internal.cuh"
#include "event_emit.cuh"
#include "evsnet_common.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxKt = 9;

struct PixParams {
  int kind, L, C, kt, ks0;
  float beta, vth, reset;
  int H, W, F, f0, t0;
  int woff[kMaxLayers + 1], boff[kMaxLayers + 1];
};

template <int CP>
__global__ void __launch_bounds__(kThreads)
evsnet_pix_kernel(PixParams P, const float* __restrict__ logl, const float* __restrict__ wg,
                  const float* __restrict__ bg, float* __restrict__ Vg, float* __restrict__ hist,
                  const float* __restrict__ last_l, et_event* events, int64_t cap,
                  unsigned long long* n_events, float* __restrict__ I_out,
                  int8_t* __restrict__ spikes) {
  // [L][kt][CP (ci)][CP (co)], then biases [L+1][CP], proj [CP], stem taps [ks0 ks0][CP (co)]
  extern __shared__ __align__(16) float sw[];
  const int L = P.L, C = P.C, kt = P.kt, hk = kt - 1, ks0 = P.ks0;
  const int tid = threadIdx.x;
  const int nw = L * kt * CP * CP;
  float* sb = sw + nw;
  float* swp = sb + (L + 1) * CP;
  float* sstem = swp + CP;
  for (int i = tid; i < nw; i += kThreads) {
    const int co = i % CP, ci = (i / CP) % CP, tau = (i / (CP * CP)) % kt, l = i / (CP * CP * kt);
    const int cin = l == 0 ? 1 : C;
    float v = 0.0f;
    if (co < C && ci < cin && !(l == 0 && ks0 > 0)) v = wg[P.woff[l] + (co * cin + ci) * kt + tau];
    sw[i] = v;
  }
  for (int i = tid; i < (L + 1) * CP; i += kThreads) {
    const int l = i / CP, c = i % CP;
    sb[i] = (l < L && c < C) ? bg[P.boff[l] + c] : ((l == L && c == 0) ? bg[P.boff[L]] : 0.0f);
  }
  for (int i = tid; i < CP; i += kThreads) swp[i] = i < C ? wg[P.woff[L] + i] : 0.0f;
  for (int i = tid; i < ks0 * ks0 * CP; i += kThreads) {
    const int co = i % CP, tap = i / CP;
    sstem[i] = co < C ? wg[P.woff[0] + co * ks0 * ks0 + tap] : 0.0f;
  }
  __syncthreads();

  const int64_t npix = (int64_t)P.H * P.W;
  const int64_t q = (int64_t)blockIdx.x * kThreads + tid;
  const bool live = q < npix;
  const uint32_t px = live ? (uint32_t)(q % P.W) : 0u, py = live ? (uint32_t)(q / P.W) : 0u;
  // history element (layer l, physical slot s, channel c) of this pixel
  auto hidx = [&](int l, int s, int c) -> int64_t { return (((int64_t)l * hk + s) * C + c) * npix + q; };
  float V = live ? Vg[q] : 0.0f;
  int head = 0;   // physical slot of the oldest input
  for (int f = P.f0; f < P.F; ++f) {
    uint32_t nev = 0;
    int S = 0;
    if (live) {
      const float cur = __ldg(logl + (int64_t)f * npix + q);
      const float prev = f == 0 ? last_l[q] : __ldg(logl + (int64_t)(f - 1) * npix + q);
      float x[CP], h[CP], acc[CP];
      x[0] = cur - prev;                          // Eq. 1
#pragma unroll
      for (int c = 1; c < CP; ++c) x[c] = 0.0f;
      for (int l = 0; l < L; ++l) {
        const int cin = l == 0 ? 1 : C;
        const float* wl = sw + l * kt * CP * CP;
#pragma unroll
        for (int co = 0; co < CP; ++co) acc[co] = sb[l * CP + co];
        if (l == 0 && ks0 > 0) {
          // spatial stem: the ks0 x ks0 neighbourhood of this step's X (zero
          // outside the image), taps in row-major order
          const int r0 = ks0 >> 1;
          for (int dy = 0; dy < ks0; ++dy) {
            const int yy = (int)py + dy - r0;
            if (yy < 0 || yy >= P.H) continue;
            for (int dx = 0; dx < ks0; ++dx) {
              const int xx = (int)px + dx - r0;
              if (xx < 0 || xx >= P.W) continue;
              const int64_t qq = (int64_t)yy * P.W + xx;
              const float xc = __ldg(logl + (int64_t)f * npix + qq);
              const float xp = f == 0 ? last_l[qq] : __ldg(logl + (int64_t)(f - 1) * npix + qq);
              const float v = xc - xp;
              const float4* w4 = reinterpret_cast<const float4*>(sstem + (dy * ks0 + dx) * CP);
#pragma unroll
              for (int j = 0; j < CP / 4; ++j) {
                const float4 w = w4[j];
                acc[4 * j] = fmaf(w.x, v, acc[4 * j]);
                acc[4 * j + 1] = fmaf(w.y, v, acc[4 * j + 1]);
                acc[4 * j + 2] = fmaf(w.z, v, acc[4 * j + 2]);
                acc[4 * j + 3] = fmaf(w.w, v, acc[4 * j + 3]);
              }
            }
          }
        } else {
        // software pipeline: the next tap's inputs are loaded while this
        // tap's products accumulate
        float nxt[CP];
        {
          const int slot0 = head < hk ? head : head - hk;
#pragma unroll
          for (int ci = 0; ci < CP; ++ci)
            nxt[ci] = ci >= cin ? 0.0f : (0 == hk ? x[ci] : hist[hidx(l, slot0, ci)]);
        }
        for (int tau = 0; tau < kt; ++tau) {
          const float* wt = wl + tau * CP * CP;
          float in[CP];
#pragma unroll
          for (int ci = 0; ci < CP; ++ci) in[ci] = nxt[ci];
          if (tau + 1 < kt) {
            const int t1 = tau + 1;
            const int slot1 = head + t1 < hk ? head + t1 : head + t1 - hk;
#pragma unroll
            for (int ci = 0; ci < CP; ++ci)
              nxt[ci] = ci >= cin ? 0.0f : (t1 == hk ? x[ci] : hist[hidx(l, slot1, ci)]);
          }
#pragma unroll
          for (int ci = 0; ci < CP; ++ci) {
            if (ci >= cin) break;
            const float v = in[ci];
            const float4* w4 = reinterpret_cast<const float4*>(wt + ci * CP);
#pragma unroll
            for (int j = 0; j < CP / 4; ++j) {
              const float4 w = w4[j];
              acc[4 * j] = fmaf(w.x, v, acc[4 * j]);
              acc[4 * j + 1] = fmaf(w.y, v, acc[4 * j + 1]);
              acc[4 * j + 2] = fmaf(w.z, v, acc[4 * j + 2]);
              acc[4 * j + 3] = fmaf(w.w, v, acc[4 * j + 3]);
            }
          }
        }
        // this step's input becomes the newest history entry (the oldest slot,
        // already read above)
        if (hk > 0) {
#pragma unroll
          for (int ci = 0; ci < CP; ++ci)
            if (ci < cin) hist[hidx(l, head, ci)] = x[ci];
        }
        }   // temporal layer
        if (P.kind == ET_NET_RESIDUAL && l >= 2 && (l % 2) == 0) {
          // closing layer of a block: h_i = ReLU(h_{i-1} + conv(a_i))
#pragma unroll
          for (int c = 0; c < CP; ++c) { h[c] = fmaxf(h[c] + acc[c], 0.0f); x[c] = h[c]; }
        } else {
#pragma unroll
          for (int c = 0; c < CP; ++c) x[c] = fmaxf(acc[c], 0.0f);
          if (l == 0 || P.kind != ET_NET_RESIDUAL) {
#pragma unroll
            for (int c = 0; c < CP; ++c) h[c] = x[c];
          }
        }
      }
      // Eq. 6 projection and BiLIF
      float I = sb[L * CP];
#pragma unroll
      for (int c = 0; c < CP; ++c) I = fmaf(swp[c], x[c], I);
      const float vp = P.beta * V + I;
      S = vp >= P.vth ? 1 : (vp <= -P.vth ? -1 : 0);
      V = vp - P.reset * (float)S;
      nev = (S != 0 && P.t0 + f >= 0) ? 1u : 0u;   // delayed labels below 0: none
      const int step = f - P.f0;
      if (I_out) I_out[(int64_t)step * npix + q] = I;
      if (spikes) spikes[(int64_t)step * npix + q] = (int8_t)S;
    }
    emit_events_warp(events, cap, n_events, nev, px, py, (uint32_t)(P.t0 + f), S);
    if (hk > 0) head = head + 1 < hk ? head + 1 : 0;
  }
  if (!live) return;
  Vg[q] = V;
  // back to oldest-first slots
  if (hk > 1 && head != 0) {
    for (int l = ks0 > 0 ? 1 : 0; l < L; ++l) {
      const int cin = l == 0 ? 1 : C;
      for (int ci = 0; ci < cin; ++ci) {
        float tmp[kMaxKt];
        for (int s = 0; s < hk; ++s) tmp[s] = hist[hidx(l, s, ci)];
        for (int tau = 0; tau < hk; ++tau) {
          const int s = head + tau < hk ? head + tau : head + tau - hk;
          hist[hidx(l, tau, ci)] = tmp[s];
        }
      }
    }
  }
}

template <int CP>
int launch(const float* logl, int32_t F, const et_evsnet_weights* net, et_evsnet_state* st,
           int32_t t0, et_event* events, int64_t cap, int64_t* n_events, float* I_out,
           int8_t* spikes, cudaStream_t stream) {
  PixParams P{};
  P.kind = net->kind; P.L = net->n_layers; P.C = net->C; P.kt = net->kt; P.ks0 = net->ks0;
  P.beta = net->beta; P.vth = net->vth; P.reset = net->reset;
  P.H = st->H; P.W = st->W; P.F = F; P.f0 = st->initialized ? 0 : 1; P.t0 = t0;
  int wo = 0, bo = 0;
  for (int l = 0; l < P.L; ++l) {
    P.woff[l] = wo; P.boff[l] = bo;
    wo += l == 0 ? P.C * (P.ks0 > 0 ? P.ks0 * P.ks0 : P.kt) : P.C * P.C * P.kt;
    bo += P.C;
  }
  P.woff[P.L] = wo; P.boff[P.L] = bo;
  const size_t smem = sizeof(float) * ((size_t)P.L * P.kt * CP * CP + (P.L + 1) * CP + CP +
                                       (size_t)P.ks0 * P.ks0 * CP);
  int dev = 0, max_smem = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if ((int)smem > max_smem) return ET_ERR_UNIMPLEMENTED;
  ET_CHECK_CUDA(cudaFuncSetAttribute(evsnet_pix_kernel<CP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  const int64_t npix = (int64_t)P.H * P.W;
  evsnet_pix_kernel<CP><<<(unsigned)((npix + kThreads - 1) / kThreads), kThreads, smem, stream>>>(
      P, logl, net->w, net->b, st->V, st->hist, st->last_l, events, cap,
      reinterpret_cast<unsigned long long*>(n_events), I_out, spikes);
  ET_CHECK_LAUNCH();
  return ET_OK;
}

}  // namespace

int et_evsnet_forward_pix(const float* logl, int32_t F, const et_evsnet_weights* net,
                          et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                          int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream) {
  if (net->ks != 1 || net->kt > kMaxKt || net->C > 32) return ET_ERR_UNIMPLEMENTED;
  if (net->C <= 16)
    return launch<16>(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
  return launch<32>(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
}
