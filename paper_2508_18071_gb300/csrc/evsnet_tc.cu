// EvSNet forward on the tcgen05 tensor cores (BF16 operands, FP32 accumulation
// in TMEM) for the spatial form: a stack of 3x3 convolutions with ReLU (Eq. 5
// with kernel extent in space), the point-wise projection (Eq. 6) and BiLIF
// (Eq. 2-3), for up to 32 channels.
//
// Each CTA owns a 32 x 16 pixel tile for the whole call and walks the frames
// in order; the membrane potentials of its pixels stay in shared memory.  For
// one step:
//   * the frame tile plus an L-pixel halo is loaded (X_k = l_k - l_{k-1}, Eq. 1);
//   * layer 0 (one input channel, 9 MACs per output) runs on CUDA cores and
//     writes BF16 activations;
//   * every further layer is an implicit GEMM on the tensor core.  Activations
//     live on a padded grid of width Wp = 32 + 2L in the K-major, no-swizzle
//     operand layout (8 channels x 16 B per row, one plane per 8 channels), so
//     the A operand of tap (dy, dx) is the same buffer with its start address
//     moved by (dy Wp + dx) rows: 9 taps = 9 descriptors, no im2col.  M = 128
//     padded positions per MMA, N = channels, K = 16 channels per instruction;
//     the accumulators of all M blocks of a layer sit side by side in TMEM;
//   * four warps read the accumulators back (tcgen05.ld, 32 lanes each), add
//     the bias, apply ReLU and the image-border zero padding, and write the
//     next layer's BF16 operand -- or, for the last layer, project to one
//     current per pixel in FP32 and run BiLIF and the event append.
// Positions in the halo that a layer does not need are computed and ignored
// (the "garbage columns" of the padded grid); they never feed a needed output.
#include "et_internal.cuh"
#include "event_emit.cuh"
#include "evsnet_common.h"
#include "tc_ptx.cuh"
#include <cuda_bf16.h>

namespace {

constexpr int TW = 32, TH = 16;
constexpr int kThreads = 128;
constexpr uint32_t kWaitIters = 1u << 22;
constexpr unsigned long long kTimeoutBit = 1ull << 62;

struct TcParams {
  int H, W, F, f0, t0, L, C;
  float beta, vth, reset;
  int Wp, Hp, rows;                     // padded grid
  int plane;                            // bytes per 8-channel plane of one activation buffer
  int act_bytes, wB_bytes;              // per activation buffer; all tensor-core weights
  int off_act1, off_wB, off_f32, off_cur, off_prev, off_V;  // smem byte offsets
  int nb1;                              // M blocks of layer 1 (the widest)
  uint32_t tmem_cols;
};

template <int CP>
__global__ void __launch_bounds__(kThreads)
evsnet_tc_kernel(TcParams P, const float* __restrict__ logl, const float* __restrict__ wg,
                 const float* __restrict__ bg, float* __restrict__ Vg,
                 const float* __restrict__ last_l, et_event* events, int64_t cap,
                 unsigned long long* n_events, float* __restrict__ I_out,
                 int8_t* __restrict__ spikes) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int bail;
  constexpr int NPL = CP / 8;           // 8-channel planes
  constexpr int KS = CP / 16;           // K steps of 16 channels
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = (P.W + TW - 1) / TW;
  const int ox = (blockIdx.x % tiles_x) * TW, oy = (blockIdx.x / tiles_x) * TH;
  const int L = P.L, Wp = P.Wp, Hp = P.Hp, C = P.C;
  const int64_t npix = (int64_t)P.H * P.W;
  unsigned char* act[2] = {sm, sm + P.off_act1};
  unsigned char* wB = sm + P.off_wB;
  float* f32 = reinterpret_cast<float*>(sm + P.off_f32);
  float* w0 = f32;                        // [CP][9]
  float* bs = w0 + CP * 9;                // [L][CP]
  float* wp = bs + L * CP;                // [CP] projection
  float* bp = wp + CP;                    // [1]
  float* cur = reinterpret_cast<float*>(sm + P.off_cur);
  float* prev = reinterpret_cast<float*>(sm + P.off_prev);
  float* Vs = reinterpret_cast<float*>(sm + P.off_V);

  // ---- one-time set-up: zero operands, stage weights, membrane potentials
  for (int i = tid; i < (2 * P.act_bytes) / 16; i += kThreads)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  {
    // packed FP32 weights: layer 0 [C][1][1][3][3], layers 1.. [C][C][1][3][3], projection [C]
    for (int i = tid; i < CP * 9; i += kThreads) {
      const int c = i / 9, t = i % 9;
      w0[i] = c < C ? wg[c * 9 + t] : 0.0f;
    }
    for (int i = tid; i < L * CP; i += kThreads) {
      const int l = i / CP, c = i % CP;
      bs[i] = c < C ? bg[l * C + c] : 0.0f;
    }
    const int wproj = 9 * C + (L - 1) * C * C * 9;
    for (int i = tid; i < CP; i += kThreads) wp[i] = i < C ? wg[wproj + i] : 0.0f;
    if (tid == 0) bp[0] = bg[L * C];
    // tensor-core weights: per layer l >= 1 and tap t, B[n = cout][k = cin] in the
    // K-major layout: (k / 8) planes of CP rows x 16 B, rows of 8 channels
    const int per_tap = CP * CP * 2;
    for (int i = tid; i < (L - 1) * 9 * CP * CP; i += kThreads) {
      const int k = i % CP, n = (i / CP) % CP, t = (i / (CP * CP)) % 9, l = 1 + i / (CP * CP * 9);
      float v = 0.0f;
      if (n < C && k < C) v = wg[9 * C + (l - 1) * C * C * 9 + (n * C + k) * 9 + t];
      unsigned char* dst = wB + ((l - 1) * 9 + t) * per_tap + (k / 8) * (CP * 16) + n * 16 + (k % 8) * 2;
      *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
    }
  }
  for (int i = tid; i < TW * TH; i += kThreads) {
    const int gx = ox + i % TW, gy = oy + i / TW;
    Vs[i] = (gx < P.W && gy < P.H) ? Vg[(int64_t)gy * P.W + gx] : 0.0f;
  }
  // previous frame's tile
  for (int i = tid; i < Hp * Wp; i += kThreads) {
    const int gx = ox - L + i % Wp, gy = oy - L + i / Wp;
    float v = 0.0f;
    if (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H)
      v = P.f0 == 0 ? last_l[(int64_t)gy * P.W + gx] : __ldg(logl + (int64_t)gy * P.W + gx);
    prev[i] = v;
  }
  if (warp == 0) tmem_alloc(&tmem_slot, P.tmem_cols);
  if (tid == 0) { mbar_init(&mma_bar, 1); bail = 0; }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0;
  const uint32_t idesc = umma_idesc_bf16(128, CP);

  for (int f = (P.f0 == 0 ? 0 : 1); f < P.F && !bail; ++f) {
    // ---- frame tile and layer 0 on CUDA cores
    for (int i = tid; i < Hp * Wp; i += kThreads) {
      const int gx = ox - L + i % Wp, gy = oy - L + i / Wp;
      cur[i] = (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H)
                   ? __ldg(logl + (int64_t)f * npix + (int64_t)gy * P.W + gx) : 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < (Hp - 2) * (Wp - 2); i += kThreads) {
      const int py = 1 + i / (Wp - 2), px = 1 + i % (Wp - 2);
      const int gx = ox - L + px, gy = oy - L + py;
      const int m = py * Wp + px;
      __align__(16) __nv_bfloat16 h[CP];
      if (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H) {
        float x[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int q = m + (t / 3 - 1) * Wp + (t % 3 - 1);
          x[t] = cur[q] - prev[q];
        }
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          float a = bs[c];
#pragma unroll
          for (int t = 0; t < 9; ++t) a = fmaf(w0[c * 9 + t], x[t], a);
          h[c] = __float2bfloat16_rn(fmaxf(a, 0.0f));
        }
      } else {
#pragma unroll
        for (int c = 0; c < CP; ++c) h[c] = __float2bfloat16_rn(0.0f);
      }
#pragma unroll
      for (int p = 0; p < NPL; ++p)
        *reinterpret_cast<uint4*>(act[0] + p * P.plane + m * 16) = reinterpret_cast<const uint4*>(h)[p];
    }
    // ---- tensor-core layers
    for (int l = 1; l < L; ++l) {
      const unsigned char* ain = act[(l - 1) & 1];
      unsigned char* aout = act[l & 1];
      const int m_start = (l + 1) * Wp;
      const int nb = ((Hp - 2 * l - 2) * Wp + 127) / 128;
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        const uint32_t abase = smem_u32(ain), bbase = smem_u32(wB + (l - 1) * 9 * CP * CP * 2);
        for (int b = 0; b < nb; ++b) {
          const int m0 = m_start + b * 128;
          for (int t = 0; t < 9; ++t) {
            const int o = (t / 3 - 1) * Wp + (t % 3 - 1);
            for (int s = 0; s < KS; ++s) {
              const uint64_t ad = umma_desc(abase + (2 * s) * P.plane + (m0 + o) * 16, P.plane, 128);
              const uint64_t bd = umma_desc(bbase + t * CP * CP * 2 + (2 * s) * (CP * 16), CP * 16, 128);
              umma_bf16(tmem + b * CP, ad, bd, idesc, (t | s) != 0);
            }
          }
        }
        umma_commit(&mma_bar);
      }
      const bool ok = mbar_wait(&mma_bar, phase, kWaitIters);
      phase ^= 1;
      if (!ok) {
        if (lane == 0) atomicOr(n_events, kTimeoutBit);
        bail = 1;
      }
      tc_fence_after();
      __syncthreads();
      if (bail) break;
      const bool last = l == L - 1;
      for (int b = 0; b < nb; ++b) {
        const int m = m_start + b * 128 + warp * 32 + lane;
        float acc[CP];
#pragma unroll
        for (int j = 0; j < CP / 16; ++j)
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + b * CP + j * 16, acc + j * 16);
        const int py = m / Wp, px = m % Wp;
        const bool need = m < Hp * Wp && py >= l + 1 && py < Hp - l - 1 && px >= l + 1 && px < Wp - l - 1;
        const int gx = ox - L + px, gy = oy - L + py;
        const bool inimg = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
        if (!last) {
          if (need) {
            __align__(16) __nv_bfloat16 h[CP];
#pragma unroll
            for (int c = 0; c < CP; ++c) h[c] = __float2bfloat16_rn(inimg ? fmaxf(acc[c] + bs[l * CP + c], 0.0f) : 0.0f);
#pragma unroll
            for (int p = 0; p < NPL; ++p)
              *reinterpret_cast<uint4*>(aout + p * P.plane + m * 16) = reinterpret_cast<const uint4*>(h)[p];
          }
        } else {
          uint32_t nev = 0;
          int S = 0;
          if (need && inimg) {
            float I = bp[0];
#pragma unroll
            for (int c = 0; c < CP; ++c) I = fmaf(wp[c], fmaxf(acc[c] + bs[l * CP + c], 0.0f), I);
            const int ti = (py - L) * TW + (px - L);
            const float vp = P.beta * Vs[ti] + I;
            S = vp >= P.vth ? 1 : (vp <= -P.vth ? -1 : 0);
            Vs[ti] = vp - P.reset * (float)S;
            nev = S != 0 ? 1u : 0u;
            const int64_t q = (int64_t)(f - (P.f0 == 0 ? 0 : 1)) * npix + (int64_t)gy * P.W + gx;
            if (I_out) I_out[q] = I;
            if (spikes) spikes[q] = (int8_t)S;
          }
          emit_events_warp(events, cap, n_events, nev, (uint32_t)gx, (uint32_t)gy, (uint32_t)(P.t0 + f), S);
        }
      }
      tc_fence_before();
    }
    __syncthreads();
    float* t = cur; cur = prev; prev = t;
  }
  __syncthreads();
  if (bail) {
    // a bounded wait gave up: the timeout bit is set in *n_events; give the MMAs
    // still in flight a second bounded wait before the TMEM is released
    mbar_wait(&mma_bar, phase ^ 1u, kWaitIters);
  } else {
    for (int i = tid; i < TW * TH; i += kThreads) {
      const int gx = ox + i % TW, gy = oy + i / TW;
      if (gx < P.W && gy < P.H) Vg[(int64_t)gy * P.W + gx] = Vs[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, P.tmem_cols);
}

template <int CP>
int launch(const float* logl, int32_t F, const et_evsnet_weights* net, et_evsnet_state* st,
           int32_t t0, et_event* events, int64_t cap, int64_t* n_events, float* I_out,
           int8_t* spikes, cudaStream_t stream) {
  TcParams P{};
  P.H = st->H; P.W = st->W; P.F = F; P.f0 = st->initialized ? 0 : 1; P.t0 = t0;
  P.L = net->n_layers; P.C = net->C;
  P.beta = net->beta; P.vth = net->vth; P.reset = net->reset;
  P.Wp = TW + 2 * P.L; P.Hp = TH + 2 * P.L;
  // rows read by the widest layer's last block stay below Hp Wp + 128
  P.rows = P.Hp * P.Wp + 128 + P.Wp;
  P.plane = P.rows * 16;
  P.act_bytes = (CP / 8) * P.plane;
  P.wB_bytes = (P.L - 1) * 9 * CP * CP * 2;
  auto al = [](int x) { return (x + 1023) & ~1023; };
  P.off_act1 = al(P.act_bytes);
  P.off_wB = P.off_act1 + al(P.act_bytes);
  P.off_f32 = P.off_wB + al(P.wB_bytes);
  const int f32_bytes = 4 * (CP * 9 + P.L * CP + CP + 4);
  P.off_cur = P.off_f32 + al(f32_bytes);
  P.off_prev = P.off_cur + al(4 * P.Hp * P.Wp);
  P.off_V = P.off_prev + al(4 * P.Hp * P.Wp);
  const int smem = P.off_V + al(4 * TW * TH);
  P.nb1 = ((P.Hp - 4) * P.Wp + 127) / 128;
  uint32_t cols = 32;
  while (cols < (uint32_t)(P.nb1 * CP)) cols <<= 1;
  if (cols > 512) return ET_ERR_UNIMPLEMENTED;
  P.tmem_cols = cols;
  int dev = 0, max_smem = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + 64 > max_smem) return ET_ERR_UNIMPLEMENTED;
  ET_CHECK_CUDA(cudaFuncSetAttribute(evsnet_tc_kernel<CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int tiles = ((P.W + TW - 1) / TW) * ((P.H + TH - 1) / TH);
  evsnet_tc_kernel<CP><<<tiles, kThreads, smem, stream>>>(
      P, logl, net->w, net->b, st->V, st->last_l, events, cap,
      reinterpret_cast<unsigned long long*>(n_events), I_out, spikes);
  ET_CHECK_LAUNCH();
  return ET_OK;
}

}  // namespace

int et_evsnet_forward_bf16(const float* logl, int32_t F, const et_evsnet_weights* net,
                           et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                           int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream) {
  // covered shape: plain stack of 3x3 spatial convolutions, at least two layers
  if (net->kind != ET_NET_STACK || net->ks != 3 || net->kt != 1 || net->n_layers < 2 ||
      net->n_layers > 6 || net->C > 32)
    return ET_ERR_UNIMPLEMENTED;
  if (net->C <= 16)
    return launch<16>(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
  return launch<32>(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
}
