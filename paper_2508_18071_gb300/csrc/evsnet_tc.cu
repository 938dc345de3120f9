// EvSNet forward on the tcgen05 tensor cores for the spatial form: a stack of
// 3x3 convolutions with ReLU (Eq. 5 with kernel extent in space), the
// point-wise projection (Eq. 6) and BiLIF (Eq. 2-3), for up to 32 channels.
// Two operand precisions, FP32 accumulation in TMEM for both:
//   BF16 (kind::f16): weights and layer inputs rounded to BF16;
//   FP8  (kind::f8f6f4, E4M3): weights scaled per output channel and layer
//        inputs scaled per layer, tile and step, each by the power of two that
//        brings a bound on its absolute maximum to at most 448 (E4M3's largest
//        finite).  Weights: their maximum.  Layer inputs: layer 0's output is
//        bounded by the tile's largest log difference times each channel's
//        sum of |w0|; the output of tensor-core layer l by the largest value of
//        its own input (taken while that input was written) times each output
//        channel's sum of |w_l|, plus the bias -- no second pass over the
//        accumulators.  E4M3 is a floating-point format, so a scale a few
//        powers of two above the tight one costs precision only in values
//        that fall below its normal range (2^-6 of the scale).
//
// Each CTA owns a 32 x 16 pixel tile for the whole call and walks the frames
// in order; the membrane potentials of its pixels stay in shared memory.  For
// one step:
//   * the frame tile plus an L-pixel halo is loaded (X_k = l_k - l_{k-1}, Eq. 1);
//   * layer 0 (one input channel, 9 MACs per output) runs on CUDA cores;
//   * every further layer is an implicit GEMM on the tensor core.  Activations
//     live on a padded grid of width Wp = 32 + 2L in the K-major, no-swizzle
//     operand layout (16-byte rows per plane: 8 BF16 or 16 FP8 channels), so
//     the A operand of tap (dy, dx) is the same buffer with its start address
//     moved by (dy Wp + dx) rows: no im2col.  An MMA has M = 128 padded
//     positions, N = channels and K = 32 bytes of operand: 16 BF16 channels of
//     one tap, 32 FP8 channels of one tap, or -- for 16 FP8 channels -- two
//     taps at once (the descriptor's leading-byte offset is the distance between
//     the two taps' rows);
//   * four warps read the accumulators back (tcgen05.ld, 32 lanes each), undo
//     the scales, add the bias, apply ReLU and the image-border zero padding,
//     and write the next layer's operand -- or, for the last layer, project to
//     one current per pixel in FP32 and run BiLIF and the event append.
// Positions in the halo that a layer does not need are computed and ignored
// (the "garbage columns" of the padded grid); they never feed a needed output.
#include "et_internal.cuh"
#include "event_emit.cuh"
#include "evsnet_common.h"
#include "tc_ptx.cuh"
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <algorithm>

namespace {

constexpr int TW = 32, TH = 16;
constexpr int kThreads = 256;         // 8 warps: warp w reads TMEM lanes 32 (w % 4) of the even (w < 4) or odd M blocks
constexpr uint32_t kWaitIters = 1u << 22;
int64_t g_wait_budget = -1;          // < 0: kWaitIters
constexpr unsigned long long kTimeoutBit = 1ull << 62;
constexpr float kE4M3Max = 448.0f;

struct TcParams {
  int H, W, F, f0, t0, L, C;
  float beta, vth, reset;
  int Wp, Hp, rows;                     // padded grid
  int plane;                            // bytes per 16-byte-row plane of one activation buffer
  int act_bytes, wB_bytes, layer_wB;    // per activation buffer; all / one layer's weights
  int off_act1, off_wB, off_f32, off_cur, off_prev, off_V;  // smem byte offsets
  int nb1;                              // M blocks of layer 1 (the widest)
  uint32_t tmem_cols;
  uint32_t wait_iters;                  // bound of the per-layer MMA waits
};

// smallest power of two >= x / 448 (1 for x == 0): the E4M3 scale of a tensor
// whose absolute maximum is x
__device__ __forceinline__ float e4m3_scale(float x) {
  if (!(x > 0.0f)) return 1.0f;
  int e;
  const float m = frexpf(x / kE4M3Max, &e);   // x / 448 = m 2^e, m in [0.5, 1)
  return ldexpf(1.0f, m == 0.5f ? e - 1 : e);
}

__device__ __forceinline__ uint8_t to_e4m3(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// store CP channel values (already scaled for FP8) as one operand row
template <int CP, bool kF8>
__device__ __forceinline__ void store_row(unsigned char* buf, int plane, int m, const float* v) {
  if constexpr (kF8) {
    __align__(16) __nv_fp8x2_storage_t h[CP / 2];
#pragma unroll
    for (int c = 0; c < CP / 2; ++c)
      h[c] = __nv_cvt_float2_to_fp8x2(make_float2(v[2 * c], v[2 * c + 1]), __NV_SATFINITE, __NV_E4M3);
#pragma unroll
    for (int p = 0; p < CP / 16; ++p)
      *reinterpret_cast<uint4*>(buf + p * plane + m * 16) = reinterpret_cast<const uint4*>(h)[p];
  } else {
    __align__(16) __nv_bfloat162 h[CP / 2];
#pragma unroll
    for (int c = 0; c < CP / 2; ++c) h[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
#pragma unroll
    for (int p = 0; p < CP / 8; ++p)
      *reinterpret_cast<uint4*>(buf + p * plane + m * 16) = reinterpret_cast<const uint4*>(h)[p];
  }
}

// number of 32-byte K steps per layer
template <int CP, bool kF8>
__host__ __device__ constexpr int ksteps() { return kF8 ? (CP == 16 ? 5 : 9) : 9 * CP / 16; }

__device__ __forceinline__ int tap_offset(int t, int Wp) { return (t / 3 - 1) * Wp + (t % 3 - 1); }

template <int CP, bool kF8>
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
  __shared__ unsigned int amax_bits;
  __shared__ float in_scale;            // FP8: scale of the current layer input
  __shared__ float out_scale;           // FP8: scale of the current layer output (next input)
  constexpr int KS = ksteps<CP, kF8>();
  constexpr int EB = kF8 ? 1 : 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = (P.W + TW - 1) / TW;
  const int ox = (blockIdx.x % tiles_x) * TW, oy = (blockIdx.x / tiles_x) * TH;
  const int L = P.L, Wp = P.Wp, Hp = P.Hp, C = P.C;
  const int64_t npix = (int64_t)P.H * P.W;
  // one operand buffer, rewritten in place: a layer's epilogue runs after all
  // of its MMAs have completed
  unsigned char* act[2] = {sm, sm};
  unsigned char* wB = sm + P.off_wB;
  float* f32 = reinterpret_cast<float*>(sm + P.off_f32);
  float* w0 = f32;                        // [CP][9]
  float* bs = w0 + CP * 9;                // [L][CP]
  float* wp = bs + L * CP;                // [CP] projection
  float* bp = wp + CP;                    // [1] (+ padding)
  float* sw = bp + 4;                     // [L][CP] FP8 weight scales
  float* l0b = sw + L * CP;               // [CP] sum_t |w0[c][t]| (FP8 layer-0 bound)
  float* gl = l0b + CP;                   // [L][CP] sum |w_l[c][.][.]| (FP8 bounds of layers 1..)
  float* cur = reinterpret_cast<float*>(sm + P.off_cur);
  float* prev = reinterpret_cast<float*>(sm + P.off_prev);
  float* Vs = reinterpret_cast<float*>(sm + P.off_V);

  // ---- one-time set-up: zero operands, stage weights, membrane potentials
  for (int i = tid; i < P.act_bytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  // packed FP32 weights: layer 0 [C][1][1][3][3], layers 1.. [C][C][1][3][3], projection [C]
  for (int i = tid; i < CP * 9; i += kThreads) {
    const int c = i / 9, t = i % 9;
    w0[i] = c < C ? wg[c * 9 + t] : 0.0f;
  }
  for (int c = tid; c < CP; c += kThreads) {
    float a = 0.0f;
    if (c < C)
      for (int t = 0; t < 9; ++t) a += fabsf(wg[c * 9 + t]);
    l0b[c] = a;
  }
  for (int i = tid; i < L * CP; i += kThreads) {
    const int l = i / CP, c = i % CP;
    bs[i] = c < C ? bg[l * C + c] : 0.0f;
    float s = 1.0f, g = 0.0f;
    if (kF8 && l >= 1 && c < C) {
      float mx = 0.0f;
      for (int k = 0; k < C * 9; ++k) {
        const float a = fabsf(wg[9 * C + (l - 1) * C * C * 9 + c * C * 9 + k]);
        mx = fmaxf(mx, a);
        g += a;
      }
      s = e4m3_scale(mx);
    }
    sw[i] = s;
    gl[i] = g;
  }
  const int wproj = 9 * C + (L - 1) * C * C * 9;
  for (int i = tid; i < CP; i += kThreads) wp[i] = i < C ? wg[wproj + i] : 0.0f;
  if (tid == 0) bp[0] = bg[L * C];
  __syncthreads();
  // tensor-core weights: per layer l >= 1 and K step j, B[n = cout][k] as two
  // 16-byte columns of CP rows
  for (int i = tid; i < (L - 1) * KS * 2 * CP * (16 / EB); i += kThreads) {
    const int e = i % (16 / EB);               // element within the 16-byte row
    const int n = (i / (16 / EB)) % CP;
    const int col = (i / (16 / EB * CP)) % 2;
    const int j = (i / (16 / EB * CP * 2)) % KS;
    const int l = 1 + i / (16 / EB * CP * 2 * KS);
    int t, k;
    if (!kF8) { t = j / (CP / 16); k = 16 * (j % (CP / 16)) + 8 * col + e; }
    else if (CP == 32) { t = j; k = 16 * col + e; }
    else { t = 2 * j + col; k = e; }
    float v = 0.0f;
    if (t < 9 && n < C && k < C) v = wg[9 * C + (l - 1) * C * C * 9 + (n * C + k) * 9 + t];
    unsigned char* dst = wB + (size_t)(l - 1) * P.layer_wB + j * (2 * CP * 16) + col * (CP * 16) + n * 16 + e * EB;
    if (kF8) *dst = to_e4m3(v / sw[l * CP + n]);
    else *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
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
  if (tid == 0) { mbar_init(&mma_bar, 1); bail = 0; amax_bits = 0u; }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0;
  const uint32_t idesc = kF8 ? umma_idesc_e4m3(128, CP) : umma_idesc_bf16(128, CP);

  for (int f = (P.f0 == 0 ? 0 : 1); f < P.F && !bail; ++f) {
    // ---- frame tile and layer 0 on CUDA cores.  FP8: layer 0's input scale
    // comes from a bound, |h_c| <= |b_c| + max|X| sum_t |w0[c][t]|, over the
    // tile's log differences (E4M3's range absorbs the slack)
    float amx = 0.0f;
    for (int i = tid; i < Hp * Wp; i += kThreads) {
      const int gx = ox - L + i % Wp, gy = oy - L + i / Wp;
      const float v = (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H)
                          ? __ldg(logl + (int64_t)f * npix + (int64_t)gy * P.W + gx) : 0.0f;
      cur[i] = v;
      if (kF8) amx = fmaxf(amx, fabsf(v - prev[i]));
    }
    if (kF8) atomicMax(&amax_bits, __float_as_uint(amx));
    __syncthreads();
    if (kF8) {
      if (tid == 0) {
        const float xm = __uint_as_float(amax_bits);
        float bound = 0.0f;
        for (int c = 0; c < C; ++c) bound = fmaxf(bound, fabsf(bs[c]) + xm * l0b[c]);
        in_scale = e4m3_scale(bound);
        amax_bits = 0u;                 // next: the largest layer-0 output
      }
      __syncthreads();
    }
    float amx0 = 0.0f;
    {
      const float inv = kF8 ? 1.0f / in_scale : 1.0f;
      for (int i = tid; i < (Hp - 2) * (Wp - 2); i += kThreads) {
        const int py = 1 + i / (Wp - 2), px = 1 + i % (Wp - 2);
        const int gx = ox - L + px, gy = oy - L + py;
        const int m = py * Wp + px;
        float h[CP];
        const bool in = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
        if (in) {
          float x[9];
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const int q = m + tap_offset(t, Wp);
            x[t] = cur[q] - prev[q];
          }
#pragma unroll
          for (int c = 0; c < CP; ++c) {
            float a = bs[c];
#pragma unroll
            for (int t = 0; t < 9; ++t) a = fmaf(w0[c * 9 + t], x[t], a);
            h[c] = fmaxf(a, 0.0f);
          }
        } else {
#pragma unroll
          for (int c = 0; c < CP; ++c) h[c] = 0.0f;
        }
        if (kF8) {
#pragma unroll
          for (int c = 0; c < CP; ++c) { amx0 = fmaxf(amx0, h[c]); h[c] *= inv; }
        }
        store_row<CP, kF8>(act[0], P.plane, m, h);
      }
    }
    if (kF8) atomicMax(&amax_bits, __float_as_uint(amx0));
    if (!kF8 && tid == 0) in_scale = 1.0f;
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
      const float s_in = in_scale;
      if (tid == 0) {
        const uint32_t abase = smem_u32(ain), bbase = smem_u32(wB + (size_t)(l - 1) * P.layer_wB);
        for (int b = 0; b < nb; ++b) {
          const int m0 = m_start + b * 128;
          for (int j = 0; j < KS; ++j) {
            uint32_t a_start, a_lbo;
            if (!kF8) {
              const int t = j / (CP / 16), s = j % (CP / 16);
              a_start = abase + (2 * s) * P.plane + (m0 + tap_offset(t, Wp)) * 16;
              a_lbo = P.plane;
            } else if (CP == 32) {
              a_start = abase + (m0 + tap_offset(j, Wp)) * 16;
              a_lbo = P.plane;
            } else {
              // taps 2j and 2j + 1 (tap 9 does not exist: its weights are zero and
              // it reads the row after tap 8)
              const int t0 = 2 * j;
              const int o0 = tap_offset(t0, Wp), o1 = t0 + 1 < 9 ? tap_offset(t0 + 1, Wp) : o0 + 1;
              a_start = abase + (m0 + o0) * 16;
              a_lbo = (uint32_t)(o1 - o0) * 16;
            }
            const uint64_t ad = umma_desc(a_start, a_lbo, 128);
            const uint64_t bd = umma_desc(bbase + j * (2 * CP * 16), CP * 16, 128);
            if constexpr (kF8) umma_e4m3(tmem + b * CP, ad, bd, idesc, j != 0);
            else umma_bf16(tmem + b * CP, ad, bd, idesc, j != 0);
          }
        }
        umma_commit(&mma_bar);
        if (kF8 && l < L - 1) {
          // the output's bound: h_c <= max(0, b_c + G_c max|input|), with a
          // margin for the E4M3 roundings of weights and inputs
          const float xm = 1.25f * __uint_as_float(amax_bits);
          float bound = 0.0f;
          for (int c = 0; c < C; ++c) bound = fmaxf(bound, fmaf(gl[l * CP + c], xm, bs[l * CP + c]));
          out_scale = e4m3_scale(bound);
        }
      }
      const bool ok = mbar_wait(&mma_bar, phase, P.wait_iters);
      phase ^= 1;
      if (!ok) {
        if (lane == 0) atomicOr(n_events, kTimeoutBit);
        bail = 1;
      }
      tc_fence_after();
      if (tid == 0) amax_bits = 0u;
      __syncthreads();
      if (bail) break;
      const bool last = l == L - 1;
      {
        const float inv_next = (kF8 && !last) ? 1.0f / out_scale : 1.0f;
        float amax = 0.0f;
        for (int b = warp >> 2; b < nb; b += 2) {
          const int m = m_start + b * 128 + (warp & 3) * 32 + lane;
          float acc[CP];
#pragma unroll
          for (int jj = 0; jj < CP / 16; ++jj)
            tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + b * CP + jj * 16, acc + jj * 16);
          const int py = m / Wp, px = m % Wp;
          const bool need = m < Hp * Wp && py >= l + 1 && py < Hp - l - 1 && px >= l + 1 && px < Wp - l - 1;
          const int gx = ox - L + px, gy = oy - L + py;
          const bool inimg = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
          float h[CP];
#pragma unroll
          for (int c = 0; c < CP; ++c) {
            const float deq = kF8 ? s_in * sw[l * CP + c] : 1.0f;
            h[c] = (need && inimg) ? fmaxf(fmaf(acc[c], deq, bs[l * CP + c]), 0.0f) : 0.0f;
          }
          if (!last) {
            if (need) {
              if (kF8) {
#pragma unroll
                for (int c = 0; c < CP; ++c) { amax = fmaxf(amax, h[c]); h[c] *= inv_next; }
              }
              store_row<CP, kF8>(aout, P.plane, m, h);
            }
          } else {
            uint32_t nev = 0;
            int S = 0;
            if (need && inimg) {
              float I = bp[0];
#pragma unroll
              for (int c = 0; c < CP; ++c) I = fmaf(wp[c], h[c], I);
              const int ti = (py - L) * TW + (px - L);
              const float vp = P.beta * Vs[ti] + I;
              S = vp >= P.vth ? 1 : (vp <= -P.vth ? -1 : 0);
              Vs[ti] = vp - P.reset * (float)S;
              nev = (S != 0 && P.t0 + f >= 0) ? 1u : 0u;   // delayed labels below 0: none
              const int64_t q = (int64_t)(f - (P.f0 == 0 ? 0 : 1)) * npix + (int64_t)gy * P.W + gx;
              if (I_out) I_out[q] = I;
              if (spikes) spikes[q] = (int8_t)S;
            }
            emit_events_warp(events, cap, n_events, nev, (uint32_t)gx, (uint32_t)gy, (uint32_t)(P.t0 + f), S);
          }
        }
        if (kF8 && !last) {
          // the largest value of the next layer's input; its scale is this output's
          atomicMax(&amax_bits, __float_as_uint(amax));
          if (tid == 0) in_scale = out_scale;
        }
      }
      tc_fence_before();
    }
    if (tid == 0) amax_bits = 0u;
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

template <int CP, bool kF8>
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
  P.act_bytes = (CP * (kF8 ? 1 : 2) / 16) * P.plane;
  P.layer_wB = ksteps<CP, kF8>() * 2 * CP * 16;
  P.wB_bytes = (P.L - 1) * P.layer_wB;
  auto al = [](int x) { return (x + 1023) & ~1023; };
  P.off_act1 = 0;
  P.off_wB = al(P.act_bytes);
  P.off_f32 = P.off_wB + al(P.wB_bytes);
  const int f32_bytes = 4 * (CP * 9 + P.L * CP + CP + 4 + P.L * CP + CP + P.L * CP);
  P.off_cur = P.off_f32 + al(f32_bytes);
  P.off_prev = P.off_cur + al(4 * P.Hp * P.Wp);
  P.off_V = P.off_prev + al(4 * P.Hp * P.Wp);
  const int smem = P.off_V + al(4 * TW * TH);
  P.nb1 = ((P.Hp - 4) * P.Wp + 127) / 128;
  uint32_t cols = 32;
  while (cols < (uint32_t)(P.nb1 * CP)) cols <<= 1;
  if (cols > 512) return ET_ERR_UNIMPLEMENTED;
  P.tmem_cols = cols;
  P.wait_iters = et_tc_wait_iters();
  int dev = 0, max_smem = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + 1024 + 64 > max_smem) return ET_ERR_UNIMPLEMENTED;
  ET_CHECK_CUDA(cudaFuncSetAttribute(evsnet_tc_kernel<CP, kF8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int tiles = ((P.W + TW - 1) / TW) * ((P.H + TH - 1) / TH);
  evsnet_tc_kernel<CP, kF8><<<tiles, kThreads, smem, stream>>>(
      P, logl, net->w, net->b, st->V, st->last_l, events, cap,
      reinterpret_cast<unsigned long long*>(n_events), I_out, spikes);
  ET_CHECK_LAUNCH();
  return ET_OK;
}

}  // namespace

extern "C" void et_set_wait_budget(int64_t polls) { g_wait_budget = polls; }

uint32_t et_tc_wait_iters() {
  return g_wait_budget < 0 ? kWaitIters : (uint32_t)std::min<int64_t>(g_wait_budget, 0xFFFFFFFFll);
}

int et_evsnet_forward_tc(const float* logl, int32_t F, const et_evsnet_weights* net,
                         et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                         int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream) {
  // covered shape: plain stack of 3x3 spatial convolutions, at least two layers
  if (net->kind != ET_NET_STACK || net->ks != 3 || net->kt != 1 || net->n_layers < 2 ||
      net->n_layers > 6 || net->C > 32)
    return ET_ERR_UNIMPLEMENTED;
  const bool f8 = net->dtype == ET_FP8;
  if (net->C <= 16)
    return f8 ? launch<16, true>(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream)
              : launch<16, false>(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
  return f8 ? launch<32, true>(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream)
            : launch<32, false>(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, stream);
}
