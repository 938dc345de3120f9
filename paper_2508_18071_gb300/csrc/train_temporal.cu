// Training of the paper's pixel-wise temporal EvSNet (Sec. 3.3, Eq. 5-6:
// convolutions along time only, kernel kt, optional residual blocks, a
// point-wise projection and BiLIF) on the GPU, FP32.
//
// With a 1x1 spatial extent every pixel is an independent 1-D network over the
// clip, so the activations are kept for the whole clip (no segment recompute
// of the convolutions is needed for the temporal coupling): layout
// [B][K][H W][C], one pixel-step's channels contiguous.  BiLIF keeps V at the
// start of every ckpt_every steps and runs its reverse recursion per segment,
// as the spatial form does.
//
// Convolution along time, causal: out[k][co] = b[co] + sum_ci,tau
// w[co][ci][tau] in[k - (kt - 1) + tau][ci]; steps before the clip are zero.
// Residual blocks (Eq. 5): a_i = ReLU(conv_{2i-1}(h_{i-1})),
// h_i = ReLU(h_{i-1} + conv_{2i}(a_i)).
#include <algorithm>
#include "et_internal.cuh"
#include "evsnet_common.h"
#include "train_api.h"

#define ET_TRY(expr)                 \
  do {                               \
    const int rc_ = (expr);          \
    if (rc_ != ET_OK) return rc_;    \
  } while (0)

namespace {

constexpr int kMaxC = 16;
constexpr int kMaxKt = 9;
constexpr float kPi = 3.14159265358979323846f;

// packed weight offset of layer l; n0 = weights per output channel of layer 0
// (kt, or ks0 * ks0 for a spatial stem)
inline int64_t twofs(int l, int C, int kt, int n0) {
  return l == 0 ? 0 : (int64_t)C * n0 + (int64_t)(l - 1) * C * C * kt;
}
inline int layer0_taps(const et_evsnet_weights* net) {
  return net->ks0 > 0 ? net->ks0 * net->ks0 : net->kt;
}

// ------------------------------------------------------- forward conv, layer 0
// One thread per (clip, step, pixel); X read as l_{k+1} - l_k from the clip's
// log frames.  A one-layer network also writes the projection I = bp + wp . out.
__global__ void __launch_bounds__(256, 4)
tconv_fwd(const float* __restrict__ logl, int B, int K, int64_t hw, int C, int kt,
          const float* __restrict__ w, const float* __restrict__ b, float* __restrict__ out,
          const float* __restrict__ wp, const float* __restrict__ bp, float* __restrict__ I) {
  constexpr int Cin = 1;
  __shared__ float sw[kMaxC * kMaxC * kMaxKt];
  for (int i = threadIdx.x; i < C * Cin * kt; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * K * hw) return;
  const int64_t p = idx % hw;
  const int k = (int)((idx / hw) % K), bc = (int)(idx / (hw * K));
  float acc[kMaxC];
#pragma unroll
  for (int co = 0; co < kMaxC; ++co) acc[co] = co < C ? b[co] : 0.0f;
  for (int tau = 0; tau < kt; ++tau) {
    const int kk = k - (kt - 1) + tau;
    if (kk < 0) continue;
    const float* lf = logl + (int64_t)bc * (K + 1) * hw;
    const float x = lf[(int64_t)(kk + 1) * hw + p] - lf[(int64_t)kk * hw + p];
#pragma unroll
    for (int co = 0; co < kMaxC; ++co)
      if (co < C) acc[co] += sw[co * kt + tau] * x;
  }
  float* dst = out + idx * C;
  float Iv = bp ? bp[0] : 0.0f;
#pragma unroll
  for (int co = 0; co < kMaxC; ++co) {
    if (co >= C) break;
    const float a = fmaxf(acc[co], 0.0f);
    dst[co] = a;
    if (I) Iv += wp[co] * a;
  }
  if (I) I[idx] = Iv;
}

// ------------------------------------------------- forward, spatial stem
// Layer 0 as a one-step ks0 x ks0 convolution of X (zero outside the image);
// one thread per (clip, step, pixel), taps in row-major order.
constexpr int kMaxStem = 7;
__global__ void __launch_bounds__(256, 4)
tstem_fwd(const float* __restrict__ logl, int B, int K, int H, int W, int C, int ks0,
          const float* __restrict__ w, const float* __restrict__ b, float* __restrict__ out,
          const float* __restrict__ wp, const float* __restrict__ bp, float* __restrict__ I) {
  __shared__ float sw[kMaxStem * kMaxStem][kMaxC];   // [tap][co]
  for (int i = threadIdx.x; i < C * ks0 * ks0; i += blockDim.x) sw[i % (ks0 * ks0)][i / (ks0 * ks0)] = w[i];
  __syncthreads();
  const int64_t hw = (int64_t)H * W;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * K * hw) return;
  const int64_t p = idx % hw;
  const int k = (int)((idx / hw) % K), bc = (int)(idx / (hw * K));
  const int y = (int)(p / W), x = (int)(p % W), r0 = ks0 >> 1;
  const float* l1 = logl + ((int64_t)bc * (K + 1) + k + 1) * hw;
  const float* l0 = l1 - hw;
  float acc[kMaxC];
#pragma unroll
  for (int co = 0; co < kMaxC; ++co) acc[co] = co < C ? b[co] : 0.0f;
  for (int dy = 0; dy < ks0; ++dy) {
    const int yy = y + dy - r0;
    if (yy < 0 || yy >= H) continue;
    for (int dx = 0; dx < ks0; ++dx) {
      const int xx = x + dx - r0;
      if (xx < 0 || xx >= W) continue;
      const int64_t q = (int64_t)yy * W + xx;
      const float v = l1[q] - l0[q];
      const float* wt = sw[dy * ks0 + dx];
#pragma unroll
      for (int co = 0; co < kMaxC; ++co)
        if (co < C) acc[co] = fmaf(wt[co], v, acc[co]);
    }
  }
  float* dst = out + idx * C;
  float Iv = bp ? bp[0] : 0.0f;
#pragma unroll
  for (int co = 0; co < kMaxC; ++co) {
    if (co >= C) break;
    const float a = fmaxf(acc[co], 0.0f);
    dst[co] = a;
    if (I) Iv += wp[co] * a;
  }
  if (I) I[idx] = Iv;
}

// --------------------------------------------------------------------- BiLIF
__device__ __forceinline__ float sg(float x, float alpha) {
  const float u = 0.5f * kPi * alpha * x;
  return 0.5f * alpha / (1.0f + u * u);
}

// One thread per (clip, pixel) over the whole clip; V at the start of every
// segment goes to V_ckpt [B][n_ckpt][hw].
__global__ void tbilif_fwd(const float* __restrict__ I, int B, int K, int64_t hw, int ck, int n_ckpt,
                           float beta, float vth, float reset, float* __restrict__ V_ckpt,
                           int8_t* __restrict__ spikes, float* __restrict__ S_on,
                           float* __restrict__ S_off, float* __restrict__ I_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * hw) return;
  const int bc = (int)(i / hw);
  const int64_t p = i % hw;
  float v = 0.0f;
  for (int k = 0; k < K; ++k) {
    if (k % ck == 0) V_ckpt[((int64_t)bc * n_ckpt + k / ck) * hw + p] = v;
    const int64_t o = ((int64_t)bc * K + k) * hw + p;
    const float Iv = I[o];
    const float vp = beta * v + Iv;
    const float on = vp >= vth ? 1.0f : 0.0f, off = -vp >= vth ? 1.0f : 0.0f;
    v = vp - reset * (on - off);
    spikes[o] = (int8_t)(on - off);
    if (S_on) { S_on[o] = on; S_off[o] = off; }
    if (I_out) I_out[o] = Iv;
  }
}

// Reverse recursion per segment (V' recomputed from the segment's checkpoint).
__global__ void tbilif_bwd(const float* __restrict__ I, int B, int K, int64_t hw, int ck, int n_ckpt,
                           float beta, float vth, float reset, float alpha,
                           const float* __restrict__ V_ckpt, const float* __restrict__ dSon,
                           const float* __restrict__ dSoff, float* __restrict__ dI) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * hw) return;
  const int bc = (int)(i / hw);
  const int64_t p = i % hw;
  float g = 0.0f;
  for (int s = n_ckpt - 1; s >= 0; --s) {
    const int k0 = s * ck, nseg = min(ck, K - k0);
    float vps[kMaxSeg];
    float v = V_ckpt[((int64_t)bc * n_ckpt + s) * hw + p];
    for (int j = 0; j < nseg; ++j) {
      const float vp = beta * v + I[((int64_t)bc * K + k0 + j) * hw + p];
      const float on = vp >= vth ? 1.0f : 0.0f, off = -vp >= vth ? 1.0f : 0.0f;
      v = vp - reset * (on - off);
      vps[j] = vp;
    }
    for (int j = nseg - 1; j >= 0; --j) {
      const float vp = vps[j];
      const float a = sg(vp - vth, alpha), c = sg(-vp - vth, alpha);
      const int64_t o = ((int64_t)bc * K + k0 + j) * hw + p;
      const float gvp = g * (1.0f - reset * (a + c)) + dSon[o] * a - dSoff[o] * c;
      dI[o] = gvp;
      g = gvp * beta;
    }
  }
}

// ------------------------------------------------------ projection backward
// dz[c] = dI wp[c] 1(h > 0); grad wp[c] += sum dI h[c]; grad bp += sum dI.
__global__ void __launch_bounds__(256)
tproj_bwd(const float* __restrict__ dI, const float* __restrict__ h, int64_t n, int C,
          const float* __restrict__ wp, float* __restrict__ dz, float* __restrict__ gwp,
          float* __restrict__ gbp) {
  __shared__ float red[kMaxC + 1][8];
  float acc[kMaxC + 1];
#pragma unroll
  for (int c = 0; c <= kMaxC; ++c) acc[c] = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = dI[i];
    acc[kMaxC] += d;
#pragma unroll
    for (int c = 0; c < kMaxC; ++c) {
      if (c >= C) break;
      const float a = h[i * C + c];
      acc[c] += d * a;
      dz[i * C + c] = a > 0.0f ? d * wp[c] : 0.0f;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c <= kMaxC; ++c) {
    float v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[c][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < C || threadIdx.x == kMaxC) {
    float v = 0.0f;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) v += red[threadIdx.x][wv];
    if (threadIdx.x < C) atomicAdd(gwp + threadIdx.x, v);
    else atomicAdd(gbp, v);
  }
}

// ------------------------------------------------- weight backward, layer 0
// grad w[co][tau] += sum dz[k][co] X[k - kt + 1 + tau]; grad b[co] += sum dz[k][co].
// Persistent blocks stage 128 pixel-steps at a time in shared memory; each
// thread owns a (co, tau) entry, one atomic per entry per block.
constexpr int kPts = 128;
__global__ void __launch_bounds__(256)
tconv_bwd_weight(const float* __restrict__ dz, const float* __restrict__ logl, int B, int K,
                 int64_t hw, int C, int kt, float* __restrict__ gw, float* __restrict__ gb) {
  constexpr int Cin = 1;
  __shared__ float sd[kPts][kMaxC];
  __shared__ float sx[kPts][kMaxKt + 1];   // [tau], padded
  constexpr int kPer = (kMaxC * kMaxKt + kMaxC + 255) / 256;
  float acc[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) acc[j] = 0.0f;
  const int nent = C * Cin * kt + C;
  const int64_t npts = (int64_t)B * K * hw;
  for (int64_t c0 = (int64_t)blockIdx.x * kPts; c0 < npts; c0 += (int64_t)gridDim.x * kPts) {
    __syncthreads();
    for (int i = threadIdx.x; i < kPts * C; i += blockDim.x) {
      const int pt = i / C, co = i % C;
      const int64_t idx = c0 + pt;
      sd[pt][co] = idx < npts ? dz[idx * C + co] : 0.0f;
    }
    for (int i = threadIdx.x; i < kPts * Cin * kt; i += blockDim.x) {
      const int pt = i / (Cin * kt), r = i % (Cin * kt), ci = r / kt, tau = r % kt;
      const int64_t idx = c0 + pt;
      float v = 0.0f;
      if (idx < npts) {
        const int64_t p = idx % hw;
        const int k = (int)((idx / hw) % K), bc = (int)(idx / (hw * K));
        const int kk = k - (kt - 1) + tau;
        if (kk >= 0) {
          const float* lf = logl + (int64_t)bc * (K + 1) * hw;
          v = lf[(int64_t)(kk + 1) * hw + p] - lf[(int64_t)kk * hw + p];
        }
      }
      sx[pt][ci * kt + tau] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int e = threadIdx.x + j * 256;
      if (e >= nent) break;
      float s = 0.0f;
      if (e < C * Cin * kt) {
        const int co = e / (Cin * kt), r = e % (Cin * kt);
        for (int pt = 0; pt < kPts; ++pt) s += sd[pt][co] * sx[pt][r];
      } else {
        const int co = e - C * Cin * kt;
        for (int pt = 0; pt < kPts; ++pt) s += sd[pt][co];
      }
      acc[j] += s;
    }
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int e = threadIdx.x + j * 256;
    if (e >= nent) break;
    if (e < C * Cin * kt) atomicAdd(gw + e, acc[j]);
    else atomicAdd(gb + (e - C * Cin * kt), acc[j]);
  }
}

// -------------------------------------- weight backward, spatial stem
// grad w[co][tap] += sum dz[k][co] X_nbr(tap)[k]; grad b[co] += sum dz[k][co]:
// the layer-0 kernel above with the taps running over the ks0 x ks0
// neighbourhood of the current step instead of over time.
__global__ void __launch_bounds__(256)
tstem_bwd_weight(const float* __restrict__ dz, const float* __restrict__ logl, int B, int K, int H,
                 int W, int C, int ks0, float* __restrict__ gw, float* __restrict__ gb) {
  constexpr int kTaps = kMaxStem * kMaxStem;
  __shared__ float sd[kPts][kMaxC];
  __shared__ float sx[kPts][kTaps + 1];
  constexpr int kPer = (kMaxC * kTaps + kMaxC + 255) / 256;
  float acc[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) acc[j] = 0.0f;
  const int nt = ks0 * ks0, r0 = ks0 >> 1;
  const int nent = C * nt + C;
  const int64_t hw = (int64_t)H * W;
  const int64_t npts = (int64_t)B * K * hw;
  for (int64_t c0 = (int64_t)blockIdx.x * kPts; c0 < npts; c0 += (int64_t)gridDim.x * kPts) {
    __syncthreads();
    for (int i = threadIdx.x; i < kPts * C; i += blockDim.x) {
      const int pt = i / C, co = i % C;
      const int64_t idx = c0 + pt;
      sd[pt][co] = idx < npts ? dz[idx * C + co] : 0.0f;
    }
    for (int i = threadIdx.x; i < kPts * nt; i += blockDim.x) {
      const int pt = i / nt, tap = i % nt;
      const int64_t idx = c0 + pt;
      float v = 0.0f;
      if (idx < npts) {
        const int64_t p = idx % hw;
        const int k = (int)((idx / hw) % K), bc = (int)(idx / (hw * K));
        const int yy = (int)(p / W) + tap / ks0 - r0, xx = (int)(p % W) + tap % ks0 - r0;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
          const float* l1 = logl + ((int64_t)bc * (K + 1) + k + 1) * hw;
          const int64_t q = (int64_t)yy * W + xx;
          v = l1[q] - l1[q - hw];
        }
      }
      sx[pt][tap] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int e = threadIdx.x + j * 256;
      if (e >= nent) break;
      float s = 0.0f;
      if (e < C * nt) {
        const int co = e / nt, tap = e % nt;
        for (int pt = 0; pt < kPts; ++pt) s += sd[pt][co] * sx[pt][tap];
      } else {
        const int co = e - C * nt;
        for (int pt = 0; pt < kPts; ++pt) s += sd[pt][co];
      }
      acc[j] += s;
    }
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int e = threadIdx.x + j * 256;
    if (e >= nent) break;
    if (e < C * nt) atomicAdd(gw + e, acc[j]);
    else atomicAdd(gb + (e - C * nt), acc[j]);
  }
}

// ------------------------------------------- C -> C layers, vectorised weights
// The layers with C input channels in a second form: weights staged as
// [tau][input][output], zero-padded to 16 x 16 per tap, so that one 16-byte
// shared load (the same address for the whole warp) feeds four FMAs; a
// pixel-step's 16 channels are read with 16-byte loads when C = 16.
constexpr int CP = 16;

template <bool kC16>
__device__ __forceinline__ void load_ch(const float* __restrict__ src, int C, float (&x)[CP]) {
  if (kC16) {
#pragma unroll
    for (int j = 0; j < CP / 4; ++j) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src) + j);
      x[4 * j] = v.x; x[4 * j + 1] = v.y; x[4 * j + 2] = v.z; x[4 * j + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < CP; ++c) x[c] = c < C ? __ldg(src + c) : 0.0f;
  }
}

// acc0[o] += sum_i w[i][o] x0[i] and acc1[o] += sum_i w[i][o] x1[i] for one tap's
// 16 x 16 block of shared weights: two steps per weight load
__device__ __forceinline__ void fma_block2(const float* __restrict__ w, const float (&x0)[CP],
                                           const float (&x1)[CP], int C, float (&acc0)[CP],
                                           float (&acc1)[CP]) {
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    if (i >= C) break;
    const float4* w4 = reinterpret_cast<const float4*>(w + i * CP);
#pragma unroll
    for (int j = 0; j < CP / 4; ++j) {
      const float4 v = w4[j];
      acc0[4 * j] = fmaf(v.x, x0[i], acc0[4 * j]);
      acc0[4 * j + 1] = fmaf(v.y, x0[i], acc0[4 * j + 1]);
      acc0[4 * j + 2] = fmaf(v.z, x0[i], acc0[4 * j + 2]);
      acc0[4 * j + 3] = fmaf(v.w, x0[i], acc0[4 * j + 3]);
      acc1[4 * j] = fmaf(v.x, x1[i], acc1[4 * j]);
      acc1[4 * j + 1] = fmaf(v.y, x1[i], acc1[4 * j + 1]);
      acc1[4 * j + 2] = fmaf(v.z, x1[i], acc1[4 * j + 2]);
      acc1[4 * j + 3] = fmaf(v.w, x1[i], acc1[4 * j + 3]);
    }
  }
}

// a pixel-step's channels, zero outside the clip's steps [0, K)
template <bool kC16>
__device__ __forceinline__ void load_step(const float* __restrict__ base, int k, int K, int64_t step,
                                          int C, float (&x)[CP]) {
  if (k < 0 || k >= K) {
#pragma unroll
    for (int c = 0; c < CP; ++c) x[c] = 0.0f;
  } else {
    load_ch<kC16>(base + k * step, C, x);
  }
}

// forward of a C -> C layer: out = ReLU(b + conv(in) [+ res]), the last layer
// also I = bp + wp . out.  One thread per (clip, pair of steps 2j and 2j + 1,
// pixel): each tap's weights serve both steps, the input of step k - kt + 2 + tau
// serving the second step at tap tau and the first at tau + 1.
template <bool kC16>
__global__ void __launch_bounds__(256, 3)
tconv16_fwd(const float* __restrict__ in, int B, int K, int64_t hw, int C, int kt,
            const float* __restrict__ w, const float* __restrict__ b, const float* __restrict__ res,
            float* __restrict__ out, const float* __restrict__ wp, const float* __restrict__ bp,
            float* __restrict__ I) {
  __shared__ __align__(16) float sw[kMaxKt * CP * CP];   // [tau][ci][co]
  for (int i = threadIdx.x; i < kt * CP * CP; i += blockDim.x) {
    const int co = i % CP, ci = (i / CP) % CP, tau = i / (CP * CP);
    sw[i] = (co < C && ci < C) ? w[(co * C + ci) * kt + tau] : 0.0f;
  }
  __syncthreads();
  const int KP = (K + 1) / 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * KP * hw) return;
  const int64_t p = t % hw;
  const int k = 2 * (int)((t / hw) % KP), bc = (int)(t / (hw * KP));
  const int64_t step = hw * C;
  const float* base = in + ((int64_t)bc * K * hw + p) * C;
  float acc0[CP], acc1[CP];
#pragma unroll
  for (int co = 0; co < CP; ++co) acc0[co] = acc1[co] = co < C ? b[co] : 0.0f;
  float xa[CP];
  load_step<kC16>(base, k - (kt - 1), K, step, C, xa);
  for (int tau = 0; tau < kt; ++tau) {
    float xb[CP];
    load_step<kC16>(base, k - (kt - 1) + tau + 1, K, step, C, xb);
    fma_block2(sw + tau * CP * CP, xa, xb, C, acc0, acc1);
#pragma unroll
    for (int c = 0; c < CP; ++c) xa[c] = xb[c];
  }
  auto finish = [&](float (&acc)[CP], int h) {
    const int64_t idx = ((int64_t)bc * K + k + h) * hw + p;
    float Iv = bp ? bp[0] : 0.0f;
#pragma unroll
    for (int co = 0; co < CP; ++co) {
      if (co >= C) break;
      const float z = res ? acc[co] + res[idx * C + co] : acc[co];
      acc[co] = fmaxf(z, 0.0f);
      if (I) Iv += wp[co] * acc[co];
    }
    if (kC16) {
#pragma unroll
      for (int j = 0; j < CP / 4; ++j)
        reinterpret_cast<float4*>(out + idx * C)[j] =
            make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
    } else {
#pragma unroll
      for (int co = 0; co < CP; ++co)
        if (co < C) out[idx * C + co] = acc[co];
    }
    if (I) I[idx] = Iv;
  };
  finish(acc0, 0);
  if (k + 1 < K) finish(acc1, 1);
}

// data backward: out[s][ci] = (add[s][ci] + sum_tau,co w[co][ci][tau] dz[s + kt - 1 - tau][co])
// 1(mask[s][ci] > 0); weights staged [tau][co][ci]; two steps per thread as above
template <bool kC16>
__global__ void __launch_bounds__(256, 3)
tconv16_bwd_data(const float* __restrict__ dz, int B, int K, int64_t hw, int C, int kt,
                 const float* __restrict__ w, const float* __restrict__ add,
                 const float* __restrict__ mask, float* __restrict__ out) {
  __shared__ __align__(16) float sw[kMaxKt * CP * CP];   // [tau][co][ci]
  for (int i = threadIdx.x; i < kt * CP * CP; i += blockDim.x) {
    const int ci = i % CP, co = (i / CP) % CP, tau = i / (CP * CP);
    sw[i] = (co < C && ci < C) ? w[(co * C + ci) * kt + tau] : 0.0f;
  }
  __syncthreads();
  const int KP = (K + 1) / 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * KP * hw) return;
  const int64_t p = t % hw;
  const int s = 2 * (int)((t / hw) % KP), bc = (int)(t / (hw * KP));
  const int64_t step = hw * C;
  const float* base = dz + ((int64_t)bc * K * hw + p) * C;
  float acc0[CP], acc1[CP];
#pragma unroll
  for (int ci = 0; ci < CP; ++ci) acc0[ci] = acc1[ci] = 0.0f;
  float gb[CP];   // dz[s + kt - tau] for the second step
  load_step<kC16>(base, s + kt, K, step, C, gb);
  for (int tau = 0; tau < kt; ++tau) {
    float ga[CP];
    load_step<kC16>(base, s + kt - 1 - tau, K, step, C, ga);
    fma_block2(sw + tau * CP * CP, ga, gb, C, acc0, acc1);
#pragma unroll
    for (int c = 0; c < CP; ++c) gb[c] = ga[c];
  }
  auto finish = [&](const float (&acc)[CP], int h) {
    const int64_t idx = ((int64_t)bc * K + s + h) * hw + p;
#pragma unroll
    for (int ci = 0; ci < CP; ++ci) {
      if (ci >= C) break;
      const int64_t o = idx * C + ci;
      const float v = add ? add[o] + acc[ci] : acc[ci];
      out[o] = mask[o] > 0.0f ? v : 0.0f;
    }
  };
  finish(acc0, 0);
  if (s + 1 < K) finish(acc1, 1);
}

// weight backward of a C -> C layer: grad w[co][ci][tau] += sum dz[k][co] in[k - kt + 1 + tau][ci],
// grad b[co] += sum dz[k][co].  Persistent blocks stage kPts16 pixel-steps:
// dz as [pt][16], the shifted inputs as [pt][tau][16].  Thread e < 16 kt owns
// (tap tau = e / 16, output quad e % 4, input quad (e / 4) % 4), 16 sums with
// two 16-byte shared loads per 16 FMAs; the next 16 threads own the bias sums.
constexpr int kPts16 = 64;
inline int twgrad_threads(int kt) { return (16 * kt + 16 + 31) / 32 * 32; }

template <bool kC16>
__global__ void __launch_bounds__(320)
tconv16_bwd_weight(const float* __restrict__ dz, const float* __restrict__ in, int B, int K,
                   int64_t hw, int C, int kt, float* __restrict__ gw, float* __restrict__ gb) {
  extern __shared__ __align__(16) float tsm[];
  float* sd = tsm;                      // [kPts16][CP]
  float* sx = tsm + kPts16 * CP;        // [kPts16][kt][CP]
  __shared__ int64_t s_row0[kPts16];    // offset of the point's pixel at step 0 of its clip
  __shared__ int s_k[kPts16];           // the point's step, -1 past the end
  const int e = threadIdx.x;
  const int tau = e / 16, cq = e % 4, iq = (e / 4) % 4;
  float acc[4][4] = {};
  float bsum = 0.0f;
  const int64_t npts = (int64_t)B * K * hw, step = hw * C;
  for (int64_t c0 = (int64_t)blockIdx.x * kPts16; c0 < npts; c0 += (int64_t)gridDim.x * kPts16) {
    __syncthreads();
    for (int pt = threadIdx.x; pt < kPts16; pt += blockDim.x) {
      const int64_t idx = c0 + pt;
      if (idx < npts) {
        const int64_t p = idx % hw;
        const int k = (int)((idx / hw) % K), bc = (int)(idx / (hw * K));
        s_row0[pt] = ((int64_t)bc * K * hw + p) * C;
        s_k[pt] = k;
      } else {
        s_row0[pt] = 0;
        s_k[pt] = -1;
      }
    }
    __syncthreads();
    if (kC16) {
      for (int i = threadIdx.x; i < kPts16 * 4; i += blockDim.x) {
        const int pt = i >> 2, j = i & 3;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (s_k[pt] >= 0) v = __ldg(reinterpret_cast<const float4*>(dz + (c0 + pt) * CP) + j);
        reinterpret_cast<float4*>(sd)[i] = v;
      }
      for (int i = threadIdx.x; i < kPts16 * kt * 4; i += blockDim.x) {
        const int pt = i / (kt * 4), r = i % (kt * 4), tt = r >> 2, j = r & 3;
        const int kk = s_k[pt] - (kt - 1) + tt;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (s_k[pt] >= 0 && kk >= 0)
          v = __ldg(reinterpret_cast<const float4*>(in + s_row0[pt] + kk * step) + j);
        reinterpret_cast<float4*>(sx)[i] = v;
      }
    } else {
      for (int i = threadIdx.x; i < kPts16 * CP; i += blockDim.x) {
        const int pt = i / CP, co = i % CP;
        sd[i] = (s_k[pt] >= 0 && co < C) ? dz[(c0 + pt) * C + co] : 0.0f;
      }
      for (int i = threadIdx.x; i < kPts16 * kt * CP; i += blockDim.x) {
        const int pt = i / (kt * CP), r = i % (kt * CP), tt = r / CP, ci = r % CP;
        const int kk = s_k[pt] - (kt - 1) + tt;
        sx[i] = (s_k[pt] >= 0 && kk >= 0 && ci < C) ? in[s_row0[pt] + kk * step + ci] : 0.0f;
      }
    }
    __syncthreads();
    if (e < 16 * kt) {
#pragma unroll 4
      for (int pt = 0; pt < kPts16; ++pt) {
        const float4 d = *reinterpret_cast<const float4*>(sd + pt * CP + 4 * cq);
        const float4 x = *reinterpret_cast<const float4*>(sx + (pt * kt + tau) * CP + 4 * iq);
        const float dv[4] = {d.x, d.y, d.z, d.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(dv[a], xv[c], acc[a][c]);
      }
    } else if (e < 16 * kt + CP) {
      const int co = e - 16 * kt;
      for (int pt = 0; pt < kPts16; ++pt) bsum += sd[pt * CP + co];
    }
  }
  if (e < 16 * kt) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int co = 4 * cq + a, ci = 4 * iq + c;
        if (co < C && ci < C) atomicAdd(gw + (co * C + ci) * kt + tau, acc[a][c]);
      }
  } else if (e < 16 * kt + C) {
    atomicAdd(gb + (e - 16 * kt), bsum);
  }
}

struct TWorkspace {
  float* act[kMaxLayers];   // [B][K][hw][C] per layer (post-activation)
  float* I;                 // [B][K][hw]
  float* dI;
  float* g[3];              // [B][K][hw][C] gradient buffers
  size_t bytes;
};

void tlayout(const et_evsnet_weights* net, const et_train_shape* sh, char* base, TWorkspace* ws) {
  const int64_t n = (int64_t)sh->B * sh->K * sh->H * sh->W;
  size_t off = 0;
  auto take = [&](size_t bytes) -> float* {
    float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  for (int l = 0; l < net->n_layers; ++l) ws->act[l] = take(sizeof(float) * n * net->C);
  ws->I = take(sizeof(float) * n);
  ws->dI = take(sizeof(float) * n);
  for (int j = 0; j < 3; ++j) ws->g[j] = take(sizeof(float) * n * net->C);
  ws->bytes = off;
}

// all layers over the whole clip: activations and I
int tforward(const float* logl, const et_train_shape* sh, const et_evsnet_weights* net,
             const TWorkspace& ws, cudaStream_t st) {
  const int C = net->C, L = net->n_layers, kt = net->kt;
  const int64_t hw = (int64_t)sh->H * sh->W, n = (int64_t)sh->B * sh->K * hw;
  const unsigned grid = (unsigned)((n + 255) / 256);
  const unsigned grid2 = (unsigned)(((int64_t)sh->B * ((sh->K + 1) / 2) * hw + 255) / 256);   // step pairs
  const int n0 = layer0_taps(net);
  const float* wp = net->w + twofs(L, C, kt, n0);
  const float* bp = net->b + (int64_t)L * C;
  if (net->ks0 > 0)
    tstem_fwd<<<grid, 256, 0, st>>>(logl, sh->B, sh->K, sh->H, sh->W, C, net->ks0, net->w, net->b,
                                    ws.act[0], wp, bp, L == 1 ? ws.I : nullptr);
  else
    tconv_fwd<<<grid, 256, 0, st>>>(logl, sh->B, sh->K, hw, C, kt, net->w, net->b, ws.act[0], wp, bp,
                                    L == 1 ? ws.I : nullptr);
  ET_CHECK_LAUNCH();
  for (int l = 1; l < L; ++l) {
    // residual form: even layers close a block and add its input
    const float* res = (net->kind == ET_NET_RESIDUAL && l % 2 == 0) ? ws.act[l - 2] : nullptr;
    if (net->dtype == ET_BF16) {
      const int rc = et_train_tct_conv(ws.act[l - 1], sh->B, sh->K, hw, C, kt, net->w + twofs(l, C, kt, n0),
                                       net->b + (int64_t)l * C, res, nullptr, ws.act[l], wp, bp,
                                       l == L - 1 ? ws.I : nullptr, false, st);
      if (rc != ET_OK) return rc;
      continue;
    }
    auto kern = C == CP ? tconv16_fwd<true> : tconv16_fwd<false>;
    kern<<<grid2, 256, 0, st>>>(ws.act[l - 1], sh->B, sh->K, hw, C, kt, net->w + twofs(l, C, kt, n0),
                               net->b + (int64_t)l * C, res, ws.act[l], wp, bp,
                               l == L - 1 ? ws.I : nullptr);
    ET_CHECK_LAUNCH();
  }
  return ET_OK;
}

}  // namespace

bool et_train_is_temporal(const et_evsnet_weights* net) {
  const bool stem_ok = net->ks0 == 0 || (net->ks0 > 0 && net->ks0 <= kMaxStem && net->ks0 % 2 == 1);
  return net->ks == 1 && net->kt >= 1 && net->kt <= kMaxKt && net->C <= kMaxC && stem_ok &&
         (net->kind == ET_NET_STACK || (net->kind == ET_NET_RESIDUAL && net->n_layers % 2 == 1));
}

size_t et_train_temporal_bytes(const et_evsnet_weights* net, const et_train_shape* sh) {
  TWorkspace ws{};
  tlayout(net, sh, nullptr, &ws);
  return ws.bytes;
}

int et_train_temporal_forward(const float* logl, const et_train_shape* sh,
                              const et_evsnet_weights* net, int8_t* spikes, float* S_on,
                              float* S_off, float* V_ckpt, float* I_out, void* workspace,
                              cudaStream_t st) {
  TWorkspace ws{};
  tlayout(net, sh, static_cast<char*>(workspace), &ws);
  int rc = tforward(logl, sh, net, ws, st);
  if (rc != ET_OK) return rc;
  const int64_t hw = (int64_t)sh->H * sh->W, npx = (int64_t)sh->B * hw;
  const int n_ckpt = (sh->K + sh->ckpt_every - 1) / sh->ckpt_every;
  tbilif_fwd<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(
      ws.I, sh->B, sh->K, hw, sh->ckpt_every, n_ckpt, net->beta, net->vth, net->reset, V_ckpt,
      spikes, S_on, S_off, I_out);
  ET_CHECK_LAUNCH();
  return ET_OK;
}

int et_train_temporal_backward(const float* logl, const et_train_shape* sh,
                               const et_evsnet_weights* net, const float* V_ckpt,
                               const float* dS_on, const float* dS_off, float alpha,
                               float* grad_w, float* grad_b, void* workspace, cudaStream_t st) {
  TWorkspace ws{};
  tlayout(net, sh, static_cast<char*>(workspace), &ws);
  int rc = tforward(logl, sh, net, ws, st);
  if (rc != ET_OK) return rc;
  const int C = net->C, L = net->n_layers, kt = net->kt, B = sh->B, K = sh->K;
  const int64_t hw = (int64_t)sh->H * sh->W, npx = (int64_t)B * hw, n = (int64_t)B * K * hw;
  const int n_ckpt = (K + sh->ckpt_every - 1) / sh->ckpt_every;
  int dev = 0, nsm = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  tbilif_bwd<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(
      ws.I, B, K, hw, sh->ckpt_every, n_ckpt, net->beta, net->vth, net->reset, alpha, V_ckpt, dS_on,
      dS_off, ws.dI);
  ET_CHECK_LAUNCH();
  const unsigned grid2 = (unsigned)((npx * ((K + 1) / 2) + 255) / 256);   // step pairs
  const unsigned wgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nsm * 8, (n + kPts - 1) / kPts));
  float* dz = ws.g[0];
  const int n0 = layer0_taps(net);
  tproj_bwd<<<nsm * 4, 256, 0, st>>>(ws.dI, ws.act[L - 1], n, C, net->w + twofs(L, C, kt, n0), dz,
                                     grad_w + twofs(L, C, kt, n0), grad_b + (int64_t)L * C);
  ET_CHECK_LAUNCH();
  const int wthr = twgrad_threads(kt);
  const size_t wsmem = sizeof(float) * kPts16 * CP * (1 + kt);
  auto wkern = C == CP ? tconv16_bwd_weight<true> : tconv16_bwd_weight<false>;
  int wblocks = 0;   // resident weight-gradient blocks per SM: one wave of persistent blocks
  ET_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wblocks, wkern, wthr, wsmem));
  const unsigned wgrid16 = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)nsm * std::max(wblocks, 1), (n + kPts16 - 1) / kPts16));
  auto dkern = C == CP ? tconv16_bwd_data<true> : tconv16_bwd_data<false>;
  auto wgrad = [&](const float* d, int l) -> int {
    if (l == 0 && net->ks0 > 0)
      tstem_bwd_weight<<<wgrid, 256, 0, st>>>(d, logl, B, K, sh->H, sh->W, C, net->ks0, grad_w, grad_b);
    else if (l == 0)
      tconv_bwd_weight<<<wgrid, 256, 0, st>>>(d, logl, B, K, hw, C, kt, grad_w, grad_b);
    else if (net->dtype == ET_BF16)
      return et_train_tct_wgrad(d, ws.act[l - 1], B, K, hw, C, kt, grad_w + twofs(l, C, kt, n0),
                                grad_b + (int64_t)l * C, st);
    else
      wkern<<<wgrid16, wthr, wsmem, st>>>(d, ws.act[l - 1], B, K, hw, C, kt, grad_w + twofs(l, C, kt, n0),
                                          grad_b + (int64_t)l * C);
    return ET_OK;
  };
  // data gradient through layer l: out = (add + conv_l^T(d)) * 1(mask > 0)
  auto dgrad = [&](const float* d, int l, const float* add, const float* mask, float* out) -> int {
    if (net->dtype == ET_BF16)
      return et_train_tct_conv(d, B, K, hw, C, kt, net->w + twofs(l, C, kt, n0), nullptr, add, mask, out,
                               nullptr, nullptr, nullptr, true, st);
    dkern<<<grid2, 256, 0, st>>>(d, B, K, hw, C, kt, net->w + twofs(l, C, kt, n0), add, mask, out);
    return ET_OK;
  };
  if (net->kind == ET_NET_STACK) {
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
      ET_TRY(wgrad(ws.g[cur], l));
      ET_CHECK_LAUNCH();
      if (l > 0) {
        ET_TRY(dgrad(ws.g[cur], l, nullptr, ws.act[l - 1], ws.g[cur ^ 1]));
        ET_CHECK_LAUNCH();
        cur ^= 1;
      }
    }
    return ET_OK;
  }
  // residual: blocks i = M..1 own layers 2i - 1 (inner) and 2i (closing)
  int cz = 0;   // buffer holding dL/dz of the current block's output
  for (int i = (L - 1) / 2; i >= 1; --i) {
    const int la = 2 * i - 1, lc = 2 * i;
    const int cy = (cz + 1) % 3, cn = (cz + 2) % 3;
    ET_TRY(wgrad(ws.g[cz], lc));
    ET_CHECK_LAUNCH();
    // dy = conv_lc^T(dz) masked by a > 0
    ET_TRY(dgrad(ws.g[cz], lc, nullptr, ws.act[la], ws.g[cy]));
    ET_CHECK_LAUNCH();
    ET_TRY(wgrad(ws.g[cy], la));
    ET_CHECK_LAUNCH();
    // dz_prev = (dz + conv_la^T(dy)) masked by h_{i-1} > 0
    ET_TRY(dgrad(ws.g[cy], la, ws.g[cz], ws.act[la - 1], ws.g[cn]));
    ET_CHECK_LAUNCH();
    cz = cn;
  }
  ET_TRY(wgrad(ws.g[cz], 0));
  ET_CHECK_LAUNCH();
  return ET_OK;
}
