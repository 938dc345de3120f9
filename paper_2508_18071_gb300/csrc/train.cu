// Training of the spatial EvSNet (stack of 3x3 convolutions + projection +
// BiLIF; the paper's temporal form is in train_temporal.cu and is dispatched
// from the entry points below) on the GPU: forward with membrane checkpoints, the paper's loss
// (Eq. 7-11) with its gradient, surrogate-gradient BPTT (Eq. 4), and Adam.
// FP32 throughout, or with BF16 weights the C -> C convolutions' forward, data
// and weight gradients on the tensor cores (train_tc.cu).
//
// Layout: B clips of K steps of H x W pixels.  Time is processed in segments of
// `ckpt_every` steps.  The forward keeps only the membrane potential V at the
// start of every segment (and the dense spikes the loss needs); the backward
// walks the segments in reverse, recomputes the segment's activations and
// membrane trajectory from the checkpoint, runs BiLIF backward through time
// inside the segment (carrying dL/dV to the previous segment), then the
// convolution backward for the segment's B x segment images.
//
// Surrogate (Eq. 4 reading): S_on = Theta(V' - Vth), S_off = Theta(-V' - Vth),
// dS_on/dV' = s(V' - Vth), dS_off/dV' = -s(-V' - Vth),
// s(x) = (alpha / 2) / (1 + (pi alpha x / 2)^2); reset V = V' - r (S_on - S_off)
// is differentiated (not detached).
#include <algorithm>
#include <mutex>
#include <cuda.h>
#include "et_internal.cuh"
#include "evsnet_common.h"
#include "train_api.h"

namespace {

constexpr int TS = 16;          // spatial tile (TS x TS pixels per block)
constexpr int kMaxC = 16;       // channels (keeps each block's tiles under 48 KB)
constexpr float kPi = 3.14159265358979323846f;

struct Net {
  int L, C;
  float beta, vth, reset;
  const float* w;   // packed
  const float* b;
};

__host__ __device__ inline int64_t wofs(int l, int C) { return l == 0 ? 0 : 9LL * C + (int64_t)(l - 1) * 9 * C * C; }

// ------------------------------------------------------ forward conv, layer 0
// out[n][co][y][x] = ReLU(b[co] + sum_ky,kx w[co][ky][kx] X[n][y+ky-1][x+kx-1]), X read as
// l_{k+1} - l_k from the clip's log frames: image n is (clip b = n / nseg, step
// k = k0 + n % nseg).  A one-layer network also writes the projection I = bp + wp . a.
__global__ void __launch_bounds__(TS * TS)
conv_fwd(const float* __restrict__ logl, int K, int k0, int nseg, int C, int H, int W,
         const float* __restrict__ w, const float* __restrict__ b, float* __restrict__ out,
         const float* __restrict__ wp, const float* __restrict__ bp, float* __restrict__ I) {
  constexpr int Cin = 1;
  __shared__ float tin[kMaxC][TS + 2][TS + 2];
  __shared__ float tw[kMaxC * kMaxC * 9];
  const int n = blockIdx.z;
  const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
  const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS;
  const int64_t hw = (int64_t)H * W;
  for (int i = threadIdx.x; i < C * Cin * 9; i += TS * TS) tw[i] = w[i];
  for (int i = threadIdx.x; i < Cin * (TS + 2) * (TS + 2); i += TS * TS) {
    const int ci = i / ((TS + 2) * (TS + 2)), r = i % ((TS + 2) * (TS + 2));
    const int yy = y0 - 1 + r / (TS + 2), xx = x0 - 1 + r % (TS + 2);
    float v = 0.0f;
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
      const int64_t g = (int64_t)yy * W + xx;
      const int bc = n / nseg, k = k0 + n % nseg;
      const float* lf = logl + (int64_t)bc * (K + 1) * hw;
      v = lf[(int64_t)(k + 1) * hw + g] - lf[(int64_t)k * hw + g];
    }
    tin[ci][r / (TS + 2)][r % (TS + 2)] = v;
  }
  __syncthreads();
  const int x = x0 + tx, y = y0 + ty;
  if (x >= W || y >= H) return;
  float Iv = bp ? bp[0] : 0.0f;
  for (int co = 0; co < C; ++co) {
    float acc = b[co];
    for (int ci = 0; ci < Cin; ++ci) {
      const float* wr = tw + (co * Cin + ci) * 9;
#pragma unroll
      for (int t = 0; t < 9; ++t) acc += wr[t] * tin[ci][ty + t / 3][tx + t % 3];
    }
    const float a = fmaxf(acc, 0.0f);
    out[((int64_t)n * C + co) * hw + (int64_t)y * W + x] = a;
    if (I) Iv += wp[co] * a;
  }
  if (I) I[(int64_t)n * hw + (int64_t)y * W + x] = Iv;
}

// ------------------------------------------------------------ BiLIF, forward
// One thread per (clip, pixel): walks the segment's steps.
__global__ void bilif_fwd(const float* __restrict__ I, int B, int K, int k0, int nseg, int64_t hw,
                          float beta, float vth, float reset, float* __restrict__ V,
                          float* __restrict__ V_ckpt, int seg, int n_ckpt, int8_t* __restrict__ spikes,
                          float* __restrict__ S_on, float* __restrict__ S_off, float* __restrict__ I_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * hw) return;
  const int bc = (int)(i / hw);
  const int64_t p = i % hw;
  float v = V[i];
  V_ckpt[((int64_t)bc * n_ckpt + seg) * hw + p] = v;
  for (int s = 0; s < nseg; ++s) {
    const float Iv = I[((int64_t)bc * nseg + s) * hw + p];
    const float vp = beta * v + Iv;
    const float on = vp >= vth ? 1.0f : 0.0f, off = -vp >= vth ? 1.0f : 0.0f;
    v = vp - reset * (on - off);
    const int64_t o = ((int64_t)bc * K + k0 + s) * hw + p;
    spikes[o] = (int8_t)(on - off);
    if (S_on) { S_on[o] = on; S_off[o] = off; }
    if (I_out) I_out[o] = Iv;
  }
  V[i] = v;
}

// ----------------------------------------------------------- BiLIF, backward
__device__ __forceinline__ float sg(float x, float alpha) {
  const float u = 0.5f * kPi * alpha * x;
  return 0.5f * alpha / (1.0f + u * u);
}

// Recomputes V' over the segment from its checkpoint, then runs the reverse
// recursion; writes dL/dI per step and carries dL/dV to the previous segment.
__global__ void bilif_bwd(const float* __restrict__ I, int B, int K, int k0, int nseg, int64_t hw,
                          float beta, float vth, float reset, float alpha,
                          const float* __restrict__ V_ckpt, int seg, int n_ckpt,
                          const float* __restrict__ dSon, const float* __restrict__ dSoff,
                          float* __restrict__ gV, float* __restrict__ dI) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * hw) return;
  const int bc = (int)(i / hw);
  const int64_t p = i % hw;
  float vps[kMaxSeg];
  float v = V_ckpt[((int64_t)bc * n_ckpt + seg) * hw + p];
  for (int s = 0; s < nseg; ++s) {
    const float vp = beta * v + I[((int64_t)bc * nseg + s) * hw + p];
    const float on = vp >= vth ? 1.0f : 0.0f, off = -vp >= vth ? 1.0f : 0.0f;
    v = vp - reset * (on - off);
    vps[s] = vp;
  }
  float g = gV[i];
  for (int s = nseg - 1; s >= 0; --s) {
    const float vp = vps[s];
    const float a = sg(vp - vth, alpha), c = sg(-vp - vth, alpha);
    const int64_t o = ((int64_t)bc * K + k0 + s) * hw + p;
    const float gvp = g * (1.0f - reset * (a + c)) + dSon[o] * a - dSoff[o] * c;
    dI[((int64_t)bc * nseg + s) * hw + p] = gvp;
    g = gvp * beta;
  }
  gV[i] = g;
}

// ------------------------------------------------------ projection backward
// dz_{L-1}[c] = dI wp[c] 1(a > 0); grad wp[c] += sum dI a[c]; grad bp += sum dI.
__global__ void __launch_bounds__(256)
proj_bwd(const float* __restrict__ dI, const float* __restrict__ a, int N, int C, int64_t hw,
         const float* __restrict__ wp, float* __restrict__ dz, float* __restrict__ gwp,
         float* __restrict__ gbp) {
  __shared__ float red[kMaxC + 1][8];
  float accw[kMaxC + 1];
  for (int c = 0; c <= C; ++c) accw[c] = 0.0f;
  const int64_t total = (int64_t)N * hw;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i / hw, p = i % hw;
    const float d = dI[i];
    accw[C] += d;
    for (int c = 0; c < C; ++c) {
      const int64_t o = (n * C + c) * hw + p;
      const float av = a[o];
      accw[c] += d * av;
      dz[o] = av > 0.0f ? d * wp[c] : 0.0f;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c <= C; ++c) {
    float v = accw[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[c][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x <= C) {
    float v = 0.0f;
    for (int wv = 0; wv < 8; ++wv) v += red[threadIdx.x][wv];
    if (threadIdx.x < C) atomicAdd(gwp + threadIdx.x, v);
    else atomicAdd(gbp, v);
  }
}

// ------------------------------------------------ conv weight backward, layer 0
// grad w[co][t] += sum_n,y,x dz[n][co][y][x] X[n][y+ky-1][x+kx-1] (X from the log
// frames as in the forward); grad b[co] += sum dz.  Persistent blocks
// accumulate over many tiles in registers, then one atomic per entry per block.
__global__ void __launch_bounds__(TS * TS)
conv_bwd_weight(const float* __restrict__ dz, const float* __restrict__ logl, int K, int k0,
                int nseg, int N, int C, int H, int W, float* __restrict__ gw, float* __restrict__ gb) {
  constexpr int Cin = 1;
  __shared__ float td[kMaxC][TS][TS];
  __shared__ float tin[kMaxC][TS + 2][TS + 2];
  constexpr int kPer = (kMaxC * kMaxC * 9 + kMaxC + TS * TS - 1) / (TS * TS);
  float acc[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) acc[j] = 0.0f;
  const int64_t hw = (int64_t)H * W;
  const int tiles_x = (W + TS - 1) / TS, tiles_y = (H + TS - 1) / TS;
  const int64_t ntiles = (int64_t)N * tiles_x * tiles_y;
  const int nent = C * Cin * 9 + C;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = (int)(tile / (tiles_x * tiles_y));
    const int tt = (int)(tile % (tiles_x * tiles_y));
    const int x0 = (tt % tiles_x) * TS, y0 = (tt / tiles_x) * TS;
    __syncthreads();
    for (int i = threadIdx.x; i < C * TS * TS; i += TS * TS) {
      const int co = i / (TS * TS), r = i % (TS * TS);
      const int yy = y0 + r / TS, xx = x0 + r % TS;
      td[co][r / TS][r % TS] = (yy < H && xx < W) ? dz[((int64_t)n * C + co) * hw + (int64_t)yy * W + xx] : 0.0f;
    }
    for (int i = threadIdx.x; i < Cin * (TS + 2) * (TS + 2); i += TS * TS) {
      const int ci = i / ((TS + 2) * (TS + 2)), r = i % ((TS + 2) * (TS + 2));
      const int yy = y0 - 1 + r / (TS + 2), xx = x0 - 1 + r % (TS + 2);
      float v = 0.0f;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
        const int64_t g = (int64_t)yy * W + xx;
        const int bc = n / nseg, k = k0 + n % nseg;
        const float* lf = logl + (int64_t)bc * (K + 1) * hw;
        v = lf[(int64_t)(k + 1) * hw + g] - lf[(int64_t)k * hw + g];
      }
      tin[ci][r / (TS + 2)][r % (TS + 2)] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int e = threadIdx.x + j * TS * TS;
      if (e >= nent) break;
      float s = 0.0f;
      if (e < C * Cin * 9) {
        const int co = e / (Cin * 9), ci = (e / 9) % Cin, t = e % 9;
        const int ky = t / 3, kx = t % 3;
        for (int py = 0; py < TS; ++py)
          for (int px = 0; px < TS; ++px) s += td[co][py][px] * tin[ci][py + ky][px + kx];
      } else {
        const int co = e - C * Cin * 9;
        for (int py = 0; py < TS; ++py)
          for (int px = 0; px < TS; ++px) s += td[co][py][px];
      }
      acc[j] += s;
    }
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int e = threadIdx.x + j * TS * TS;
    if (e >= nent) break;
    if (e < C * Cin * 9) atomicAdd(gw + e, acc[j]);
    else atomicAdd(gb + (e - C * Cin * 9), acc[j]);
  }
}

// ------------------------------------------- C -> C layers, register-blocked
// The layers with C input channels (all but the first) in a second form: the
// 16 x 16 tile (+ halo) of all channels is staged channel-interleaved in shared
// memory, 16 floats per position, the four 16-byte groups of position m
// permuted by (m >> 1) & 3 so that eight consecutive positions read a group
// from eight different bank quads.  Channels are zero-padded to 16.
constexpr int CP = 16;
constexpr int TP = TS + 2;     // tile with halo

__device__ __forceinline__ int cidx(int m, int g) { return m * CP + 4 * (g ^ ((m >> 1) & 3)); }

// plane-major [c][y][x] tile (rows y0 - h .., columns x0 - h .., tw x th) ->
// interleaved shared memory; zero outside the image and for c >= C
__device__ __forceinline__ void stage(float* __restrict__ s, const float* __restrict__ g, int C,
                                      int H, int W, int x0, int y0, int h, int tw, int th) {
  const int64_t hw = (int64_t)H * W;
  for (int i = threadIdx.x; i < CP * tw * th; i += blockDim.x) {
    const int c = i / (tw * th), r = i % (tw * th);
    const int yy = y0 - h + r / tw, xx = x0 - h + r % tw;
    float v = 0.0f;
    if (c < C && yy >= 0 && yy < H && xx >= 0 && xx < W) v = g[(int64_t)c * hw + (int64_t)yy * W + xx];
    s[cidx(r, c >> 2) + (c & 3)] = v;
  }
}

// acc[k][c] += sum over taps t and input channels of wt[t][ci][4 cg + c] x[m_k + off(t)][ci]
// (off(t) = (t / 3 - 1, t % 3 - 1) on a TP-wide tile); 4 positions x 4 channels
// per thread, 8 vector loads per 64 FMAs
__device__ __forceinline__ void conv_block(const float* __restrict__ sx, const float* __restrict__ wt,
                                           const int (&m)[4], int cg, float (&acc)[4][4]) {
#pragma unroll 1
  for (int t = 0; t < 9; ++t) {
    const int toff = (t / 3 - 1) * TP + (t % 3 - 1);
    const float* w = wt + t * CP * CP + 4 * cg;
    int mk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) mk[k] = m[k] + toff;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const float4 wa = *reinterpret_cast<const float4*>(w + (4 * g + 0) * CP);
      const float4 wb = *reinterpret_cast<const float4*>(w + (4 * g + 1) * CP);
      const float4 wc = *reinterpret_cast<const float4*>(w + (4 * g + 2) * CP);
      const float4 wd = *reinterpret_cast<const float4*>(w + (4 * g + 3) * CP);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 x = *reinterpret_cast<const float4*>(sx + cidx(mk[k], g));
        acc[k][0] = fmaf(wa.x, x.x, acc[k][0]); acc[k][1] = fmaf(wa.y, x.x, acc[k][1]);
        acc[k][2] = fmaf(wa.z, x.x, acc[k][2]); acc[k][3] = fmaf(wa.w, x.x, acc[k][3]);
        acc[k][0] = fmaf(wb.x, x.y, acc[k][0]); acc[k][1] = fmaf(wb.y, x.y, acc[k][1]);
        acc[k][2] = fmaf(wb.z, x.y, acc[k][2]); acc[k][3] = fmaf(wb.w, x.y, acc[k][3]);
        acc[k][0] = fmaf(wc.x, x.z, acc[k][0]); acc[k][1] = fmaf(wc.y, x.z, acc[k][1]);
        acc[k][2] = fmaf(wc.z, x.z, acc[k][2]); acc[k][3] = fmaf(wc.w, x.z, acc[k][3]);
        acc[k][0] = fmaf(wd.x, x.w, acc[k][0]); acc[k][1] = fmaf(wd.y, x.w, acc[k][1]);
        acc[k][2] = fmaf(wd.z, x.w, acc[k][2]); acc[k][3] = fmaf(wd.w, x.w, acc[k][3]);
      }
    }
  }
}

// Thread layout of the 256-thread blocks below: warp w, lane (pg = lane / 4,
// cg = lane % 4) computes channels 4 cg .. 4 cg + 3 at the tile positions
// w * 32 + k * 8 + pg, k = 0..3.
__device__ __forceinline__ void tile_positions(int (&pix)[4], int (&m)[4]) {
  const int warp = threadIdx.x >> 5, pg = (threadIdx.x & 31) >> 2;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    pix[k] = warp * 32 + k * 8 + pg;
    m[k] = (pix[k] / TS + 1) * TP + pix[k] % TS + 1;
  }
}

// forward: out = ReLU(b + conv(in)); the last layer also I = bp + wp . out
__global__ void __launch_bounds__(TS * TS)
conv16_fwd(const float* __restrict__ in, int C, int H, int W, const float* __restrict__ w,
           const float* __restrict__ b, float* __restrict__ out, const float* __restrict__ wp,
           const float* __restrict__ bp, float* __restrict__ I) {
  __shared__ __align__(16) float sx[TP * TP * CP];
  __shared__ __align__(16) float sw[9 * CP * CP];    // [t][ci][co]
  __shared__ __align__(16) float sb[CP], swp[CP];
  const int n = blockIdx.z, x0 = blockIdx.x * TS, y0 = blockIdx.y * TS;
  const int64_t hw = (int64_t)H * W;
  for (int i = threadIdx.x; i < 9 * CP * CP; i += TS * TS) {
    const int co = i % CP, ci = (i / CP) % CP, t = i / (CP * CP);
    sw[i] = (co < C && ci < C) ? w[(co * C + ci) * 9 + t] : 0.0f;
  }
  if (threadIdx.x < CP) {
    sb[threadIdx.x] = threadIdx.x < C ? b[threadIdx.x] : 0.0f;
    swp[threadIdx.x] = (I && threadIdx.x < C) ? wp[threadIdx.x] : 0.0f;
  }
  stage(sx, in + (int64_t)n * C * hw, C, H, W, x0, y0, 1, TP, TP);
  __syncthreads();
  const int cg = threadIdx.x & 3;
  int pix[4], m[4];
  tile_positions(pix, m);
  float acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[k][c] = sb[4 * cg + c];
  conv_block(sx, sw, m, cg, acc);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int x = x0 + pix[k] % TS, y = y0 + pix[k] / TS;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[k][c] = fmaxf(acc[k][c], 0.0f);
      if (x < W && y < H && 4 * cg + c < C)
        out[((int64_t)n * C + 4 * cg + c) * hw + (int64_t)y * W + x] = acc[k][c];
    }
  }
  if (I) {
    // Eq. 6: the 4 channel lanes of a position sum their parts; lane cg writes position cg
    float mine = 0.0f;
    int pmine = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s = swp[4 * cg] * acc[k][0];
      s = fmaf(swp[4 * cg + 1], acc[k][1], s);
      s = fmaf(swp[4 * cg + 2], acc[k][2], s);
      s = fmaf(swp[4 * cg + 3], acc[k][3], s);
      s += __shfl_xor_sync(0xFFFFFFFFu, s, 1);
      s += __shfl_xor_sync(0xFFFFFFFFu, s, 2);
      if (k == cg) { mine = s; pmine = pix[k]; }
    }
    const int x = x0 + pmine % TS, y = y0 + pmine / TS;
    if (x < W && y < H) I[(int64_t)n * hw + (int64_t)y * W + x] = bp[0] + mine;
  }
}

// data backward: dzp[ci] = (sum_co,t w[co][ci][t] dz[co] at the mirrored tap) 1(a_prev > 0),
// i.e. the forward block with weights w'[t][co][ci] = w[co][ci][8 - t]
__global__ void __launch_bounds__(TS * TS)
conv16_bwd_data(const float* __restrict__ dz, int C, int H, int W, const float* __restrict__ w,
                const float* __restrict__ a_prev, float* __restrict__ dzp) {
  __shared__ __align__(16) float sx[TP * TP * CP];
  __shared__ __align__(16) float sw[9 * CP * CP];    // [t][co][ci]
  const int n = blockIdx.z, x0 = blockIdx.x * TS, y0 = blockIdx.y * TS;
  const int64_t hw = (int64_t)H * W;
  for (int i = threadIdx.x; i < 9 * CP * CP; i += TS * TS) {
    const int ci = i % CP, co = (i / CP) % CP, t = i / (CP * CP);
    sw[i] = (co < C && ci < C) ? w[(co * C + ci) * 9 + (8 - t)] : 0.0f;
  }
  stage(sx, dz + (int64_t)n * C * hw, C, H, W, x0, y0, 1, TP, TP);
  __syncthreads();
  const int cg = threadIdx.x & 3;
  int pix[4], m[4];
  tile_positions(pix, m);
  float acc[4][4] = {};
  conv_block(sx, sw, m, cg, acc);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int x = x0 + pix[k] % TS, y = y0 + pix[k] / TS;
    if (x >= W || y >= H) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (4 * cg + c >= C) continue;
      const int64_t o = ((int64_t)n * C + 4 * cg + c) * hw + (int64_t)y * W + x;
      dzp[o] = a_prev[o] > 0.0f ? acc[k][c] : 0.0f;
    }
  }
}

// weight backward: grad w[co][ci][t] += sum_n,p dz[n][co][p] in[n][ci][p + off(t)],
// grad b[co] += sum dz.  Persistent blocks of 160 threads: thread e < 144 owns
// (tap t = e / 16, output quad e % 4, input quad (e / 4) % 4), 16 sums; threads
// 144..159 own the bias sums of one output channel each.  One atomic per entry
// per block at the end.
constexpr int kWThreads = 160;
__global__ void __launch_bounds__(kWThreads)
conv16_bwd_weight(const float* __restrict__ dz, const float* __restrict__ in, int N, int C, int H,
                  int W, float* __restrict__ gw, float* __restrict__ gb) {
  __shared__ __align__(16) float sd[TS * TS * CP];
  __shared__ __align__(16) float sx[TP * TP * CP];
  const int e = threadIdx.x;
  const int t = e / 16, cq = e % 4, iq = (e / 4) % 4;
  const int toff = (t / 3) * TP + t % 3;          // tap offset from the tile position's halo corner
  float acc[4][4] = {};
  float bsum = 0.0f;
  const int64_t hw = (int64_t)H * W;
  const int tiles_x = (W + TS - 1) / TS, tiles_y = (H + TS - 1) / TS;
  const int64_t ntiles = (int64_t)N * tiles_x * tiles_y;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = (int)(tile / (tiles_x * tiles_y));
    const int tt = (int)(tile % (tiles_x * tiles_y));
    const int x0 = (tt % tiles_x) * TS, y0 = (tt / tiles_x) * TS;
    __syncthreads();
    stage(sd, dz + (int64_t)n * C * hw, C, H, W, x0, y0, 0, TS, TS);
    stage(sx, in + (int64_t)n * C * hw, C, H, W, x0, y0, 1, TP, TP);
    __syncthreads();
    if (e < 144) {
#pragma unroll 2
      for (int py = 0; py < TS; ++py) {
#pragma unroll 4
        for (int px = 0; px < TS; ++px) {
          const int p = py * TS + px, q = py * TP + px + toff;
          const float4 d = *reinterpret_cast<const float4*>(sd + cidx(p, cq));
          const float4 x = *reinterpret_cast<const float4*>(sx + cidx(q, iq));
          const float dv[4] = {d.x, d.y, d.z, d.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(dv[a], xv[c], acc[a][c]);
        }
      }
    } else {
      const int co = e - 144;
      for (int p = 0; p < TS * TS; ++p) bsum += sd[cidx(p, co >> 2) + (co & 3)];
    }
  }
  if (e < 144) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int co = 4 * cq + a, ci = 4 * iq + c;
        if (co < C && ci < C) atomicAdd(gw + (co * C + ci) * 9 + t, acc[a][c]);
      }
  } else if (e - 144 < C) {
    atomicAdd(gb + (e - 144), bsum);
  }
}

// ------------------------------------------------------------ loss (Eq. 7-11)
// One thread per (clip, pixel) over the K steps:
//   L = sum over polarities of 1/2 [EMD(E, S) + EMD(E_rev, S_rev)] + lambda |sum|S| - sum|E||,
//   EMD(E, S) = (1/K) sum_i |c_i|, c_i = sum_{j<=i} (S_j - E_j),
// averaged over the B H W pixels.  The reversed EMD uses c'_i = T - c_{i-1}.
// Gradients: dEMD/dS_j = (1/K) sum_{i>=j} sgn c_i, dEMD_rev/dS_j = (1/K) sum_{i<=j} sgn c'_i.
__device__ __forceinline__ float sgnf(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

__global__ void __launch_bounds__(256)
emd_count_loss(const int8_t* __restrict__ spikes, const float* __restrict__ E, int B, int K,
               int64_t hw, float lambda, float* __restrict__ loss, float* __restrict__ dSon,
               float* __restrict__ dSoff) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t npx = (int64_t)B * hw;
  float l_emd = 0.0f, l_cnt = 0.0f;
  if (i < npx) {
    const int bc = (int)(i / hw);
    const int64_t p = i % hw;
    const int64_t base = (int64_t)bc * K * hw + p;
    // pass 1: totals
    float Ton = 0.0f, Toff = 0.0f, nS = 0.0f, nE = 0.0f;
    for (int k = 0; k < K; ++k) {
      const int s = spikes[base + k * hw];
      const float e = E[base + k * hw];
      const float son = s > 0 ? 1.0f : 0.0f, soff = s < 0 ? 1.0f : 0.0f;
      Ton += son - fmaxf(e, 0.0f);
      Toff += soff - fmaxf(-e, 0.0f);
      nS += son + soff;
      nE += fabsf(e);
    }
    // pass 2: losses and the totals of sgn c
    float con = 0.0f, coff = 0.0f, Son = 0.0f, Soff = 0.0f, lon = 0.0f, loff = 0.0f;
    for (int k = 0; k < K; ++k) {
      const int s = spikes[base + k * hw];
      const float e = E[base + k * hw];
      const float rpon = Ton - con, rpoff = Toff - coff;          // c'_k = T - c_{k-1}
      con += (s > 0 ? 1.0f : 0.0f) - fmaxf(e, 0.0f);
      coff += (s < 0 ? 1.0f : 0.0f) - fmaxf(-e, 0.0f);
      lon += fabsf(con) + fabsf(rpon);
      loff += fabsf(coff) + fabsf(rpoff);
      Son += sgnf(con);
      Soff += sgnf(coff);
    }
    const float invK = 1.0f / (float)K, inv = 1.0f / (float)npx;
    l_emd = 0.5f * invK * (lon + loff);
    l_cnt = fabsf(nS - nE);
    const float gc = lambda * sgnf(nS - nE);
    // pass 3: gradients
    con = coff = 0.0f;
    float pre_on = 0.0f, pre_off = 0.0f, rev_on = 0.0f, rev_off = 0.0f;
    for (int k = 0; k < K; ++k) {
      const int s = spikes[base + k * hw];
      const float e = E[base + k * hw];
      const float rpon = Ton - con, rpoff = Toff - coff;
      rev_on += sgnf(rpon);
      rev_off += sgnf(rpoff);
      const float g_on = 0.5f * invK * ((Son - pre_on) + rev_on) + gc;
      const float g_off = 0.5f * invK * ((Soff - pre_off) + rev_off) + gc;
      dSon[base + k * hw] = g_on * inv;
      dSoff[base + k * hw] = g_off * inv;
      con += (s > 0 ? 1.0f : 0.0f) - fmaxf(e, 0.0f);
      coff += (s < 0 ? 1.0f : 0.0f) - fmaxf(-e, 0.0f);
      pre_on += sgnf(con);
      pre_off += sgnf(coff);
    }
    l_emd *= inv;
    l_cnt *= inv;
  }
  // block reduction, one atomic per block and term
  __shared__ float r1[8], r2[8];
  for (int o = 16; o > 0; o >>= 1) {
    l_emd += __shfl_xor_sync(0xFFFFFFFFu, l_emd, o);
    l_cnt += __shfl_xor_sync(0xFFFFFFFFu, l_cnt, o);
  }
  if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = l_emd; r2[threadIdx.x >> 5] = l_cnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.0f, c = 0.0f;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) { a += r1[wv]; c += r2[wv]; }
    atomicAdd(loss + 1, a);
    atomicAdd(loss + 2, c);
    atomicAdd(loss, a + lambda * c);
  }
}

// ------------------------------------------------------------------- Adam
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

struct Workspace {
  float* act[kMaxLayers];   // [nseg B][C][H][W] per layer
  float* I;                 // [nseg B][H][W]
  float* dI;                // [nseg B][H][W]
  float* dz[2];             // [nseg B][C][H][W]
  float* V;                 // [B][H][W] running membrane / carried gradient
  size_t bytes;
};

bool layout(const et_evsnet_weights* net, const et_train_shape* sh, char* base, Workspace* ws) {
  const int64_t hw = (int64_t)sh->H * sh->W;
  const int64_t img = (int64_t)sh->ckpt_every * sh->B;
  size_t off = 0;
  auto take = [&](size_t bytes) -> float* {
    float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  for (int l = 0; l < net->n_layers; ++l) ws->act[l] = take(sizeof(float) * img * net->C * hw);
  ws->I = take(sizeof(float) * img * hw);
  ws->dI = take(sizeof(float) * img * hw);
  ws->dz[0] = take(sizeof(float) * img * net->C * hw);
  ws->dz[1] = take(sizeof(float) * img * net->C * hw);
  ws->V = take(sizeof(float) * sh->B * hw);
  ws->bytes = off;
  return true;
}

int check(const et_evsnet_weights* net, const et_train_shape* sh) {
  if (!net || !sh || !net->w || !net->b) return ET_ERR_ARG;
  if (sh->B < 1 || sh->K < 1 || sh->H < 1 || sh->W < 1 || sh->ckpt_every < 1) return ET_ERR_ARG;
  if (net->n_layers < 1 || net->n_layers > kMaxLayers || net->C < 1) return ET_ERR_UNIMPLEMENTED;
  const bool spatial = net->kind == ET_NET_STACK && net->ks == 3 && net->kt == 1 && net->C <= kMaxC &&
                       net->ks0 == 0;
  if (!spatial && !et_train_is_temporal(net)) return ET_ERR_UNIMPLEMENTED;
  // BF16: the C -> C convolutions of the spatial form, or of the temporal form
  // (kt <= 7), on the tensor cores
  if (net->dtype != ET_F32 &&
      !(net->dtype == ET_BF16 && (spatial || (!spatial && et_train_tct_supported(net)))))
    return ET_ERR_UNIMPLEMENTED;
  if (sh->ckpt_every > kMaxSeg) return ET_ERR_UNIMPLEMENTED;
  return ET_OK;
}

// forward of one segment's convolutions: activations and I for the B x nseg images
int seg_forward(const float* logl, const et_train_shape* sh, const et_evsnet_weights* net,
                const Workspace& ws, int k0, int nseg, cudaStream_t st) {
  const int H = sh->H, W = sh->W, C = net->C, L = net->n_layers;
  const int N = sh->B * nseg;
  dim3 grid((W + TS - 1) / TS, (H + TS - 1) / TS, N);
  const float* wproj = net->w + wofs(L, C);
  const float* bproj = net->b + (int64_t)L * C;
  for (int l = 0; l < L; ++l) {
    const bool last = l == L - 1;
    if (l == 0)
      conv_fwd<<<grid, TS * TS, 0, st>>>(logl, sh->K, k0, nseg, C, H, W, net->w, net->b, ws.act[0],
                                         wproj, bproj, last ? ws.I : nullptr);
    else if (net->dtype == ET_BF16) {
      const int rc = et_train_tc_conv(ws.act[l - 1], N, C, H, W, net->w + wofs(l, C),
                                      net->b + (int64_t)l * C, ws.act[l], wproj, bproj,
                                      last ? ws.I : nullptr, nullptr, false, st);
      if (rc != ET_OK) return rc;
    } else
      conv16_fwd<<<grid, TS * TS, 0, st>>>(ws.act[l - 1], C, H, W, net->w + wofs(l, C),
                                           net->b + (int64_t)l * C, ws.act[l], wproj, bproj,
                                           last ? ws.I : nullptr);
    ET_CHECK_LAUNCH();
  }
  return ET_OK;
}

}  // namespace

extern "C" int et_train_workspace_bytes(const et_evsnet_weights* net, const et_train_shape* sh,
                                        size_t* bytes) {
  const int rc = check(net, sh);
  if (rc != ET_OK) return rc;
  if (!bytes) return ET_ERR_ARG;
  if (et_train_is_temporal(net)) {
    *bytes = et_train_temporal_bytes(net, sh);
    return ET_OK;
  }
  Workspace ws{};
  layout(net, sh, nullptr, &ws);
  *bytes = ws.bytes;
  return ET_OK;
}

extern "C" int et_evsnet_train_forward(const float* logl, const et_train_shape* sh,
                                       const et_evsnet_weights* net, int8_t* spikes, float* S_on,
                                       float* S_off, float* V_ckpt, float* I_out, void* workspace,
                                       size_t ws_bytes, void* stream_) {
  int rc = check(net, sh);
  if (rc != ET_OK) return rc;
  if (!logl || !spikes || !V_ckpt || !workspace || ((S_on == nullptr) != (S_off == nullptr)))
    return ET_ERR_ARG;
  if (et_train_is_temporal(net)) {
    if (ws_bytes < et_train_temporal_bytes(net, sh)) return ET_ERR_ARG;
    return et_train_temporal_forward(logl, sh, net, spikes, S_on, S_off, V_ckpt, I_out, workspace,
                                     (cudaStream_t)stream_);
  }
  Workspace ws{};
  layout(net, sh, nullptr, &ws);
  if (ws_bytes < ws.bytes) return ET_ERR_ARG;
  layout(net, sh, static_cast<char*>(workspace), &ws);
  cudaStream_t st = (cudaStream_t)stream_;
  const int64_t hw = (int64_t)sh->H * sh->W;
  const int n_ckpt = (sh->K + sh->ckpt_every - 1) / sh->ckpt_every;
  ET_CHECK_CUDA(cudaMemsetAsync(ws.V, 0, sizeof(float) * sh->B * hw, st));
  for (int s = 0; s < n_ckpt; ++s) {
    const int k0 = s * sh->ckpt_every, nseg = std::min(sh->ckpt_every, sh->K - k0);
    rc = seg_forward(logl, sh, net, ws, k0, nseg, st);
    if (rc != ET_OK) return rc;
    const int64_t n = (int64_t)sh->B * hw;
    bilif_fwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ws.I, sh->B, sh->K, k0, nseg, hw, net->beta,
                                                           net->vth, net->reset, ws.V, V_ckpt, s, n_ckpt,
                                                           spikes, S_on, S_off, I_out);
    ET_CHECK_LAUNCH();
  }
  return ET_OK;
}

extern "C" int et_emd_count_loss(const int8_t* spikes, const float* E, const et_train_shape* sh,
                                 float lambda, float* loss, float* dS_on, float* dS_off,
                                 void* stream_) {
  if (!sh || !spikes || !E || !loss || !dS_on || !dS_off) return ET_ERR_ARG;
  if (sh->B < 1 || sh->K < 1 || sh->H < 1 || sh->W < 1) return ET_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream_;
  const int64_t hw = (int64_t)sh->H * sh->W, n = (int64_t)sh->B * hw;
  ET_CHECK_CUDA(cudaMemsetAsync(loss, 0, 3 * sizeof(float), st));
  emd_count_loss<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(spikes, E, sh->B, sh->K, hw, lambda,
                                                                loss, dS_on, dS_off);
  ET_CHECK_LAUNCH();
  return ET_OK;
}

extern "C" int et_evsnet_train_backward(const float* logl, const et_train_shape* sh,
                                        const et_evsnet_weights* net, const float* V_ckpt,
                                        const float* dS_on, const float* dS_off, float alpha,
                                        float* grad_w, float* grad_b, void* workspace,
                                        size_t ws_bytes, void* stream_) {
  int rc = check(net, sh);
  if (rc != ET_OK) return rc;
  if (!logl || !V_ckpt || !dS_on || !dS_off || !grad_w || !grad_b || !workspace) return ET_ERR_ARG;
  if (et_train_is_temporal(net)) {
    if (ws_bytes < et_train_temporal_bytes(net, sh)) return ET_ERR_ARG;
    return et_train_temporal_backward(logl, sh, net, V_ckpt, dS_on, dS_off, alpha, grad_w, grad_b,
                                      workspace, (cudaStream_t)stream_);
  }
  Workspace ws{};
  layout(net, sh, nullptr, &ws);
  if (ws_bytes < ws.bytes) return ET_ERR_ARG;
  layout(net, sh, static_cast<char*>(workspace), &ws);
  cudaStream_t st = (cudaStream_t)stream_;
  const int H = sh->H, W = sh->W, C = net->C, L = net->n_layers;
  const int64_t hw = (int64_t)H * W;
  const int n_ckpt = (sh->K + sh->ckpt_every - 1) / sh->ckpt_every;
  int dev = 0, nsm = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int wblocks = 0;   // resident weight-gradient blocks per SM: one wave of persistent blocks
  ET_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wblocks, conv16_bwd_weight, kWThreads, 0));
  wblocks = std::max(wblocks, 1);
  ET_CHECK_CUDA(cudaMemsetAsync(ws.V, 0, sizeof(float) * sh->B * hw, st));   // dL/dV after the last step
  float* gwp = grad_w + wofs(L, C);
  float* gbp = grad_b + (int64_t)L * C;
  for (int s = n_ckpt - 1; s >= 0; --s) {
    const int k0 = s * sh->ckpt_every, nseg = std::min(sh->ckpt_every, sh->K - k0);
    const int N = sh->B * nseg;
    rc = seg_forward(logl, sh, net, ws, k0, nseg, st);
    if (rc != ET_OK) return rc;
    const int64_t n = (int64_t)sh->B * hw;
    bilif_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ws.I, sh->B, sh->K, k0, nseg, hw, net->beta,
                                                           net->vth, net->reset, alpha, V_ckpt, s,
                                                           n_ckpt, dS_on, dS_off, ws.V, ws.dI);
    ET_CHECK_LAUNCH();
    proj_bwd<<<nsm * 4, 256, 0, st>>>(ws.dI, ws.act[L - 1], N, C, hw, net->w + wofs(L, C), ws.dz[0],
                                      gwp, gbp);
    ET_CHECK_LAUNCH();
    dim3 grid((W + TS - 1) / TS, (H + TS - 1) / TS, N);
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
      if (l == 0)
        conv_bwd_weight<<<nsm * 2, TS * TS, 0, st>>>(ws.dz[cur], logl, sh->K, k0, nseg, N, C, H, W,
                                                     grad_w + wofs(0, C), grad_b);
      else if (net->dtype == ET_BF16) {
        rc = et_train_tc_wgrad(ws.dz[cur], ws.act[l - 1], N, C, H, W, grad_w + wofs(l, C),
                               grad_b + (int64_t)l * C, st);
        if (rc != ET_OK) return rc;
      } else
        conv16_bwd_weight<<<nsm * wblocks, kWThreads, 0, st>>>(ws.dz[cur], ws.act[l - 1], N, C, H, W,
                                                               grad_w + wofs(l, C), grad_b + (int64_t)l * C);
      ET_CHECK_LAUNCH();
      if (l > 0) {
        if (net->dtype == ET_BF16) {
          rc = et_train_tc_conv(ws.dz[cur], N, C, H, W, net->w + wofs(l, C), nullptr, ws.dz[cur ^ 1],
                                nullptr, nullptr, nullptr, ws.act[l - 1], true, st);
          if (rc != ET_OK) return rc;
        } else {
          conv16_bwd_data<<<grid, TS * TS, 0, st>>>(ws.dz[cur], C, H, W, net->w + wofs(l, C),
                                                    ws.act[l - 1], ws.dz[cur ^ 1]);
          ET_CHECK_LAUNCH();
        }
        cur ^= 1;
      }
    }
  }
  return ET_OK;
}

extern "C" int et_adam_step(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                            float b1, float b2, float eps, int32_t step, void* stream_) {
  if (!p || !g || !m || !v || n < 0 || step < 1) return ET_ERR_ARG;
  if (n == 0) return ET_OK;
  const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream_>>>(p, g, m, v, n, lr, b1, b2,
                                                                             eps, bc1, bc2);
  ET_CHECK_LAUNCH();
  return ET_OK;
}

// ---------------------------------------------------------------------------
// Backward without a caller workspace.
//
// Some callers cannot hand the library a device workspace: a plugin that lives
// inside a host framework whose caching allocator owns all device memory and
// forbids side allocations, or a loop that must not call cudaMalloc / cudaFree
// because those calls may synchronise the whole device.  For them this entry
// point runs the same backward with its scratch in a fixed array compiled into
// the library.  The array exists once per device that loads the library and is
// kept until the process exits.
namespace {
constexpr size_t kStaticWorkspaceBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kMaxDevices = 64;
std::mutex g_static_ws_mutex;
// Per device: the array's device address and the unique id of the context it
// was looked up in.  A module's __device__ arrays live in one context; after
// cudaDeviceReset (or any teardown of the primary context) the next context
// loads the module again and the array may sit elsewhere, so the address is
// looked up again whenever the current context's id differs.
struct StaticWs {
  void* ptr;
  unsigned long long ctx_id;
};
StaticWs g_static_ws[kMaxDevices] = {};
// Driver calls reached through the runtime's entry-point query (the library
// links only the runtime).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the calling thread's current context; 0 if none is current yet.
int current_context_id(unsigned long long* id) {
  *id = 0;
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return ET_ERR_CUDA;
    g_ctx_get_current = (CtxGetCurrentFn)f1;
    g_ctx_get_id = (CtxGetIdFn)f2;
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return ET_ERR_CUDA;
  if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return ET_ERR_CUDA;
  return ET_OK;
}
}  // namespace

// Device memory; host code must not use this name as an address (on the host it
// only stands for the symbol).  Its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

extern "C" size_t et_train_static_workspace_capacity(void) { return kStaticWorkspaceBytes; }

extern "C" int et_evsnet_train_backward_static(const float* logl, const et_train_shape* sh,
                                               const et_evsnet_weights* net, const float* V_ckpt,
                                               const float* dS_on, const float* dS_off, float alpha,
                                               float* grad_w, float* grad_b, void* stream) {
  int rc = check(net, sh);
  if (rc != ET_OK) return rc;
  // scratch of either form (the temporal one keeps whole-clip activations)
  size_t need = 0;
  if (et_train_is_temporal(net)) {
    need = et_train_temporal_bytes(net, sh);
  } else {
    Workspace ws{};
    layout(net, sh, nullptr, &ws);
    need = ws.bytes;
  }
  if (need > kStaticWorkspaceBytes) return ET_ERR_CAPACITY;   // shape too large for the array
  int dev = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return ET_ERR_ARG;
  void* base = nullptr;
  {
    // first call on this device (with it current), or first call in a new
    // context of it: look up the array's device address
    std::lock_guard<std::mutex> lock(g_static_ws_mutex);
    unsigned long long id = 0;
    rc = current_context_id(&id);
    if (rc != ET_OK) return rc;
    if (!g_static_ws[dev].ptr || id == 0 || g_static_ws[dev].ctx_id != id) {
      void* p = nullptr;
      ET_CHECK_CUDA(cudaGetSymbolAddress(&p, g_static_workspace));
      // the lookup makes the device's primary context current if none was
      rc = current_context_id(&id);
      if (rc != ET_OK) return rc;
      g_static_ws[dev].ptr = p;
      g_static_ws[dev].ctx_id = id;
    }
    base = g_static_ws[dev].ptr;
  }
  // the backward clears the part of the scratch that must start at zero (the
  // carried membrane gradient of the spatial form) and overwrites the rest
  // before reading it
  return et_evsnet_train_backward(logl, sh, net, V_ckpt, dS_on, dS_off, alpha, grad_w, grad_b, base,
                                  kStaticWorkspaceBytes, stream);
}
