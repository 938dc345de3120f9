// EvSNet forward in FP32 for the spatial form of the workloads: a plain stack
// of 3x3 convolutions with ReLU (Eq. 5 with a spatial kernel, kt = 1) of up to
// 16 channels, the point-wise projection (Eq. 6) and BiLIF (Eq. 2-3).
//
// Each CTA owns a 32 x 16 pixel tile for the whole call and walks the frames;
// the membrane potentials of its pixels stay in shared memory.  Per step the
// log frame tile with an L-pixel halo is loaded (X = l_k - l_{k-1}, Eq. 1) and
// the layers run one after the other on shrinking regions of the padded tile
// (layer l is computed L - 1 - l pixels beyond the tile), with zero padding
// outside the image.
//
// Activations are stored channel-interleaved in shared memory, 16 floats per
// position, the four 16-byte channel groups of position m permuted by
// ((m >> 1) & 3) so that eight consecutive positions read one group from eight
// different bank quads.  In layers 1.. a thread computes 4 output channels for
// 4 positions: per tap and group of 4 input channels it loads 4 weight vectors
// (shared by the 8 position lanes of its channel group) and 4 activation
// vectors (shared by the 4 channel lanes of its position) for 64 FMAs.  In the
// last layer the 4 channel lanes of a position sum their parts of the
// projection with two shuffles and each takes one position for BiLIF.
#include "et_internal.cuh"
#include "event_emit.cuh"
#include "evsnet_common.h"

namespace {

constexpr int TW = 32, TH = 16;
constexpr int CP = 16;            // channels as stored (C <= 16, zero padded)

struct SParams {
  int L;
  float beta, vth, reset;
  int H, W, F, f0, t0;
  int Wp, Hp;
  int off_act1, off_b, off_w0, off_wl, off_wp, off_cur, off_prev, off_V;
};

__device__ __forceinline__ int act_idx(int m, int g) { return m * CP + 4 * (g ^ ((m >> 1) & 3)); }

__device__ __forceinline__ float4 relu4(float a, float b, float c, float d) {
  return make_float4(fmaxf(a, 0.0f), fmaxf(b, 0.0f), fmaxf(c, 0.0f), fmaxf(d, 0.0f));
}

template <int kThreads>
__global__ void __launch_bounds__(kThreads)
evsnet_f32s_kernel(SParams P, int C, const float* __restrict__ logl, const float* __restrict__ wg,
                   const float* __restrict__ bg, float* __restrict__ Vg,
                   const float* __restrict__ last_l, et_event* events, int64_t cap,
                   unsigned long long* n_events, float* __restrict__ I_out,
                   int8_t* __restrict__ spikes) {
  extern __shared__ __align__(16) float sm[];
  const int L = P.L, Wp = P.Wp, Hp = P.Hp, tid = threadIdx.x;
  constexpr int kWarps = kThreads / 32;
  const int warp = tid >> 5, lane = tid & 31, pg = lane >> 2, cg = lane & 3;
  float* const act0 = sm;                         // [Hp Wp][CP], permuted groups
  float* const act1 = sm + P.off_act1;
  float* const sb = sm + P.off_b;                 // [L][CP] biases, then the projection bias
  float* const w0 = sm + P.off_w0;                // [9][CP]
  float* const wl = sm + P.off_wl;                // [L-1][9][CP (ci)][CP (co)]
  float* const wp = sm + P.off_wp;                // [CP]
  float* cur = sm + P.off_cur;                    // log frame over the padded tile
  float* prev = sm + P.off_prev;
  float* const Vs = sm + P.off_V;                 // [TH][TW]
  const int tiles_x = (P.W + TW - 1) / TW;
  const int ox = (blockIdx.x % tiles_x) * TW, oy = (blockIdx.x / tiles_x) * TH;
  const int64_t npix = (int64_t)P.H * P.W;

  // packed FP32 weights: layer 0 [C][1][3][3], layers 1.. [C][C][3][3], projection [C]
  for (int i = tid; i < 9 * CP; i += kThreads) {
    const int t = i / CP, co = i % CP;
    w0[i] = co < C ? wg[co * 9 + t] : 0.0f;
  }
  for (int i = tid; i < (L - 1) * 9 * CP * CP; i += kThreads) {
    const int co = i % CP, ci = (i / CP) % CP, t = (i / (CP * CP)) % 9, l = 1 + i / (CP * CP * 9);
    wl[i] = (co < C && ci < C) ? wg[9 * C + (l - 1) * C * C * 9 + (co * C + ci) * 9 + t] : 0.0f;
  }
  for (int i = tid; i < L * CP; i += kThreads) {
    const int l = i / CP, c = i % CP;
    sb[i] = c < C ? bg[l * C + c] : 0.0f;
  }
  for (int i = tid; i < CP; i += kThreads) wp[i] = i < C ? wg[9 * C + (L - 1) * C * C * 9 + i] : 0.0f;
  if (tid == 0) sb[L * CP] = bg[L * C];
  for (int i = tid; i < TW * TH; i += kThreads) {
    const int gx = ox + i % TW, gy = oy + i / TW;
    Vs[i] = (gx < P.W && gy < P.H) ? Vg[(int64_t)gy * P.W + gx] : 0.0f;
  }
  // the frame before the first step: the caller's last frame, or frame 0 when
  // the state is fresh (the first step is then frame 1)
  for (int i = tid; i < Hp * Wp; i += kThreads) {
    const int gx = ox - L + i % Wp, gy = oy - L + i / Wp;
    float v = 0.0f;
    if (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H)
      v = P.f0 == 0 ? last_l[(int64_t)gy * P.W + gx] : __ldg(logl + (int64_t)gy * P.W + gx);
    prev[i] = v;
  }

  for (int f = P.f0; f < P.F; ++f) {
    for (int i = tid; i < Hp * Wp; i += kThreads) {
      const int gx = ox - L + i % Wp, gy = oy - L + i / Wp;
      cur[i] = (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H)
                   ? __ldg(logl + (int64_t)f * npix + (int64_t)gy * P.W + gx) : 0.0f;
    }
    __syncthreads();
    // layer 0 (one input channel) on rows / columns [1, Hp - 1) x [1, Wp - 1):
    // one thread per position, all channels
    {
      const int rw = Wp - 2;
      for (int i = tid; i < (Hp - 2) * rw; i += kThreads) {
        const int py = 1 + i / rw, px = 1 + i % rw, m = py * Wp + px;
        const int gx = ox - L + px, gy = oy - L + py;
        float acc[CP];
#pragma unroll
        for (int c = 0; c < CP; ++c) acc[c] = sb[c];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int q = m + (t / 3 - 1) * Wp + (t % 3 - 1);
          const float x = cur[q] - prev[q];                     // Eq. 1
          const float4* w4 = reinterpret_cast<const float4*>(w0 + t * CP);
#pragma unroll
          for (int j = 0; j < CP / 4; ++j) {
            const float4 w = w4[j];
            acc[4 * j] = fmaf(w.x, x, acc[4 * j]);
            acc[4 * j + 1] = fmaf(w.y, x, acc[4 * j + 1]);
            acc[4 * j + 2] = fmaf(w.z, x, acc[4 * j + 2]);
            acc[4 * j + 3] = fmaf(w.w, x, acc[4 * j + 3]);
          }
        }
        const bool in = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
#pragma unroll
        for (int j = 0; j < CP / 4; ++j)
          *reinterpret_cast<float4*>(act0 + act_idx(m, j)) =
              in ? relu4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3])
                 : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
    }
    __syncthreads();
    // layers 1 .. L-1; the last one only on the tile, into projection + BiLIF
    for (int l = 1; l < L; ++l) {
      const float* ain = (l & 1) ? act0 : act1;
      float* aout = (l & 1) ? act1 : act0;
      const float* wlay = wl + (l - 1) * 9 * CP * CP + 4 * cg;
      const bool last = l == L - 1;
      const int r0 = last ? L : l + 1, r1 = last ? L + TH : Hp - l - 1;
      const int c0 = last ? L : l + 1, c1 = last ? L + TW : Wp - l - 1;
      const int rw = c1 - c0, n = (r1 - r0) * rw;
      const int nchunks = (n + 31) / 32;
      // warp-uniform chunks of 32 positions: position k of lane (pg, cg) is
      // chunk * 32 + k * 8 + pg
      for (int j = warp; j < nchunks; j += kWarps) {
        int m[4];
        bool st[4], in[4];
        int gxk[4], gyk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int idx = j * 32 + k * 8 + pg;
          st[k] = idx < n;
          const int ic = st[k] ? idx : n - 1;
          const int py = r0 + ic / rw, px = c0 + ic % rw;
          m[k] = py * Wp + px;
          gxk[k] = ox - L + px; gyk[k] = oy - L + py;
          in[k] = st[k] && gxk[k] >= 0 && gxk[k] < P.W && gyk[k] >= 0 && gyk[k] < P.H;
        }
        float acc[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[k][c] = sb[l * CP + 4 * cg + c];
#pragma unroll 3
        for (int t = 0; t < 9; ++t) {
          const int toff = (t / 3 - 1) * Wp + (t % 3 - 1);
          const float* wt = wlay + t * CP * CP;
          int mk[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) mk[k] = m[k] + toff;
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const float4 wa = *reinterpret_cast<const float4*>(wt + (4 * g + 0) * CP);
            const float4 wb = *reinterpret_cast<const float4*>(wt + (4 * g + 1) * CP);
            const float4 wc = *reinterpret_cast<const float4*>(wt + (4 * g + 2) * CP);
            const float4 wd = *reinterpret_cast<const float4*>(wt + (4 * g + 3) * CP);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float4 x = *reinterpret_cast<const float4*>(ain + act_idx(mk[k], g));
              acc[k][0] = fmaf(wa.x, x.x, acc[k][0]);
              acc[k][1] = fmaf(wa.y, x.x, acc[k][1]);
              acc[k][2] = fmaf(wa.z, x.x, acc[k][2]);
              acc[k][3] = fmaf(wa.w, x.x, acc[k][3]);
              acc[k][0] = fmaf(wb.x, x.y, acc[k][0]);
              acc[k][1] = fmaf(wb.y, x.y, acc[k][1]);
              acc[k][2] = fmaf(wb.z, x.y, acc[k][2]);
              acc[k][3] = fmaf(wb.w, x.y, acc[k][3]);
              acc[k][0] = fmaf(wc.x, x.z, acc[k][0]);
              acc[k][1] = fmaf(wc.y, x.z, acc[k][1]);
              acc[k][2] = fmaf(wc.z, x.z, acc[k][2]);
              acc[k][3] = fmaf(wc.w, x.z, acc[k][3]);
              acc[k][0] = fmaf(wd.x, x.w, acc[k][0]);
              acc[k][1] = fmaf(wd.y, x.w, acc[k][1]);
              acc[k][2] = fmaf(wd.z, x.w, acc[k][2]);
              acc[k][3] = fmaf(wd.w, x.w, acc[k][3]);
            }
          }
        }
        if (!last) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (st[k])
              *reinterpret_cast<float4*>(aout + act_idx(m[k], cg)) =
                  in[k] ? relu4(acc[k][0], acc[k][1], acc[k][2], acc[k][3])
                        : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else {
          // Eq. 6: each channel lane's part of the projection, summed over the
          // 4 lanes of the position (the same sum in every lane)
          const float4 wpv = *reinterpret_cast<const float4*>(wp + 4 * cg);
          float Ik[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            float s = wpv.x * fmaxf(acc[k][0], 0.0f);
            s = fmaf(wpv.y, fmaxf(acc[k][1], 0.0f), s);
            s = fmaf(wpv.z, fmaxf(acc[k][2], 0.0f), s);
            s = fmaf(wpv.w, fmaxf(acc[k][3], 0.0f), s);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            Ik[k] = sb[L * CP] + s;
          }
          // lane cg takes position k = cg
          float I = Ik[0];
          int mm = m[0], gx = gxk[0], gy = gyk[0];
          bool own = in[0];
#pragma unroll
          for (int k = 1; k < 4; ++k)
            if (cg == k) { I = Ik[k]; mm = m[k]; gx = gxk[k]; gy = gyk[k]; own = in[k]; }
          uint32_t nev = 0;
          int S = 0;
          if (own) {
            const int ti = (mm / Wp - L) * TW + (mm % Wp - L);
            const float vp = P.beta * Vs[ti] + I;               // Eq. 2-3
            S = vp >= P.vth ? 1 : (vp <= -P.vth ? -1 : 0);
            Vs[ti] = vp - P.reset * (float)S;
            nev = (S != 0 && P.t0 + f >= 0) ? 1u : 0u;   // delayed labels below 0: none
            const int64_t o = (int64_t)(f - P.f0) * npix + (int64_t)gy * P.W + gx;
            if (I_out) I_out[o] = I;
            if (spikes) spikes[o] = (int8_t)S;
          }
          emit_events_warp(events, cap, n_events, nev, (uint32_t)(own ? gx : 0),
                           (uint32_t)(own ? gy : 0), (uint32_t)(P.t0 + f), S);
        }
      }
      __syncthreads();
    }
    float* t = cur; cur = prev; prev = t;
  }
  for (int i = tid; i < TW * TH; i += kThreads) {
    const int gx = ox + i % TW, gy = oy + i / TW;
    if (gx < P.W && gy < P.H) Vg[(int64_t)gy * P.W + gx] = Vs[i];
  }
}

}  // namespace

int et_evsnet_forward_f32s(const float* logl, int32_t F, const et_evsnet_weights* net,
                           et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                           int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream) {
  if (net->kind != ET_NET_STACK || net->ks != 3 || net->kt != 1 || net->n_layers < 2 || net->C > CP)
    return ET_ERR_UNIMPLEMENTED;
  SParams P{};
  P.L = net->n_layers;
  P.beta = net->beta; P.vth = net->vth; P.reset = net->reset;
  P.H = st->H; P.W = st->W; P.F = F; P.f0 = st->initialized ? 0 : 1; P.t0 = t0;
  P.Wp = TW + 2 * P.L; P.Hp = TH + 2 * P.L;
  auto al4 = [](int x) { return (x + 3) & ~3; };           // 16-byte alignment in floats
  const int act = P.Hp * P.Wp * CP;
  int off = 2 * act;
  P.off_act1 = act;
  P.off_b = off; off += al4(P.L * CP + 1);
  P.off_w0 = off; off += 9 * CP;
  P.off_wl = off; off += (P.L - 1) * 9 * CP * CP;
  P.off_wp = off; off += CP;
  P.off_cur = off; off += al4(P.Hp * P.Wp);
  P.off_prev = off; off += al4(P.Hp * P.Wp);
  P.off_V = off; off += TW * TH;
  const size_t smem = sizeof(float) * (size_t)off;
  int dev = 0, max_smem = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)max_smem) return ET_ERR_UNIMPLEMENTED;
  int sm_smem = 0;
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  // one CTA per SM (deep networks: the activation buffers take most of the
  // shared memory) gets 16 warps to hide the shared-memory latency; two or
  // more per SM keep 8 warps each (a finer split of the layer regions)
  const int tiles = ((P.W + TW - 1) / TW) * ((P.H + TH - 1) / TH);
  auto run = [&](auto kern, int threads) -> int {
    ET_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<tiles, threads, smem, stream>>>(P, net->C, logl, net->w, net->b, st->V, st->last_l, events, cap,
                                           reinterpret_cast<unsigned long long*>(n_events), I_out, spikes);
    ET_CHECK_LAUNCH();
    return ET_OK;
  };
  if (2 * (smem + 1024) > (size_t)sm_smem) return run(evsnet_f32s_kernel<512>, 512);
  return run(evsnet_f32s_kernel<256>, 256);
}
