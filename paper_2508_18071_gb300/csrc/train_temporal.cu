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

namespace {

constexpr int kMaxC = 16;
constexpr int kMaxKt = 9;
constexpr float kPi = 3.14159265358979323846f;

__host__ __device__ inline int64_t twofs(int l, int C, int kt) {
  return l == 0 ? 0 : (int64_t)C * kt + (int64_t)(l - 1) * C * C * kt;
}

// --------------------------------------------------------------- forward conv
// One thread per (clip, step, pixel).  res (optional) is added before the ReLU;
// the last layer also writes the projection I = bp + wp . out.
template <bool kFromLogl>
__global__ void __launch_bounds__(256)
tconv_fwd(const float* __restrict__ in, const float* __restrict__ logl, int B, int K, int64_t hw,
          int Cin, int C, int kt, const float* __restrict__ w, const float* __restrict__ b,
          const float* __restrict__ res, float* __restrict__ out, const float* __restrict__ wp,
          const float* __restrict__ bp, float* __restrict__ I) {
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
    if (kFromLogl) {
      const float* lf = logl + (int64_t)bc * (K + 1) * hw;
      const float x = lf[(int64_t)(kk + 1) * hw + p] - lf[(int64_t)kk * hw + p];
#pragma unroll
      for (int co = 0; co < kMaxC; ++co)
        if (co < C) acc[co] += sw[co * kt + tau] * x;
    } else {
      const float* src = in + (((int64_t)bc * K + kk) * hw + p) * Cin;
      for (int ci = 0; ci < Cin; ++ci) {
        const float x = src[ci];
#pragma unroll
        for (int co = 0; co < kMaxC; ++co)
          if (co < C) acc[co] += sw[(co * Cin + ci) * kt + tau] * x;
      }
    }
  }
  float* dst = out + idx * C;
  float Iv = bp ? bp[0] : 0.0f;
#pragma unroll
  for (int co = 0; co < kMaxC; ++co) {
    if (co >= C) break;
    const float z = res ? acc[co] + res[idx * C + co] : acc[co];
    const float a = fmaxf(z, 0.0f);
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

// ---------------------------------------------------------- data backward
// out[s][ci] = (add[s][ci] + sum_tau,co w[co][ci][tau] dz[s + kt - 1 - tau][co]) 1(mask[s][ci] > 0)
__global__ void __launch_bounds__(256)
tconv_bwd_data(const float* __restrict__ dz, int B, int K, int64_t hw, int Cin, int C, int kt,
               const float* __restrict__ w, const float* __restrict__ add,
               const float* __restrict__ mask, float* __restrict__ out) {
  __shared__ float sw[kMaxC * kMaxC * kMaxKt];
  for (int i = threadIdx.x; i < C * Cin * kt; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * K * hw) return;
  const int64_t p = idx % hw;
  const int s = (int)((idx / hw) % K), bc = (int)(idx / (hw * K));
  float acc[kMaxC];
#pragma unroll
  for (int ci = 0; ci < kMaxC; ++ci) acc[ci] = 0.0f;
  for (int tau = 0; tau < kt; ++tau) {
    const int k = s + kt - 1 - tau;
    if (k >= K) continue;
    const float* d = dz + (((int64_t)bc * K + k) * hw + p) * C;
    for (int co = 0; co < C; ++co) {
      const float g = d[co];
#pragma unroll
      for (int ci = 0; ci < kMaxC; ++ci)
        if (ci < Cin) acc[ci] += sw[(co * Cin + ci) * kt + tau] * g;
    }
  }
#pragma unroll
  for (int ci = 0; ci < kMaxC; ++ci) {
    if (ci >= Cin) break;
    const int64_t o = idx * Cin + ci;
    const float v = add ? add[o] + acc[ci] : acc[ci];
    out[o] = mask[o] > 0.0f ? v : 0.0f;
  }
}

// -------------------------------------------------------- weight backward
// grad w[co][ci][tau] += sum dz[k][co] in[k - kt + 1 + tau][ci]; grad b[co] += sum dz[k][co].
// Persistent blocks stage 32 pixel-steps at a time in shared memory; each
// thread owns a few (co, ci, tau) entries, one atomic per entry per block.
constexpr int kPts = 32;
template <bool kFromLogl>
__global__ void __launch_bounds__(256)
tconv_bwd_weight(const float* __restrict__ dz, const float* __restrict__ in,
                 const float* __restrict__ logl, int B, int K, int64_t hw, int Cin, int C, int kt,
                 float* __restrict__ gw, float* __restrict__ gb) {
  __shared__ float sd[kPts][kMaxC];
  __shared__ float sx[kPts][kMaxC * kMaxKt + 1];   // [ci][tau], padded
  constexpr int kPer = (kMaxC * kMaxC * kMaxKt + kMaxC + 255) / 256;
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
          if (kFromLogl) {
            const float* lf = logl + (int64_t)bc * (K + 1) * hw;
            v = lf[(int64_t)(kk + 1) * hw + p] - lf[(int64_t)kk * hw + p];
          } else {
            v = in[(((int64_t)bc * K + kk) * hw + p) * Cin + ci];
          }
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
  const float* wp = net->w + twofs(L, C, kt);
  const float* bp = net->b + (int64_t)L * C;
  tconv_fwd<true><<<grid, 256, 0, st>>>(nullptr, logl, sh->B, sh->K, hw, 1, C, kt, net->w, net->b,
                                        nullptr, ws.act[0], wp, bp, L == 1 ? ws.I : nullptr);
  ET_CHECK_LAUNCH();
  for (int l = 1; l < L; ++l) {
    // residual form: even layers close a block and add its input
    const float* res = (net->kind == ET_NET_RESIDUAL && l % 2 == 0) ? ws.act[l - 2] : nullptr;
    tconv_fwd<false><<<grid, 256, 0, st>>>(ws.act[l - 1], nullptr, sh->B, sh->K, hw, C, C, kt,
                                           net->w + twofs(l, C, kt), net->b + (int64_t)l * C, res,
                                           ws.act[l], wp, bp, l == L - 1 ? ws.I : nullptr);
    ET_CHECK_LAUNCH();
  }
  return ET_OK;
}

}  // namespace

bool et_train_is_temporal(const et_evsnet_weights* net) {
  return net->ks == 1 && net->kt >= 1 && net->kt <= kMaxKt && net->C <= kMaxC &&
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
  const unsigned grid = (unsigned)((n + 255) / 256);
  const unsigned wgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nsm * 8, (n + kPts - 1) / kPts));
  float* dz = ws.g[0];
  tproj_bwd<<<nsm * 4, 256, 0, st>>>(ws.dI, ws.act[L - 1], n, C, net->w + twofs(L, C, kt), dz,
                                     grad_w + twofs(L, C, kt), grad_b + (int64_t)L * C);
  ET_CHECK_LAUNCH();
  auto wgrad = [&](const float* d, int l) {
    if (l == 0)
      tconv_bwd_weight<true><<<wgrid, 256, 0, st>>>(d, nullptr, logl, B, K, hw, 1, C, kt, grad_w, grad_b);
    else
      tconv_bwd_weight<false><<<wgrid, 256, 0, st>>>(d, ws.act[l - 1], nullptr, B, K, hw, C, C, kt,
                                                     grad_w + twofs(l, C, kt), grad_b + (int64_t)l * C);
  };
  if (net->kind == ET_NET_STACK) {
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
      wgrad(ws.g[cur], l);
      ET_CHECK_LAUNCH();
      if (l > 0) {
        tconv_bwd_data<<<grid, 256, 0, st>>>(ws.g[cur], B, K, hw, C, C, kt, net->w + twofs(l, C, kt),
                                             nullptr, ws.act[l - 1], ws.g[cur ^ 1]);
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
    wgrad(ws.g[cz], lc);
    ET_CHECK_LAUNCH();
    // dy = conv_lc^T(dz) masked by a > 0
    tconv_bwd_data<<<grid, 256, 0, st>>>(ws.g[cz], B, K, hw, C, C, kt, net->w + twofs(lc, C, kt),
                                         nullptr, ws.act[la], ws.g[cy]);
    ET_CHECK_LAUNCH();
    wgrad(ws.g[cy], la);
    ET_CHECK_LAUNCH();
    // dz_prev = (dz + conv_la^T(dy)) masked by h_{i-1} > 0
    tconv_bwd_data<<<grid, 256, 0, st>>>(ws.g[cy], B, K, hw, C, C, kt, net->w + twofs(la, C, kt),
                                         ws.g[cz], ws.act[la - 1], ws.g[cn]);
    ET_CHECK_LAUNCH();
    cz = cn;
  }
  wgrad(ws.g[cz], 0);
  ET_CHECK_LAUNCH();
  return ET_OK;
}
