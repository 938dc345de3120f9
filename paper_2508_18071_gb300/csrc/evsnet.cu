// EvSNet forward on CUDA cores in FP32 (paper Eq. 1, 5, 6 with the BiLIF of
// Eq. 2-3).  This is the reference-precision path; the tensor-core BF16 path
// lives in evsnet_tc.cu.
//
// One CTA owns a spatial tile for the whole call: it walks the frames in
// order, keeps each owned pixel's membrane potential in a register, keeps the
// causal temporal history of every layer's input in shared memory, and
// recomputes the spatial halo that the ks x ks convolutions need (the halo
// shrinks by ks/2 per layer).  Only X (read), the events and, optionally, the
// projection output / dense spikes touch HBM inside the time loop.
#include <algorithm>
#include "et_internal.cuh"
#include "event_emit.cuh"
#include "evsnet_common.h"

namespace {

struct Params {
  int kind, L, C, kt, ks, r;
  float beta, vth, reset;
  int H, W, F, f0, t0;
  int TX, TY;
  int e_out[kMaxLayers], off_out[kMaxLayers], off_hist[kMaxLayers];
  int woff[kMaxLayers + 1], boff[kMaxLayers + 1];
  int off_x, e_x, off_w, off_b, nw, nb;
};

__device__ __forceinline__ int rw(const Params& P, int e) { return P.TX + 2 * e; }
__device__ __forceinline__ int rsz(const Params& P, int e) { return (P.TX + 2 * e) * (P.TY + 2 * e); }

__global__ void evsnet_f32_kernel(Params P, const float* __restrict__ logl, const float* __restrict__ wg,
                                  const float* __restrict__ bg, float* __restrict__ Vg,
                                  float* __restrict__ histg, float* __restrict__ last_l,
                                  et_event* events, int64_t cap, unsigned long long* n_events,
                                  float* __restrict__ I_out, int8_t* __restrict__ spikes) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ox = blockIdx.x * P.TX, oy = blockIdx.y * P.TY;
  const int64_t npix = (int64_t)P.H * P.W;
  const int hk = P.kt - 1;
  float* sw = sm + P.off_w;
  float* sb = sm + P.off_b;
  for (int i = tid; i < P.nw; i += nthr) sw[i] = wg[i];
  for (int i = tid; i < P.nb; i += nthr) sb[i] = bg[i];
  // temporal history of each layer's input, oldest first
  if (hk > 0) {
    for (int l = 0; l < P.L; ++l) {
      const int cin = l == 0 ? 1 : P.C;
      const int e = l == 0 ? P.e_x : P.e_out[l - 1];
      const int n = rsz(P, e), w = rw(P, e);
      float* h = sm + P.off_hist[l];
      for (int i = tid; i < hk * cin * n; i += nthr) {
        const int pos = i % n, rest = i / n, ci = rest % cin, tau = rest / cin;
        const int gx = ox - e + pos % w, gy = oy - e + pos / w;
        float v = 0.0f;
        if (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H)
          v = histg[(((int64_t)l * hk + tau) * P.C + ci) * npix + (int64_t)gy * P.W + gx];
        h[(tau * cin + ci) * n + pos] = v;
      }
    }
  }
  const int tx = tid % P.TX, ty = tid / P.TX;
  const int px = ox + tx, py = oy + ty;
  const bool own = px < P.W && py < P.H;
  const int64_t q = (int64_t)py * P.W + px;
  float V = own ? Vg[q] : 0.0f;
  int head = 0;
  __syncthreads();
  for (int f = P.f0; f < P.F; ++f) {
    // Eq. 1: X_k = l_k - l_{k-1} over the input region (zero outside the image)
    {
      const int n = rsz(P, P.e_x), w = rw(P, P.e_x);
      float* sx = sm + P.off_x;
      for (int i = tid; i < n; i += nthr) {
        const int gx = ox - P.e_x + i % w, gy = oy - P.e_x + i / w;
        float v = 0.0f;
        if (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H) {
          const int64_t g = (int64_t)gy * P.W + gx;
          const float cur = __ldg(logl + (int64_t)f * npix + g);
          const float prev = f == 0 ? last_l[g] : __ldg(logl + (int64_t)(f - 1) * npix + g);
          v = cur - prev;
        }
        sx[i] = v;
      }
    }
    __syncthreads();
    for (int l = 0; l < P.L; ++l) {
      const int cin = l == 0 ? 1 : P.C;
      const int ei = l == 0 ? P.e_x : P.e_out[l - 1];
      const int eo = P.e_out[l];
      const int ni = rsz(P, ei), wi = rw(P, ei);
      const int no = rsz(P, eo), wo = rw(P, eo);
      const float* in = l == 0 ? sm + P.off_x : sm + P.off_out[l - 1];
      const float* hist = sm + (hk > 0 ? P.off_hist[l] : 0);
      float* out = sm + P.off_out[l];
      const bool resid = P.kind == ET_NET_RESIDUAL && l >= 2 && (l % 2) == 0;
      const float* wl = sw + P.woff[l];
      const int d = ei - eo;   // = r
      for (int i = tid; i < P.C * no; i += nthr) {
        const int co = i / no, pos = i % no;
        const int lx = pos % wo, ly = pos / wo;
        const int gx = ox - eo + lx, gy = oy - eo + ly;
        float v = 0.0f;
        if (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H) {
          float acc = sb[P.boff[l] + co];
          for (int ci = 0; ci < cin; ++ci) {
            for (int tau = 0; tau < P.kt; ++tau) {
              const float* src = tau == hk ? in + ci * ni
                                           : hist + ((((head + tau) % hk) * cin) + ci) * ni;
              const float* wr = wl + ((co * cin + ci) * P.kt + tau) * P.ks * P.ks;
              for (int dy = 0; dy < P.ks; ++dy)
                for (int dx = 0; dx < P.ks; ++dx)
                  acc += wr[dy * P.ks + dx] * src[(ly + d + dy - P.r) * wi + (lx + d + dx - P.r)];
            }
          }
          if (resid) {
            const int er = P.e_out[l - 2], wr2 = rw(P, er);
            acc += sm[P.off_out[l - 2] + co * rsz(P, er) + (ly + er - eo) * wr2 + (lx + er - eo)];
          }
          v = fmaxf(acc, 0.0f);
        }
        out[i] = v;
      }
      __syncthreads();
    }
    // push every layer's input into its history (the oldest slot is replaced)
    if (hk > 0) {
      for (int l = 0; l < P.L; ++l) {
        const int cin = l == 0 ? 1 : P.C;
        const int e = l == 0 ? P.e_x : P.e_out[l - 1];
        const int n = rsz(P, e);
        const float* in = l == 0 ? sm + P.off_x : sm + P.off_out[l - 1];
        float* h = sm + P.off_hist[l] + head * cin * n;
        for (int i = tid; i < cin * n; i += nthr) h[i] = in[i];
      }
      head = (head + 1) % hk;
    }
    // Eq. 6 projection + BiLIF (Eq. 2-3) on the owned pixels
    const int step = f - P.f0;
    uint32_t nev = 0;
    int S = 0;
    if (own) {
      const int eo = P.e_out[P.L - 1];
      const int no = rsz(P, eo);
      const float* hL = sm + P.off_out[P.L - 1];
      float I = sb[P.boff[P.L]];
      for (int c = 0; c < P.C; ++c) I += sw[P.woff[P.L] + c] * hL[c * no + (ty + eo) * rw(P, eo) + tx + eo];
      const float vp = P.beta * V + I;
      S = vp >= P.vth ? 1 : (vp <= -P.vth ? -1 : 0);
      V = vp - P.reset * (float)S;
      nev = (S != 0 && P.t0 + f >= 0) ? 1u : 0u;   // delayed labels below 0: none
      if (I_out) I_out[(int64_t)step * npix + q] = I;
      if (spikes) spikes[(int64_t)step * npix + q] = (int8_t)S;
    }
    emit_events_warp(events, cap, n_events, nev, (uint32_t)px, (uint32_t)py,
                     (uint32_t)(P.t0 + f), S);
    __syncthreads();
  }
  // last_l is read at halo pixels by neighbouring CTAs during their first step,
  // so the caller copies the last frame into it after the kernel.
  if (own) Vg[q] = V;
  if (hk > 0) {
    for (int l = 0; l < P.L; ++l) {
      const int cin = l == 0 ? 1 : P.C;
      const int e = l == 0 ? P.e_x : P.e_out[l - 1];
      const int n = rsz(P, e), w = rw(P, e);
      const float* h = sm + P.off_hist[l];
      for (int i = tid; i < hk * cin * P.TX * P.TY; i += nthr) {
        const int p = i % (P.TX * P.TY), rest = i / (P.TX * P.TY), ci = rest % cin, tau = rest / cin;
        const int lx = p % P.TX, ly = p / P.TX;
        const int gx = ox + lx, gy = oy + ly;
        if (gx >= P.W || gy >= P.H) continue;
        const int pos = (ly + e) * w + lx + e;
        histg[(((int64_t)l * hk + tau) * P.C + ci) * npix + (int64_t)gy * P.W + gx] =
            h[((((head + tau) % hk) * cin) + ci) * n + pos];
      }
    }
  }
}

// first layout that fits in shared memory
bool plan(Params& P, size_t& smem, int max_smem) {
  static const int cand_sp[][2] = {{16, 8}, {16, 4}, {8, 4}, {32, 1}};
  static const int cand_pt[][2] = {{32, 4}, {32, 2}, {32, 1}};
  const auto* cand = P.ks > 1 ? cand_sp : cand_pt;
  const int nc = P.ks > 1 ? 4 : 3;
  for (int c = 0; c < nc; ++c) {
    P.TX = cand[c][0]; P.TY = cand[c][1];
    auto sz = [&](int e) { return (P.TX + 2 * e) * (P.TY + 2 * e); };
    int off = 0;
    P.e_x = P.r * P.L;
    P.off_x = off; off += sz(P.e_x);
    for (int l = 0; l < P.L; ++l) {
      P.e_out[l] = P.r * (P.L - 1 - l);
      P.off_out[l] = off; off += P.C * sz(P.e_out[l]);
    }
    for (int l = 0; l < P.L; ++l) {
      const int cin = l == 0 ? 1 : P.C;
      const int e = l == 0 ? P.e_x : P.e_out[l - 1];
      P.off_hist[l] = off;
      off += (P.kt - 1) * cin * sz(e);
    }
    P.off_w = off; off += P.nw;
    P.off_b = off; off += P.nb;
    smem = sizeof(float) * (size_t)off;
    if ((int)smem <= max_smem) return true;
  }
  return false;
}

}  // namespace

int et_evsnet_forward_f32(const float* logl, int32_t F, const et_evsnet_weights* net,
                          et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                          int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream) {
  Params P{};
  P.kind = net->kind; P.L = net->n_layers; P.C = net->C; P.kt = net->kt; P.ks = net->ks;
  P.r = net->ks / 2;
  P.beta = net->beta; P.vth = net->vth; P.reset = net->reset;
  P.H = st->H; P.W = st->W; P.F = F; P.f0 = st->initialized ? 0 : 1; P.t0 = t0;
  int wo = 0, bo = 0;
  for (int l = 0; l < P.L; ++l) {
    P.woff[l] = wo; P.boff[l] = bo;
    wo += P.C * (l == 0 ? 1 : P.C) * P.kt * P.ks * P.ks; bo += P.C;
  }
  P.woff[P.L] = wo; P.boff[P.L] = bo;
  P.nw = wo + P.C; P.nb = bo + 1;
  int dev = 0, max_smem = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  size_t smem = 0;
  if (!plan(P, smem, max_smem)) return ET_ERR_UNIMPLEMENTED;
  ET_CHECK_CUDA(cudaFuncSetAttribute(evsnet_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  dim3 grid((P.W + P.TX - 1) / P.TX, (P.H + P.TY - 1) / P.TY);
  evsnet_f32_kernel<<<grid, P.TX * P.TY, smem, stream>>>(
      P, logl, net->w, net->b, st->V, st->hist, st->last_l, events, cap,
      reinterpret_cast<unsigned long long*>(n_events), I_out, spikes);
  ET_CHECK_LAUNCH();
  return ET_OK;
}
