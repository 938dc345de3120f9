// BF16 tensor-core convolutions for training the paper's pixel-wise temporal
// EvSNet (Eq. 5: causal convolutions of kernel kt along time between C <= 16
// channels; Sec. 3.3 training): the forward of a C -> C layer, the data
// gradient through it, and its weight gradient, on tcgen05 with BF16 operands
// and FP32 accumulation in TMEM.  Layer 0 (one input channel or a spatial
// stem), the projection, BiLIF and the loss stay FP32 on the CUDA cores
// (train_temporal.cu); activations and gradients stay FP32 in global memory
// ([B][K][H W][C], a pixel-step's channels contiguous), rounded to BF16 where
// they enter an MMA.
//
// Forward and data gradient (tct_conv): a CTA owns 128 consecutive pixels of
// one clip and walks its K steps two at a time -- forward in time for the
// forward, backward in time for the data gradient, which in reversed time is
// the same causal convolution with each tap's weights transposed.  The inputs
// of the last kt + 1 steps sit in a ring of shared-memory slots (128 pixels x
// 16 channels, K-major no-swizzle: two 2 KB planes of 8 channels); slot i of a
// chunk feeds its first step through tap i and its second through tap i - 1,
// so one MMA per slot (M = 128 pixels, K = 16 channels, N = 32: the window
// [W_i ; W_(i-1)] of the layer's taps stored in descending order) covers both
// steps, N = 16 for the first and last slot.  The next chunk's inputs are
// loaded into registers while the MMAs run.
//
// Weight gradient (tct_wgrad): the reduction over pixel-steps is the MMA's K
// dimension, so the operands are staged transposed: for every step, the input
// (channels as rows, pixels along K) into a doubled ring (each step written at
// slots j and j + 8 of 16, so the 8 consecutive slots of steps k - 7 .. k are
// always contiguous) and dL/dz the same way.  D[(tau', ci), co] =
// sum_p in[k - 7 + tau'][p][ci] dz[k][p][co] with M = 128 rows (8 slots x 16
// channels), N = 16, K = 16 pixels per MMA, accumulated in TMEM over the
// CTA's steps and pixels; window slot tau' holds tap tau = tau' - 8 + kt of
// the layer (slots below 8 - kt are not taps).  The bias gradient is summed
// on the CUDA cores while staging.
//
// MMA waits are bounded (et_set_wait_budget); on expiry the kernel writes NaN
// to the outputs it has not finished (the loss then reports it), waits a
// second bounded time for its MMAs in flight and frees its TMEM.
#include "et_internal.cuh"
#include "evsnet_common.h"
#include "tc_ptx.cuh"
#include "train_api.h"
#include <cuda_bf16.h>
#include <algorithm>

namespace {

constexpr int TP = 128;                  // pixels per CTA = MMA M (forward) = TMEM lanes
constexpr int CP = 16;                   // channels, zero-padded
constexpr int kMaxKtTc = 7;              // ring of kt + 1 <= 8 slots
constexpr int kSlot = TP * CP * 2;       // bytes of one ring slot
constexpr int kPlane = TP * 16;          // bytes of 8 channels of 128 rows
constexpr uint32_t kDrainIters = 1u << 22;

// two floats as one 32-bit word of BF16 (round to nearest even), low half first
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// a pixel-step's CP channels (zero beyond C) from FP32 global memory
template <bool kC16>
__device__ __forceinline__ void load16(const float* __restrict__ src, int C, bool ok, float (&x)[CP]) {
  if (!ok) {
#pragma unroll
    for (int c = 0; c < CP; ++c) x[c] = 0.0f;
    return;
  }
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

// row m of a ring slot: channels 0-7 in plane 0, 8-15 in plane 1
__device__ __forceinline__ void store_slot(unsigned char* slot, int m, const float (&v)[CP]) {
  *reinterpret_cast<uint4*>(slot + m * 16) =
      make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
  *reinterpret_cast<uint4*>(slot + kPlane + m * 16) =
      make_uint4(pack2(v[8], v[9]), pack2(v[10], v[11]), pack2(v[12], v[13]), pack2(v[14], v[15]));
}

// ---------------------------------------------------------------- conv
// kBwd = false: out[s] = ReLU(b + sum_tau W_tau in[s - (kt-1) + tau] (+ res[s])),
//               and I[s] = bp + wp . out[s] when I is not null;
// kBwd = true:  out[s] = (add[s] + sum_tau W_tau^T in[s + (kt-1) - tau]) * 1(mask[s] > 0),
//               in = dL/dz of the layer's output, out = dL/dz of its input.
struct ConvArgs {
  const float* in;
  int B, K, C, kt;
  int64_t hw;
  const float* w;       // [co][ci][tau]
  const float* b;       // bias (forward)
  const float* extra;   // res (forward) or add (data gradient), may be null
  const float* mask;    // data gradient: the layer input's activation
  float* out;
  const float* wp;      // forward, last layer: projection
  const float* bp;
  float* I;
  uint32_t wait_iters;
};

template <bool kBwd, bool kC16>
__global__ void __launch_bounds__(TP)
tct_conv(ConvArgs A) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int bail;
  __shared__ float sb[CP], swp[CP];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int C = A.C, K = A.K, kt = A.kt, R = kt + 1;
  const int64_t hw = A.hw;
  const int64_t tiles = (hw + TP - 1) / TP;
  const int bc = (int)(blockIdx.x / tiles);
  const int64_t p = (blockIdx.x % tiles) * TP + tid;
  const bool live = p < hw;
  unsigned char* ring = sm;                                    // [R] slots
  unsigned char* wB = sm + (size_t)R * kSlot;                  // kt blocks x 2 planes
  // B strip: block b holds tap kt - 1 - b; row n, K index k:
  //   forward: n = output channel, k = input channel: w[n][k][tau]
  //   data gradient: n = input channel, k = output channel: w[k][n][tau]
  for (int i = tid; i < kt * CP * CP; i += TP) {
    const int k = i % CP, n = (i / CP) % CP, tau = i / (CP * CP);
    float v = 0.0f;
    if (n < C && k < C) v = kBwd ? A.w[((int64_t)k * C + n) * kt + tau] : A.w[((int64_t)n * C + k) * kt + tau];
    unsigned char* dst = wB + (k >> 3) * (kt * CP * 16) + ((kt - 1 - tau) * CP + n) * 16 + (k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
  }
  for (int i = tid; i < R * kSlot / 16; i += TP) reinterpret_cast<uint4*>(ring)[i] = make_uint4(0, 0, 0, 0);
  if (tid < CP) {
    sb[tid] = (!kBwd && A.b && tid < C) ? A.b[tid] : 0.0f;
    swp[tid] = (!kBwd && A.wp && tid < C) ? A.wp[tid] : 0.0f;
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 32);
  if (tid == 0) { mbar_init(&mma_bar, 1); bail = 0; }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t idesc16 = umma_idesc_bf16(TP, CP), idesc32 = umma_idesc_bf16(TP, 2 * CP);
  const uint64_t a_desc0 = umma_desc(smem_u32(ring), kPlane, 128);
  const uint64_t b_desc0 = umma_desc(smem_u32(wB), kt * CP * 16, 128);
  constexpr uint64_t kBlock = (CP * 16) >> 4;
  const float bpv = (!kBwd && A.bp) ? A.bp[0] : 0.0f;
  // processing order u = 0 .. K-1 is time s = u (forward) or s = K-1-u (data gradient)
  auto step_of = [&](int u) { return kBwd ? K - 1 - u : u; };
  auto row = [&](int s) -> int64_t { return ((int64_t)bc * K + s) * hw + p; };
  const int nch = (K + 1) / 2;
  float nx[2][CP];                       // the next chunk's inputs
  auto load_chunk = [&](int c) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int u = 2 * c + j;
      load16<kC16>(A.in + (live && u < K ? row(step_of(u)) : 0) * C, C, live && u < K, nx[j]);
    }
  };
  load_chunk(0);
  uint32_t phase = 0;
  int c = 0;
  for (; c < nch; ++c) {
    const int u0 = 2 * c, tc = min(2, K - u0);
#pragma unroll
    for (int j = 0; j < 2; ++j)
      if (j < tc) store_slot(ring + (size_t)((u0 + j) % R) * kSlot, tid, nx[j]);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const int p0 = ((u0 - (kt - 1)) % R + R) % R;
      auto a_of = [&](int i) {
        const int pos = p0 + i >= R ? p0 + i - R : p0 + i;
        return a_desc0 + (uint64_t)pos * (kSlot >> 4);
      };
      umma_bf16(tmem, a_of(0), b_desc0 + (uint64_t)(kt - 1) * kBlock, idesc16, 0);
      if (tc > 1) umma_bf16(tmem + CP, a_of(kt), b_desc0, idesc16, 0);
      for (int i = 1; i < kt; ++i) umma_bf16(tmem, a_of(i), b_desc0 + (uint64_t)(kt - 1 - i) * kBlock, idesc32, 1);
      umma_commit(&mma_bar);
    }
    if (c + 1 < nch) load_chunk(c + 1);
    const bool ok = mbar_wait(&mma_bar, phase, A.wait_iters);
    phase ^= 1;
    if (!ok) bail = 1;
    tc_fence_after();
    __syncthreads();
    if (bail) break;
    float acc[2][CP];
    tmem_ld16(tmem + lane_base, acc[0]);
    tmem_ld16(tmem + lane_base + CP, acc[1]);
    for (int j = 0; j < tc; ++j) {
      if (!live) break;
      const int s = step_of(u0 + j);
      float* o = A.out + row(s) * C;
      float v[CP];
      float Iv = bpv;
#pragma unroll
      for (int co = 0; co < CP; ++co) {
        if (!kBwd) {
          float z = acc[j][co] + sb[co];
          if (A.extra && co < C) z += A.extra[row(s) * C + co];
          v[co] = fmaxf(z, 0.0f);
          Iv = fmaf(swp[co], v[co], Iv);
        } else {
          float z = acc[j][co];
          if (co < C) {
            if (A.extra) z += A.extra[row(s) * C + co];
            z = A.mask[row(s) * C + co] > 0.0f ? z : 0.0f;
          }
          v[co] = z;
        }
      }
      if (kC16) {
#pragma unroll
        for (int q = 0; q < CP / 4; ++q)
          reinterpret_cast<float4*>(o)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        for (int co = 0; co < C; ++co) o[co] = v[co];
      }
      if (!kBwd && A.I) A.I[row(s)] = Iv;
    }
    tc_fence_before();
  }
  if (bail) {
    // unfinished steps: NaN, so that the loss shows the failure
    if (live)
      for (int u = 2 * c; u < K; ++u) {
        const int s = step_of(u);
        for (int co = 0; co < C; ++co) A.out[row(s) * C + co] = __int_as_float(0x7fc00000);
        if (!kBwd && A.I) A.I[row(s)] = __int_as_float(0x7fc00000);
      }
    mbar_wait(&mma_bar, phase ^ 1u, kDrainIters);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

// ---------------------------------------------------------------- weight gradient
// grad w[co][ci][tau] += sum_{k,p} dz[k][p][co] in[k - (kt-1) + tau][p][ci],
// grad b[co] += sum_{k,p} dz[k][p][co]; one CTA per 128 pixels of a clip.
constexpr int kWSlots = 16;                       // doubled ring of 8 steps
constexpr int kWRows = kWSlots * CP;              // 256 rows (slot, ci) of 16 B per 8-pixel chunk
constexpr int kWChunk = kWRows * 16;              // bytes per 8-pixel chunk of the input ring
constexpr int kWABytes = (TP / 8) * kWChunk;      // 64 KB
constexpr int kWBBytes = (TP / 8) * CP * 16;      // 4 KB: dz^T, [chunk][co][8 pixels]

__device__ __forceinline__ void st_bf16(unsigned char* p, float v) {
  *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
}

template <bool kC16>
__global__ void __launch_bounds__(TP)
tct_wgrad(const float* __restrict__ dz, const float* __restrict__ in, int B, int K, int64_t hw, int C,
          int kt, float* __restrict__ gw, float* __restrict__ gb, uint32_t wait_iters) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int bail;
  __shared__ float red[TP / 32][CP];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tiles = (hw + TP - 1) / TP;
  const int bc = (int)(blockIdx.x / tiles);
  const int64_t p = (blockIdx.x % tiles) * TP + tid;
  const bool live = p < hw;
  unsigned char* Abuf = sm;
  unsigned char* Bbuf = sm + kWABytes;
  for (int i = tid; i < (kWABytes + kWBBytes) / 16; i += TP) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tmem_alloc(&tmem_slot, 32);
  if (tid == 0) { mbar_init(&mma_bar, 1); bail = 0; }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = umma_idesc_bf16(TP, CP);
  // this thread's column in the transposed buffers: chunk tid / 8, element tid % 8
  unsigned char* acol = Abuf + (tid >> 3) * kWChunk + (tid & 7) * 2;
  unsigned char* bcol = Bbuf + (tid >> 3) * (CP * 16) + (tid & 7) * 2;
  auto row = [&](int s) -> int64_t { return ((int64_t)bc * K + s) * hw + p; };
  float gbp[CP];
#pragma unroll
  for (int c = 0; c < CP; ++c) gbp[c] = 0.0f;
  float nx[CP], nd[CP];
  load16<kC16>(in + (live ? row(0) : 0) * C, C, live, nx);
  load16<kC16>(dz + (live ? row(0) : 0) * C, C, live, nd);
  uint32_t phase = 0;
  for (int k = 0; k < K; ++k) {
    // stage step k: input at slots k % 8 and k % 8 + 8, dz^T
    const int q = k & 7;
#pragma unroll
    for (int c = 0; c < CP; ++c) {
      st_bf16(acol + (q * CP + c) * 16, nx[c]);
      st_bf16(acol + ((q + 8) * CP + c) * 16, nx[c]);
      st_bf16(bcol + c * 16, nd[c]);
      gbp[c] += nd[c];
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      // window: the 8 slots of steps k - 7 .. k, rows base * 16 ..
      const int base = (k + 1) & 7;
      const uint64_t a0 = umma_desc(smem_u32(Abuf) + base * CP * 16, kWChunk, 128);
      const uint64_t b0 = umma_desc(smem_u32(Bbuf), CP * 16, 128);
      for (int j = 0; j < TP / 16; ++j)
        umma_bf16(tmem, a0 + (uint64_t)(2 * j) * (kWChunk >> 4), b0 + (uint64_t)(2 * j) * ((CP * 16) >> 4), idesc,
                  (k > 0 || j > 0) ? 1u : 0u);
      umma_commit(&mma_bar);
    }
    if (k + 1 < K) {
      load16<kC16>(in + (live ? row(k + 1) : 0) * C, C, live, nx);
      load16<kC16>(dz + (live ? row(k + 1) : 0) * C, C, live, nd);
    }
    const bool ok = mbar_wait(&mma_bar, phase, wait_iters);
    phase ^= 1;
    if (!ok) bail = 1;
    tc_fence_after();
    __syncthreads();
    if (bail) break;
  }
  if (bail) {
    mbar_wait(&mma_bar, phase ^ 1u, kDrainIters);
    if (tid == 0) atomicAdd(gw, __int_as_float(0x7fc00000));   // the gradient reports the failure
  } else {
    // lane tid = row (slot offset tau', input channel ci): tap tau = tau' - 8 + kt
    float d[CP];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), d);
    const int tp = tid / CP, ci = tid % CP, tau = tp - 8 + kt;
    if (tau >= 0 && ci < C)
      for (int co = 0; co < C; ++co) atomicAdd(gw + ((int64_t)co * C + ci) * kt + tau, d[co]);
#pragma unroll
    for (int c = 0; c < CP; ++c) {
      float v = live ? gbp[c] : 0.0f;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
      if (lane == 0) red[warp][c] = v;
    }
    __syncthreads();
    if (tid < C) {
      float v = 0.0f;
      for (int wv = 0; wv < TP / 32; ++wv) v += red[wv][tid];
      atomicAdd(gb + tid, v);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

}  // namespace

// ---------------------------------------------------------------- host
bool et_train_tct_supported(const et_evsnet_weights* net) {
  return net->kt >= 1 && net->kt <= kMaxKtTc && net->C >= 1 && net->C <= CP;
}

int et_train_tct_conv(const float* in, int B, int K, int64_t hw, int C, int kt, const float* w, const float* b,
                      const float* extra, const float* mask, float* out, const float* wp, const float* bp,
                      float* I, bool data_grad, cudaStream_t st) {
  if (kt < 1 || kt > kMaxKtTc || C < 1 || C > CP || B < 1 || K < 1 || hw < 1) return ET_ERR_UNIMPLEMENTED;
  ConvArgs A{in, B, K, C, kt, hw, w, b, extra, mask, out, wp, bp, I, et_tc_wait_iters()};
  const size_t smem = (size_t)(kt + 1) * kSlot + (size_t)kt * CP * CP * 2;
  const int64_t blocks = (int64_t)B * ((hw + TP - 1) / TP);
  if (blocks > 0x7FFFFFFF) return ET_ERR_ARG;
  auto launch = [&](auto kern) -> int {
    ET_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)blocks, TP, smem, st>>>(A);
    ET_CHECK_LAUNCH();
    return ET_OK;
  };
  if (data_grad) return C == CP ? launch(tct_conv<true, true>) : launch(tct_conv<true, false>);
  return C == CP ? launch(tct_conv<false, true>) : launch(tct_conv<false, false>);
}

int et_train_tct_wgrad(const float* dz, const float* in, int B, int K, int64_t hw, int C, int kt, float* gw,
                       float* gb, cudaStream_t st) {
  if (kt < 1 || kt > kMaxKtTc || C < 1 || C > CP || B < 1 || K < 1 || hw < 1) return ET_ERR_UNIMPLEMENTED;
  const size_t smem = (size_t)kWABytes + kWBBytes;
  const int64_t blocks = (int64_t)B * ((hw + TP - 1) / TP);
  if (blocks > 0x7FFFFFFF) return ET_ERR_ARG;
  auto kern = C == CP ? tct_wgrad<true> : tct_wgrad<false>;
  ET_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)blocks, TP, smem, st>>>(dz, in, B, K, hw, C, kt, gw, gb, et_tc_wait_iters());
  ET_CHECK_LAUNCH();
  return ET_OK;
}
