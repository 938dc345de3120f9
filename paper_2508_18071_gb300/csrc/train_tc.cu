// BF16 tensor-core convolutions for training the spatial EvSNet (the C -> C
// 3x3 layers of Eq. 5): the forward of a layer and the data gradient through
// it as implicit GEMMs, and its weight gradient as an im2col GEMM, all on
// tcgen05 with BF16 operands and FP32 accumulation in TMEM.  Layer 0, BiLIF
// and the loss stay in FP32 on the CUDA cores (train.cu).
//
// Persistent CTAs (weights staged, TMEM allocated once) walk 32 x 15 output
// tiles of the images.  The input tile with a
// one-pixel halo (34 x 17 positions) is converted to BF16 into the K-major,
// no-swizzle operand layout: two planes of 16-byte rows, plane 0 holding
// channels 0-7 and plane 1 channels 8-15 of every position of the padded grid
// (width 34).  The A operand of tap (dy, dx) is that buffer with its start
// moved by (dy * 34 + dx) rows, so an MMA of M = 128 consecutive grid
// positions, N = 16 output channels and K = 16 input channels covers one tap;
// 9 MMAs per block of 128 positions, 4 blocks per tile (510 grid positions
// from the first output row on; the two halo columns of each row are
// computed and dropped).  Four warps per block read the accumulators back
// (tcgen05.ld, 32 lanes each) and apply the epilogue:
//   forward:        out = ReLU(acc + b) (FP32, plane-major like the FP32
//                   path), and for the last layer I = bp + wp . out (Eq. 6);
//   data gradient:  dzp = acc * 1(a_prev > 0), weights w[co][ci][8 - t] so
//                   that the same tap offsets serve the transposed conv.
#include "et_internal.cuh"
#include "evsnet_common.h"
#include "tc_ptx.cuh"
#include "train_api.h"
#include <cuda_bf16.h>
#include <algorithm>

namespace {

constexpr int TW = 32, TH = 15;
constexpr int Wp = TW + 2, Hp = TH + 2;            // padded grid 34 x 17
constexpr int CP = 16;
constexpr int kThreads = 256;
constexpr int kLead = 8;                            // zero rows before position 0 (taps reach -35)
constexpr int kMStart = Wp;                         // grid position of the first output row
constexpr int kNB = (TH * Wp + 127) / 128;          // M blocks per tile (4)
constexpr int kRows = (kLead + kMStart + kNB * 128 + Wp + 1 + 7) / 8 * 8;   // operand rows (592)
constexpr int kPlane = kRows * 16;                  // bytes per 8-channel plane
constexpr int kWB = 9 * 2 * CP * 16;                // weight operand bytes
constexpr uint32_t kTmemCols = kNB * CP;            // 64
constexpr uint32_t kDrainIters = 1u << 22;          // bound of the wait before freeing TMEM after a timeout

static_assert(kNB * CP == 64, "TMEM allocation is a power of two >= 32 columns");
static_assert(kLead >= Wp + 1 - kMStart, "the lead rows cover the first block's upper-left tap");

__device__ __forceinline__ int tap_offset(int t) { return (t / 3 - 1) * Wp + (t % 3 - 1); }

__global__ void __launch_bounds__(kThreads)
tc_conv16(const float* __restrict__ in, int N, int C, int H, int W, const float* __restrict__ w,
          const float* __restrict__ b, float* __restrict__ out, const float* __restrict__ wp,
          const float* __restrict__ bp, float* __restrict__ I, const float* __restrict__ a_prev,
          int data_grad, uint32_t wait_iters) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float sb[CP], swp[CP];
  __shared__ int bail;
  unsigned char* act = sm;                          // [2 planes][kRows][16 B]
  unsigned char* wB = sm + 2 * kPlane;              // [9 taps][2 planes][16 rows][16 B]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t hw = (int64_t)H * W;
  const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
  const int64_t ntiles = (int64_t)N * tiles_x * tiles_y;

  // ---- once per CTA: weights as B[n][k] per tap, TMEM, the MMA barrier
  for (int i = tid; i < 9 * 2 * CP * 8; i += kThreads) {
    const int e = i % 8, r = (i / 8) % CP, col = (i / (8 * CP)) % 2, t = i / (8 * CP * 2);
    const int k = 8 * col + e;                      // K index (input channel of the GEMM)
    float v = 0.0f;
    if (r < C && k < C)
      v = data_grad ? w[(k * C + r) * 9 + (8 - t)] : w[(r * C + k) * 9 + t];
    *reinterpret_cast<__nv_bfloat16*>(wB + t * (2 * CP * 16) + col * (CP * 16) + r * 16 + e * 2) =
        __float2bfloat16_rn(v);
  }
  if (tid < CP) {
    sb[tid] = (!data_grad && tid < C) ? b[tid] : 0.0f;
    swp[tid] = (I && tid < C) ? wp[tid] : 0.0f;
  }
  if (tid == 0) bail = 0;
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  if (tid == 0) mbar_init(&mma_bar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0;

  // ---- persistent loop over (image, tile)
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = (int)(tile / (tiles_x * tiles_y));
    const int tt = (int)(tile % (tiles_x * tiles_y));
    const int x0 = (tt % tiles_x) * TW, y0 = (tt / tiles_x) * TH;
    const float* src = in + (int64_t)n * C * hw;
    // the input tile as A rows (zero outside the image and in the padding rows)
    for (int r = tid; r < kRows; r += kThreads) {
      const int p = r - kLead;                      // grid position of this row
      float v[CP];
      const int py = p / Wp, px = p - py * Wp;
      const int gx = x0 - 1 + px, gy = y0 - 1 + py;
      const bool inside = p >= 0 && p < Hp * Wp && gx >= 0 && gx < W && gy >= 0 && gy < H;
#pragma unroll
      for (int c = 0; c < CP; ++c)
        v[c] = (inside && c < C) ? __ldg(src + (int64_t)c * hw + (int64_t)gy * W + gx) : 0.0f;
      __align__(16) __nv_bfloat162 h[CP / 2];
#pragma unroll
      for (int c = 0; c < CP / 2; ++c) h[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
      *reinterpret_cast<uint4*>(act + r * 16) = reinterpret_cast<const uint4*>(h)[0];
      *reinterpret_cast<uint4*>(act + kPlane + r * 16) = reinterpret_cast<const uint4*>(h)[1];
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    // 9 MMAs per block of 128 grid positions, one thread issues them all
    if (tid == 0) {
      const uint32_t abase = smem_u32(act), bbase = smem_u32(wB);
      const uint32_t idesc = umma_idesc_bf16(128, CP);
      for (int blk = 0; blk < kNB; ++blk) {
        const int m0 = kLead + kMStart + blk * 128;
        for (int t = 0; t < 9; ++t) {
          const uint64_t ad = umma_desc(abase + (uint32_t)(m0 + tap_offset(t)) * 16, kPlane, 128);
          const uint64_t bd = umma_desc(bbase + t * (2 * CP * 16), CP * 16, 128);
          umma_bf16(tmem + blk * CP, ad, bd, idesc, t != 0);
        }
      }
      umma_commit(&mma_bar);
    }
    // every thread of the CTA takes the same branch below (tcgen05.ld is warp-wide)
    const bool ok = __syncthreads_and(mbar_wait(&mma_bar, phase, wait_iters) ? 1 : 0) != 0;
    phase ^= 1u;
    tc_fence_after();

    // epilogue: warp w reads TMEM lanes 32 (w % 4) of blocks w / 4 and w / 4 + 2
    const float* prev = data_grad ? a_prev + (int64_t)n * C * hw : nullptr;
    float* dst = out + (int64_t)n * C * hw;
    for (int blk = warp >> 2; blk < kNB; blk += 2) {
      const int m = kMStart + blk * 128 + (warp & 3) * 32 + lane;
      float acc[CP];
      if (ok) tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + blk * CP, acc);
      const int py = m / Wp, px = m - py * Wp;
      const int gx = x0 - 1 + px, gy = y0 - 1 + py;
      const bool valid = py >= 1 && py <= TH && px >= 1 && px <= TW && gx < W && gy < H;
      if (!valid) continue;
      const int64_t g = (int64_t)gy * W + gx;
      if (!ok) {
        // the MMAs did not complete within the bound: the outputs are NaN
        for (int c = 0; c < C; ++c) dst[(int64_t)c * hw + g] = __int_as_float(0x7fc00000);
        if (I && !data_grad) I[(int64_t)n * hw + g] = __int_as_float(0x7fc00000);
        continue;
      }
      if (data_grad) {
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          if (c >= C) break;
          const int64_t o = (int64_t)c * hw + g;
          dst[o] = prev[o] > 0.0f ? acc[c] : 0.0f;
        }
      } else {
        float Iv = I ? bp[0] : 0.0f;
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          if (c >= C) break;
          const float a = fmaxf(acc[c] + sb[c], 0.0f);
          dst[(int64_t)c * hw + g] = a;
          Iv += swp[c] * a;
        }
        if (I) I[(int64_t)n * hw + g] = Iv;
      }
    }
    if (!ok && tid == 0) {
      // still in flight after the bound: wait (again bounded) before the operands
      // and the accumulators are reused; give up on the launch if that fails too
      if (!mbar_wait(&mma_bar, phase ^ 1u, kDrainIters)) bail = 1;
    }
    // the next tile rewrites the operands and the accumulators
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (bail) break;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ------------------------------------------------------------ weight gradient
// grad w[co][ci][t] = sum over images and positions p of dz[co][p] a[ci][p + off(t)]
// as a GEMM D[(t, ci)][co] = sum_p A[(t, ci)][p] B[co][p] with BF16 operands:
// M = 144 rows (t, ci) in two M-blocks of 128 (rows 0-127: taps 0-7; rows
// 128-143: tap 8, the rest of that block discarded), N = 16, K = positions.
// Persistent CTAs walk 16 x 8 position tiles; per tile the FP32 activation
// (with halo) and dz tiles are staged in shared memory by coalesced loads, then
// the A operand is built as their im2col (each 16-byte piece = 8 consecutive x
// of one channel, shifted by the tap) and B from 8-position pieces of dz,
// K-major, in 16 chunks of 8 positions: A [chunk][144 rows][16 B], B [chunk][16
// rows][16 B].
// The accumulators stay in TMEM across all of the CTA's tiles; one atomic per
// entry and CTA at the end.  The bias gradient (sum of dz) is summed in FP32
// alongside.
constexpr int WTW = 16, WTH = 8;                    // position tile
constexpr int kChunks = WTW * WTH / 8;              // 16 K chunks of 8 positions
constexpr int kArows = 9 * CP;                      // 144 A rows (t, ci)
constexpr int kAbytes = ((kChunks - 1) * kArows + 256) * 16;   // the last chunk's second M-block reads 256 rows
constexpr int kBbytes = kChunks * CP * 16;
constexpr uint32_t kWTmemCols = 32;                 // two M-blocks x 16 columns

__global__ void __launch_bounds__(kThreads)
tc_wgrad16(const float* __restrict__ dz, const float* __restrict__ act, int N, int C, int H, int W,
           float* __restrict__ gw, float* __restrict__ gb, uint32_t wait_iters) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float sbias[CP];
  __shared__ int bail;
  unsigned char* A = sm;
  unsigned char* Bop = sm + kAbytes;
  float* sa = reinterpret_cast<float*>(sm + kAbytes + kBbytes);   // [CP][WTH + 2][WTW + 2]
  float* sd = sa + CP * (WTH + 2) * (WTW + 2);                     // [CP][WTH][WTW]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t hw = (int64_t)H * W;
  const int tiles_x = (W + WTW - 1) / WTW, tiles_y = (H + WTH - 1) / WTH;
  const int64_t ntiles = (int64_t)N * tiles_x * tiles_y;
  // rows of the last chunk's second M-block beyond the 144 real ones are read
  // by the MMA: keep them zero
  for (int i = tid; i < (256 - kArows) * 16 / 16; i += kThreads)
    reinterpret_cast<uint4*>(A + ((kChunks - 1) * kArows + kArows) * 16)[i] = make_uint4(0, 0, 0, 0);
  if (tid < CP) sbias[tid] = 0.0f;
  if (tid == 0) bail = 0;
  if (warp == 0) tmem_alloc(&tmem_slot, kWTmemCols);
  if (tid == 0) mbar_init(&mma_bar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = umma_idesc_bf16(128, CP);
  uint32_t phase = 0;
  bool first = true;
  // the FP32 tiles of the next tile are loaded into registers while the
  // current one is converted and multiplied: activations with a one-pixel halo
  // [ci][10][18] and dz [co][8][16], element i = tid + j * kThreads
  constexpr int kSa = CP * (WTH + 2) * (WTW + 2), kSd = CP * WTH * WTW;
  constexpr int kRa = (kSa + kThreads - 1) / kThreads, kRd = kSd / kThreads;
  static_assert(kSd % kThreads == 0, "dz tile elements per thread");
  float ra[kRa], rd[kRd];
  auto fetch = [&](int64_t tile) {
    const int n = (int)(tile / (tiles_x * tiles_y));
    const int tt = (int)(tile % (tiles_x * tiles_y));
    const int x0 = (tt % tiles_x) * WTW, y0 = (tt / tiles_x) * WTH;
    const float* a_n = act + (int64_t)n * C * hw;
    const float* d_n = dz + (int64_t)n * C * hw;
#pragma unroll
    for (int j = 0; j < kRa; ++j) {
      const int i = tid + j * kThreads;
      const int c = i / ((WTH + 2) * (WTW + 2)), r = i % ((WTH + 2) * (WTW + 2));
      const int y = y0 - 1 + r / (WTW + 2), x = x0 - 1 + r % (WTW + 2);
      ra[j] = (i < kSa && c < C && y >= 0 && y < H && x >= 0 && x < W)
                  ? __ldg(a_n + (int64_t)c * hw + (int64_t)y * W + x) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < kRd; ++j) {
      const int i = tid + j * kThreads;
      const int c = i / (WTH * WTW), r = i % (WTH * WTW);
      const int y = y0 + r / WTW, x = x0 + r % WTW;
      rd[j] = (c < C && y < H && x < W) ? __ldg(d_n + (int64_t)c * hw + (int64_t)y * W + x) : 0.0f;
    }
  };
  if (blockIdx.x < ntiles) fetch(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < ntiles && !bail; tile += gridDim.x) {
#pragma unroll
    for (int j = 0; j < kRa; ++j)
      if (tid + j * kThreads < kSa) sa[tid + j * kThreads] = ra[j];
#pragma unroll
    for (int j = 0; j < kRd; ++j) sd[tid + j * kThreads] = rd[j];
    __syncthreads();
    if (tile + gridDim.x < ntiles) fetch(tile + gridDim.x);
    // A pieces: (chunk kc, row m = t * 16 + ci) = 8 consecutive x of channel ci,
    // shifted by tap t
    for (int i = tid; i < kChunks * kArows; i += kThreads) {
      const int kc = i / kArows, m = i % kArows, t = m / CP, ci = m % CP;
      const float* src = sa + (ci * (WTH + 2) + kc / 2 + t / 3) * (WTW + 2) + 8 * (kc % 2) + t % 3;
      __align__(16) __nv_bfloat162 h[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(src[2 * e], src[2 * e + 1]);
      *reinterpret_cast<uint4*>(A + (kc * kArows + m) * 16) = *reinterpret_cast<const uint4*>(h);
    }
    // B pieces: (chunk kc, row co); 128 threads also sum one dz row each for
    // the bias gradient
    for (int i = tid; i < kChunks * CP; i += kThreads) {
      const int kc = i / CP, co = i % CP;
      const float4* src = reinterpret_cast<const float4*>(sd + (co * WTH + kc / 2) * WTW + 8 * (kc % 2));
      const float4 u = src[0], v = src[1];
      __align__(16) __nv_bfloat162 h[4] = {__floats2bfloat162_rn(u.x, u.y), __floats2bfloat162_rn(u.z, u.w),
                                           __floats2bfloat162_rn(v.x, v.y), __floats2bfloat162_rn(v.z, v.w)};
      *reinterpret_cast<uint4*>(Bop + (kc * CP + co) * 16) = *reinterpret_cast<const uint4*>(h);
    }
    if (tid < CP * WTH) {
      const float* row = sd + tid * WTW;
      float sum = 0.0f;
      for (int x = 0; x < WTW; ++x) sum += row[x];
      atomicAdd(&sbias[tid / WTH], sum);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t abase = smem_u32(A), bbase = smem_u32(Bop);
      for (int j = 0; j < kChunks / 2; ++j) {
        const uint64_t bd = umma_desc(bbase + (2 * j) * CP * 16, CP * 16, 128);
        for (int mb = 0; mb < 2; ++mb) {
          const uint64_t ad = umma_desc(abase + ((2 * j) * kArows + mb * 128) * 16, kArows * 16, 128);
          umma_bf16(tmem + mb * CP, ad, bd, idesc, (first && j == 0) ? 0u : 1u);
        }
      }
      umma_commit(&mma_bar);
    }
    first = false;
    // the operands are rewritten for the next tile only after these MMAs completed
    const bool ok = __syncthreads_and(mbar_wait(&mma_bar, phase, wait_iters) ? 1 : 0) != 0;
    phase ^= 1u;
    tc_fence_after();
    if (!ok) {
      if (tid == 0) bail = 1;
      __syncthreads();
    }
  }
  __syncthreads();
  if (bail) {
    // a wait ran out: the gradients of this launch are NaN; wait (bounded)
    // for the MMAs still in flight before freeing TMEM
    if (tid == 0) {
      mbar_wait(&mma_bar, phase ^ 1u, kDrainIters);
      for (int i = 0; i < C * C * 9; ++i) atomicAdd(gw + i, __int_as_float(0x7fc00000));
    }
  } else if (!first) {
    // D rows (t, ci) on TMEM lanes: M-block 0 = taps 0-7 (warps 0-3), M-block 1
    // lanes 0-15 = tap 8 (warp 4)
    if (warp < 5) {
      const int mb = warp == 4 ? 1 : 0;
      float d[CP];
      tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + mb * CP, d);
      const int row = mb * 128 + (warp & 3) * 32 + lane;
      if (row < kArows) {
        const int t = row / CP, ci = row % CP;
        if (ci < C)
          for (int co = 0; co < C; ++co) atomicAdd(gw + (co * C + ci) * 9 + t, d[co]);
      }
    }
    if (tid < C) atomicAdd(gb + tid, sbias[tid]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kWTmemCols);
}

}  // namespace

// CTAs of 256 threads a persistent tensor-core kernel can keep on one SM:
// bounded by threads, registers, shared memory (with the static part and the
// per-CTA reservation) and TMEM columns (512 per SM)
static int resident_ctas(const void* kern, size_t dyn_smem, uint32_t tmem_cols, int* per_sm, int* nsm) {
  int dev = 0, sm_smem = 0, sm_regs = 0;
  cudaFuncAttributes fa{};
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  ET_CHECK_CUDA(cudaFuncGetAttributes(&fa, kern));
  ET_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int n = 2048 / kThreads;
  n = std::min(n, sm_regs / std::max(1, fa.numRegs * kThreads));
  n = std::min(n, sm_smem / (int)(dyn_smem + fa.sharedSizeBytes + 1024));
  n = std::min(n, (int)(512 / tmem_cols));
  *per_sm = std::max(n, 1);
  return ET_OK;
}

int et_train_tc_conv(const float* in, int N, int C, int H, int W, const float* w, const float* b,
                     float* out, const float* wp, const float* bp, float* I, const float* a_prev,
                     bool data_grad, cudaStream_t stream) {
  if (C < 1 || C > CP) return ET_ERR_UNIMPLEMENTED;
  const size_t smem = 2 * (size_t)kPlane + kWB;
  ET_CHECK_CUDA(cudaFuncSetAttribute(tc_conv16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, nsm = 0;
  const int rc = resident_ctas(reinterpret_cast<const void*>(tc_conv16), smem, kTmemCols, &per_sm, &nsm);
  if (rc != ET_OK) return rc;
  const int64_t tiles = (int64_t)N * ((W + TW - 1) / TW) * ((H + TH - 1) / TH);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)nsm * per_sm));
  tc_conv16<<<grid, kThreads, smem, stream>>>(in, N, C, H, W, w, b, out, wp, bp, I, a_prev, data_grad ? 1 : 0,
                                              et_tc_wait_iters());
  ET_CHECK_LAUNCH();
  return ET_OK;
}

int et_train_tc_wgrad(const float* dz, const float* act, int N, int C, int H, int W, float* gw,
                      float* gb, cudaStream_t stream) {
  if (C < 1 || C > CP) return ET_ERR_UNIMPLEMENTED;
  const size_t smem = (size_t)kAbytes + kBbytes + sizeof(float) * CP * ((WTH + 2) * (WTW + 2) + WTH * WTW);
  ET_CHECK_CUDA(cudaFuncSetAttribute(tc_wgrad16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, nsm = 0;
  const int rc = resident_ctas(reinterpret_cast<const void*>(tc_wgrad16), smem, kWTmemCols, &per_sm, &nsm);
  if (rc != ET_OK) return rc;
  const int64_t tiles = (int64_t)N * ((W + WTW - 1) / WTW) * ((H + WTH - 1) / WTH);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)nsm * std::max(per_sm, 1)));
  tc_wgrad16<<<grid, kThreads, smem, stream>>>(dz, act, N, C, H, W, gw, gb, et_tc_wait_iters());
  ET_CHECK_LAUNCH();
  return ET_OK;
}
