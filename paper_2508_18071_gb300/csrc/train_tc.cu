// BF16 tensor-core convolutions for training the spatial EvSNet (the C -> C
// 3x3 layers of Eq. 5): the forward of a layer and the data gradient through
// it, both as implicit GEMMs on tcgen05 with BF16 operands and FP32
// accumulation in TMEM.  Layer 0, the weight gradients, BiLIF and the loss stay
// in FP32 on the CUDA cores (train.cu).
//
// One CTA computes a 32 x 15 output tile of one image.  The input tile with a
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
tc_conv16(const float* __restrict__ in, int C, int H, int W, const float* __restrict__ w,
          const float* __restrict__ b, float* __restrict__ out, const float* __restrict__ wp,
          const float* __restrict__ bp, float* __restrict__ I, const float* __restrict__ a_prev,
          int data_grad, uint32_t wait_iters) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float sb[CP], swp[CP];
  unsigned char* act = sm;                          // [2 planes][kRows][16 B]
  unsigned char* wB = sm + 2 * kPlane;              // [9 taps][2 planes][16 rows][16 B]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = blockIdx.z, x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
  const int64_t hw = (int64_t)H * W;
  const float* src = in + (int64_t)n * C * hw;

  // ---- operands: weights as B[n][k] per tap, the input tile as A rows
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
  for (int r = tid; r < kRows; r += kThreads) {
    const int p = r - kLead;                        // grid position of this row
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
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  if (tid == 0) mbar_init(&mma_bar, 1);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // ---- 9 MMAs per block of 128 grid positions, one thread issues them all
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
  const bool ok = __syncthreads_and(mbar_wait(&mma_bar, 0, wait_iters) ? 1 : 0) != 0;
  tc_fence_after();

  // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) of blocks w / 4 and w / 4 + 2
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
    // still in flight after the bound: wait (again bounded) before freeing TMEM
    mbar_wait(&mma_bar, 0, kDrainIters);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int et_train_tc_conv(const float* in, int N, int C, int H, int W, const float* w, const float* b,
                     float* out, const float* wp, const float* bp, float* I, const float* a_prev,
                     bool data_grad, cudaStream_t stream) {
  if (C < 1 || C > CP) return ET_ERR_UNIMPLEMENTED;
  const size_t smem = 2 * (size_t)kPlane + kWB;
  ET_CHECK_CUDA(cudaFuncSetAttribute(tc_conv16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, N);
  tc_conv16<<<grid, kThreads, smem, stream>>>(in, C, H, W, w, b, out, wp, bp, I, a_prev, data_grad ? 1 : 0,
                                              et_tc_wait_iters());
  ET_CHECK_LAUNCH();
  return ET_OK;
}
