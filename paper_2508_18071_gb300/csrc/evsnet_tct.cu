// EvSNet forward on the tcgen05 tensor cores for the pixel-wise temporal form:
// the paper's network (Sec. 4.1, Eq. 5: convolutions of kernel kt along time,
// plain stack or residual blocks; Eq. 6 projection; BiLIF of Eq. 2-3), with or
// without a one-step spatial stem as layer 0.  BF16 or FP8 (E4M3) operands
// (the weights of layers 1.. and their inputs), FP32 accumulation in TMEM;
// layer 0, the residual sums, the projection and BiLIF stay FP32.
//
// A CTA owns a tile of 128 consecutive pixels for the whole call: one TMEM
// lane per pixel and three groups of 128 threads, one thread per pixel each
// (warps w, w + 4, w + 8 share TMEM lane quarter w); group g runs the
// epilogues of every third tensor-core layer counting down from the last, so
// that consecutive layers' epilogues run at once in different warps; group 1
// also runs layer 0 (FP8: groups 1 and 2, 8 channels each), group 0 the
// projection and BiLIF.  A thirteenth warp's
// one thread issues every MMA and TMA copy, so that issuing never holds up
// the epilogues.  The input history of every layer >= 1 (its
// last kt inputs) lives in shared memory as a ring of kt + kT - 1 slots, each
// slot one step of 128 pixels x 16 channels in the K-major, no-swizzle operand
// layout (two 2 KB planes of 8 channels, 16-byte rows), so the A operand of tap
// tau is simply the slot of step s - (kt - 1) + tau.  The kT = 2 steps of a
// chunk read kt + 1 slots; slot i feeds output step j through tap i - j, so
// one MMA per slot with N = 32 computes both steps' shares at once: its B
// operand is the window [W_i ; W_(i-1)] of the layer's taps stored in
// descending order as one strip (rows W_(kt-1), ..., W_0), and only the first
// and last slot, which feed one step each, take N = 16 MMAs.  A layer's two
// steps are kt + 1 MMAs (M = 128, K = 16), accumulated in two groups of 16
// TMEM columns.
//
// The layers run as a wavefront over chunks: in round tau, layer 0 (CUDA
// cores) computes chunk tau and tensor-core layer l chunk tau - l + 1.  One
// barrier per round makes the rings' new slots visible to the tensor core;
// the issuing thread then issues every layer's MMAs, last layer first, with
// one commit per layer, and the pixel warps run each layer's epilogue as soon
// as its commit arrives (bias, ReLU, residual add, BF16 rounding into the next
// layer's ring; after the last layer the projection and BiLIF).  Layer l's
// epilogue overwrites slots that layer l + 1's MMAs of the same round read;
// those were issued earlier, and a commit covers every earlier MMA.  The FP32
// input of each residual block waits for its closing layer in TMEM (two
// chunks per block).  The caller's FP32 history state ([layer][kt-1][C][H][W])
// is read into the rings at the start and written back at the end; values
// written by this kernel are BF16-rounded, so a later call of the BF16 path
// reads them back exactly.
//
// The 3 x 3 stem's input: when the image width is a multiple of 128 (a tile is
// then one row segment), each chunk's log frames f - 1 .. f + 1, rows y - 1 ..
// y + 1 and columns x0 - 4 .. x0 + 131 arrive as one TMA box
// (cp.async.bulk.tensor.3d; the tensor map covers the caller's log frames,
// zero-filled outside the image, which is the stem's zero padding), issued two
// chunks ahead by the issuing thread into one of two buffers and waited on
// through that buffer's mbarrier; the first chunk of a call, whose previous
// frame may be the state's, is loaded by the threads.  Layer 0 of chunk
// tau + 1 is computed in registers while round tau's MMAs run and stored into
// layer 1's ring after the round's last epilogue.
//
// FP8: a layer's MMAs sum taps of several steps, so its input scale is one
// power of two for the whole call (the caller's calibrated scales), and the
// weights carry one per output channel.  A ring slot is then 16 bytes per
// pixel, and one K = 32 MMA covers two consecutive slots (their rows are the
// two 16-byte columns of the operand); with N = 32 = (step, output channel)
// its B block holds [[W_i, W_(i-1)], [W_(i+1), W_i]] for the slot pair
// (i, i + 1), so a layer's two steps take (kt + 2) / 2 MMAs.  The ring is
// kept twice over (every store also goes R positions on) so that the window's
// slot pairs never wrap.  The two steps of a pair sum their taps in different
// orders in both precisions: results depend on a step's place in its pair
// (FP32 rounding), so calls with even step counts reproduce one call exactly.
//
// MMA waits are bounded; on expiry the kernel sets bit 62 of the event count,
// leaves the membrane and history state untouched, waits (bounded) for its
// MMAs in flight and frees its TMEM.
#include "et_internal.cuh"
#include "event_emit.cuh"
#include "evsnet_common.h"
#include "tc_ptx.cuh"
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cstring>

namespace {

constexpr int TP = 128;                 // pixels per tile = MMA M = TMEM lanes
constexpr int CP = 16;                  // channels (C <= 16, zero-padded)
constexpr int kT = 2;                   // steps per MMA round trip (the MMA schedule assumes 2)
static_assert(kT == 2, "one N = 32 MMA per middle slot covers exactly two steps");
constexpr int kMaxKt = 7;
constexpr int kMaxStem = 7;
constexpr int kSlot = TP * CP * 2;      // bytes of one ring slot (BF16)
constexpr int kSlot8 = TP * CP;         // bytes of one ring slot (FP8: 16 channels = one 16-byte row)
constexpr int kPair8 = 2 * 2 * CP * 16; // bytes of one FP8 B block: K = 2 slots x N = 2 steps x 16 channels
constexpr float kE4M3Max = 448.0f;
constexpr int kPlane = TP * 16;         // bytes of 8 channels of 128 rows
constexpr int kHalf = CP / 2;            // channels of one operand plane
constexpr int kGroups = 3;              // worker groups, one thread per pixel each
constexpr int kStemGroup = 1;           // the group that also runs layer 0
constexpr int kWorkers = kGroups * TP;
constexpr int kThreads = kWorkers + 32; // and one warp that issues the MMAs and the TMA copies
constexpr int kIssuer = kWorkers;       // its issuing thread
// TMEM: kT x 16 accumulator columns per tensor-core layer, then the FP32
// block inputs of up to three residual blocks for three chunks
constexpr int kHbCol = (kMaxLayers - 1) * kT * 16;
constexpr uint32_t kTmemCols = 512;
static_assert(kHbCol + 3 * 3 * kT * 16 <= (int)kTmemCols, "TMEM columns");
constexpr unsigned long long kTimeoutBit = 1ull << 62;
constexpr uint32_t kDrainIters = 1u << 22;   // bound of the waits for work in flight after a bail

struct TctParams {
  int H, W, F, f0, t0;
  int L, C, kt, ks0, kind;
  float beta, vth, reset;
  int R;                                // ring slots per layer: kt + kT - 1
  int woff[kMaxLayers + 1];             // packed weight offsets per layer (+ projection)
  int off_wB, off_f32, off_xbuf;        // shared-memory byte offsets
  int tma;                              // the stem's input tiles come by TMA
  uint32_t wait_iters;
  const float* scales;                  // FP8: input scale of tensor-core layer l at [l - 1]
  unsigned int* amax;                   // calibration: largest input of layer l + 1 at [l] (float bits), or NULL
};

// the TMA box of the 3 x 3 stem: columns x0 - 4 .. x0 + 131, 3 rows, 3 frames
constexpr int kBoxW = TP + 8;
constexpr int kBoxFloats = kBoxW * 3 * 3;
constexpr uint32_t kBoxBytes = kBoxFloats * 4;
// the two box buffers start 128-byte aligned (a TMA destination's alignment)
constexpr int kBoxStride = (kBoxFloats + 31) / 32 * 32;

__device__ __forceinline__ int ring_pos(int s, int R) { return ((s % R) + R) % R; }

// two floats as one 32-bit word of BF16 (round to nearest even), low half first
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// smallest power of two >= x / 448 (1 for x == 0): the E4M3 scale of values
// whose absolute maximum is x
__host__ __device__ __forceinline__ float e4m3_scale(float x) {
  if (!(x > 0.0f)) return 1.0f;
  int e;
  const float m = frexpf(x / kE4M3Max, &e);   // x / 448 = m 2^e, m in [0.5, 1)
  return ldexpf(1.0f, m == 0.5f ? e - 1 : e);
}

// four floats as four E4M3 bytes (saturating), the first in the low byte
__device__ __forceinline__ uint32_t pack_e4m3(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

__device__ __forceinline__ float2 unpack_e4m3x2(uint32_t two) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)two, __NV_E4M3);
  return __half22float2(*reinterpret_cast<const __half2*>(&h));
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t w) {
  __nv_bfloat162 h;
  *reinterpret_cast<uint32_t*>(&h) = w;
  return __bfloat1622float2(h);
}

// all 16 channels of one pixel, BF16-rounded, as row m of a ring slot (plane
// 0: channels 0-7, plane 1: channels 8-15), and back
__device__ __forceinline__ void store_row(unsigned char* slot, int m, const float* v) {
  *reinterpret_cast<uint4*>(slot + m * 16) =
      make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
  *reinterpret_cast<uint4*>(slot + kPlane + m * 16) =
      make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
}

__device__ __forceinline__ void load_half(const unsigned char* slot, int hc, int m, float (&v)[kHalf]) {
  const uint4 a = *reinterpret_cast<const uint4*>(slot + hc * kPlane + m * 16);
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = unpack_bf16(w[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

__device__ __forceinline__ void load_row(const unsigned char* slot, int m, float (&v)[CP]) {
  float lo[kHalf], hi[kHalf];
  load_half(slot, 0, m, lo);
  load_half(slot, 1, m, hi);
#pragma unroll
  for (int c = 0; c < kHalf; ++c) {
    v[c] = lo[c];
    v[kHalf + c] = hi[c];
  }
}

// FP8: the 16 channels of one pixel divided by the layer's input scale (inv =
// its reciprocal), as row m of a ring slot and of the slot's copy R positions
// on, if it has one (the ring is kept twice so that every window of slots is
// contiguous)
__device__ __forceinline__ void store_row8(unsigned char* slot, unsigned char* copy, int m, const float* v,
                                           float inv) {
  uint4 r;
  r.x = pack_e4m3(v[0] * inv, v[1] * inv, v[2] * inv, v[3] * inv);
  r.y = pack_e4m3(v[4] * inv, v[5] * inv, v[6] * inv, v[7] * inv);
  r.z = pack_e4m3(v[8] * inv, v[9] * inv, v[10] * inv, v[11] * inv);
  r.w = pack_e4m3(v[12] * inv, v[13] * inv, v[14] * inv, v[15] * inv);
  *reinterpret_cast<uint4*>(slot + m * 16) = r;
  if (copy) *reinterpret_cast<uint4*>(copy + m * 16) = r;
}

// and back, times the scale
__device__ __forceinline__ void load_row8(const unsigned char* slot, int m, float sc, float (&v)[CP]) {
  const uint4 a = *reinterpret_cast<const uint4*>(slot + m * 16);
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f0 = unpack_e4m3x2(w[i] & 0xFFFFu), f1 = unpack_e4m3x2(w[i] >> 16);
    v[4 * i] = f0.x * sc;
    v[4 * i + 1] = f0.y * sc;
    v[4 * i + 2] = f1.x * sc;
    v[4 * i + 3] = f1.y * sc;
  }
}

template <bool kF8, bool kCal>
__global__ void __launch_bounds__(kThreads, 1)
evsnet_tct_kernel(const __grid_constant__ CUtensorMap tmap, TctParams P, const float* __restrict__ logl,
                  const float* __restrict__ wg, const float* __restrict__ bg, float* __restrict__ Vg,
                  float* __restrict__ hist, const float* __restrict__ last_l, et_event* events, int64_t cap,
                  unsigned long long* n_events, float* __restrict__ I_out,
                  int8_t* __restrict__ spikes) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t lbar[kMaxLayers];  // commit of tensor-core layer l's MMAs in a round
  __shared__ uint64_t tma_bar[2];       // the two TMA box buffers
  __shared__ uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int bail;
  const int L = P.L, C = P.C, kt = P.kt, R = P.R, hk = kt - 1, ks0 = P.ks0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p = tid & (TP - 1);         // pixel of the tile = TMEM lane
  const int grp = tid >> 7;             // worker group (4 = the issuing warp)
  // group g runs the epilogues of the tensor-core layers l with
  // (L - 1 - l) % 3 == g (the last layer, with the projection and BiLIF, in
  // group 0), so that consecutive layers' epilogues run in different warps
  auto owns = [&](int l) { return (L - 1 - l) % kGroups == grp; };
  const int64_t npix = (int64_t)P.H * P.W;
  const int64_t q = (int64_t)blockIdx.x * TP + p;
  const bool worker = tid < kWorkers;
  const bool stem_grp = grp == kStemGroup;
  // layer 0: the stem group alone (BF16), or split by channel halves between
  // groups 1 and 2 (FP8: its shorter MMA stream leaves layer 0 on the round's
  // critical path); the X ring of a temporal layer 0 is then written by both,
  // each with the value it reads back itself
  constexpr int kSC = kF8 ? CP / 2 : CP;          // layer-0 channels per participating thread
  const bool stem_part = kF8 ? (grp == 1 || grp == 2) : stem_grp;
  const int c_lo = (kF8 && grp == 2) ? CP / 2 : 0;   // its first channel
  const bool live = worker && q < npix;
  const int px = live ? (int)(q % P.W) : 0, py = live ? (int)(q / P.W) : 0;
  constexpr int kSB = kF8 ? kSlot8 : kSlot;                    // bytes per ring slot
  // slots per layer.  FP8: positions R .. RS - 1 repeat 0 .. RS - R - 1; a
  // window starts below R and its slot pairs end at kt + 1 (kt odd) or kt + 2
  // (kt even) slots, so the copy of position R - 1 is needed for even kt only
  const int RS = kF8 ? ((kt & 1) ? 2 * R - 1 : 2 * R) : R;
  unsigned char* rings = sm;                                   // [L-1][RS] slots
  unsigned char* wB = sm + P.off_wB;                           // BF16: [L-1][kt] 16 x 16; FP8: [L-1][pairs] kPair8
  float* f32 = reinterpret_cast<float*>(sm + P.off_f32);
  float* bs = f32;                                             // [L][CP] biases
  float* wp = bs + L * CP;                                     // [CP] projection
  float* bp = wp + CP;                                         // [1] (+ pad)
  float* w0 = bp + 4;                                          // [taps][CP] layer 0
  const int taps0 = ks0 > 0 ? ks0 * ks0 : kt;
  float* xh = w0 + taps0 * CP;                                 // [R][TP] layer-0 X ring (temporal layer 0)
  float* dq = xh + (ks0 == 0 ? R * TP : 0);                    // FP8: [L][CP] weight scale, then x input scale
  float* isc = dq + L * CP;                                    // FP8: [kMaxLayers] 1 / input scale of layer l
  float* scl = isc + kMaxLayers;                               // FP8: [kMaxLayers] input scale of layer l
  const int npairs = (kt + 2) / 2;                             // FP8: MMAs per layer (slot pairs)
  float* xbuf = reinterpret_cast<float*>(sm + P.off_xbuf);     // [2][3 frames][3 rows][kBoxW] (TMA)
  auto slot_of = [&](int l, int pos) { return rings + ((size_t)(l - 1) * RS + pos) * kSB; };
  // a pixel's 16 channels into ring position pos of layer l (both copies in FP8)
  auto put_row = [&](int l, int pos, const float* v) {
    if constexpr (kF8) store_row8(slot_of(l, pos), pos + R < RS ? slot_of(l, pos + R) : nullptr, p, v, isc[l]);
    else store_row(slot_of(l, pos), p, v);
  };
  // history element (layer l, oldest-first slot j, channel c) of this pixel in the state
  auto hidx = [&](int l, int j, int c) -> int64_t { return (((int64_t)l * hk + j) * C + c) * npix + q; };

  // ---- set-up: weights, biases, history rings
  for (int i = tid; i < L * CP; i += kThreads) {
    const int l = i / CP, c = i % CP;
    bs[i] = c < C ? bg[l * C + c] : 0.0f;
  }
  for (int i = tid; i < CP; i += kThreads) wp[i] = i < C ? wg[P.woff[L] + i] : 0.0f;
  if (tid == 0) bp[0] = bg[L * C];
  for (int i = tid; i < taps0 * CP; i += kThreads) {
    const int t = i / CP, c = i % CP;
    w0[i] = c < C ? wg[c * taps0 + t] : 0.0f;                 // layer 0: [C][1][taps]
  }
  if constexpr (!kF8) {
    // B operands: one strip per layer l >= 1 of kt blocks of 16 rows, block b
    // holding tap kt - 1 - b (rows n = output channel, K = input channel in two
    // planes of 8, each plane kt x 16 rows of 16 bytes)
    // (one 16-byte row of 8 input channels per iteration: its loads in flight together)
    for (int r = tid; r < (L - 1) * 2 * kt * CP; r += kThreads) {
      const int n = r % CP, b = (r / CP) % kt, pl = (r / (CP * kt)) % 2, l = 1 + r / (2 * CP * kt);
      const int tau = kt - 1 - b;
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = pl * 8 + e;
        v[e] = (n < C && k < C) ? __ldg(wg + P.woff[l] + (n * C + k) * kt + tau) : 0.0f;
      }
      *reinterpret_cast<uint4*>(wB + (size_t)(l - 1) * kt * (CP * CP * 2) + pl * (kt * CP * 16) + (b * CP + n) * 16) =
          make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
  } else {
    // the FP32 weights of layers 1.. staged in the ring area (free until the
    // ring is zeroed below), read once with coalesced loads
    float* wst = reinterpret_cast<float*>(rings);
    const int wbase = P.woff[1], nw = P.woff[L] - P.woff[1];
#pragma unroll 4
    for (int i = tid; i < nw; i += kThreads) wst[i] = __ldg(wg + wbase + i);
    for (int l = tid; l < kMaxLayers; l += kThreads) {
      const float sc = (l >= 1 && l < L) ? P.scales[l - 1] : 1.0f;
      scl[l] = sc;
      isc[l] = 1.0f / sc;
    }
    __syncthreads();
    // weight scales per layer and output channel (their maximum to <= 448)
    for (int i = tid; i < L * CP; i += kThreads) {
      const int l = i / CP, co = i % CP;
      float mx = 0.0f;
      if (l >= 1 && co < C)
        for (int k = 0; k < C * kt; ++k) mx = fmaxf(mx, fabsf(wst[P.woff[l] - wbase + co * C * kt + k]));
      dq[i] = e4m3_scale(mx);
    }
    __syncthreads();
    // B operands: per layer l >= 1 one block per pair of slots (2 pi, 2 pi + 1)
    // of the window: K = the two slots' 16 channels (two 16-byte columns of 32
    // rows), N = 32 = (step j, output channel); slot i feeds step j through tap
    // i - j (zero outside 0 .. kt - 1)
    // (one 16-byte row of 16 input channels per iteration; the weight scales
    // are powers of two, so multiplying by their reciprocals is exact)
    for (int row = tid; row < (L - 1) * npairs * 2 * 2 * CP; row += kThreads) {
      const int n = row % (2 * CP), r = (row / (2 * CP)) % 2, pi = (row / (4 * CP)) % npairs;
      const int l = 1 + row / (4 * CP * npairs);
      const int j = n / CP, co = n % CP, tau = 2 * pi + r - j;
      const bool on = tau >= 0 && tau < kt && co < C;
      const float inv = 1.0f / dq[l * CP + co];
      float v[CP];
#pragma unroll
      for (int ci = 0; ci < CP; ++ci)
        v[ci] = (on && ci < C) ? wst[P.woff[l] - wbase + (co * C + ci) * kt + tau] * inv : 0.0f;
      *reinterpret_cast<uint4*>(wB + ((size_t)(l - 1) * npairs + pi) * kPair8 + r * (2 * CP * 16) + n * 16) =
          make_uint4(pack_e4m3(v[0], v[1], v[2], v[3]), pack_e4m3(v[4], v[5], v[6], v[7]),
                     pack_e4m3(v[8], v[9], v[10], v[11]), pack_e4m3(v[12], v[13], v[14], v[15]));
    }
    __syncthreads();
    // dequantisation factor of layer l's accumulators: weight scale x input
    // scale; the rings zeroed: a slot pair may take one slot the call never
    // writes (with zero weights), whose bytes must not be E4M3 NaNs
    for (int i = tid; i < L * CP; i += kThreads) dq[i] *= scl[i / CP];
    for (int i = tid; i < (L - 1) * RS * kSlot8 / 16; i += kThreads)
      reinterpret_cast<uint4*>(rings)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
  }
  // ring slots of steps -(kt-1) .. -1 from the state (oldest first): group g
  // fills the slots j with j % 3 == g (both channel halves), a layer's loads
  // issued before its stores
  for (int l = 1; l < L; ++l) {
    constexpr int kJ = (kMaxKt - 1 + kGroups - 1) / kGroups;
    float v[kJ][CP];
#pragma unroll
    for (int jj = 0; jj < kJ; ++jj) {
      const int j = jj * kGroups + grp;
#pragma unroll
      for (int c = 0; c < CP; ++c) v[jj][c] = (j < hk && live && c < C) ? hist[hidx(l, j, c)] : 0.0f;
    }
#pragma unroll
    for (int jj = 0; jj < kJ; ++jj) {
      const int j = jj * kGroups + grp;
      if (worker && j < hk) put_row(l, ring_pos(j - hk, R), v[jj]);
    }
  }
  if (ks0 == 0 && stem_grp)
    for (int j = 0; j < hk; ++j) xh[ring_pos(j - hk, R) * TP + p] = live ? hist[hidx(0, j, 0)] : 0.0f;
  float V = (live && grp == 0) ? Vg[q] : 0.0f;
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  if (tid == 0) {
    for (int l = 0; l < kMaxLayers; ++l) mbar_init(&lbar[l], 1);
    mbar_init(&tma_bar[0], 1);
    mbar_init(&tma_bar[1], 1);
    mbar_init(&drain_bar, 1);
    bail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t idesc16 = umma_idesc_bf16(TP, CP), idesc32 = umma_idesc_bf16(TP, 2 * CP);
  const uint32_t idesc8 = umma_idesc_e4m3(TP, 2 * CP);
  // A: K-adjacent 16-byte columns are the two channel planes of a BF16 slot,
  // or two consecutive FP8 slots; B: the two planes of a BF16 tap strip, or the
  // two slot columns of an FP8 pair block
  const uint64_t a_desc0 = umma_desc(smem_u32(rings), kF8 ? kSlot8 : kPlane, 128);
  const uint64_t b_desc0 = umma_desc(smem_u32(wB), kF8 ? 2 * CP * 16 : kt * CP * 16, 128);
  // TMEM columns: layer l's accumulators (both steps, 16 channels each) at
  // 32 (l - 1); the FP32 block inputs of the residual form (block b, chunk c)
  // at kHbCol + 32 (3 b + c % 3): a block input written for chunk c + 2 never
  // meets the one read for chunk c
  auto acc_col = [&](int l) { return tmem + lane_base + (uint32_t)((l - 1) * kT * CP); };
  auto hb_col = [&](int b, int c) { return tmem + lane_base + (uint32_t)(kHbCol + (3 * b + c % 3) * kT * CP); };
  uint32_t lphase = 0;                  // bit l: parity of the next completion of lbar[l] this thread waits for
  const bool residual = P.kind == ET_NET_RESIDUAL;

  const int S = P.F - P.f0;             // steps of this call
  const int nch = (S + kT - 1) / kT;    // chunks of kT steps
  // 3 x 3 stem: the nine neighbours' X of the steps of a chunk, loaded a chunk
  // ahead so that their latency hides behind the tensor-core layers
  float xn[kT][9];
  auto load_x9 = [&](int s_first) {
#pragma unroll
    for (int j = 0; j < kT; ++j) {
      const int f = P.f0 + s_first + j;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int yy = py + t / 3 - 1, xx = px + t % 3 - 1;
        const bool in = live && s_first + j < S && yy >= 0 && yy < P.H && xx >= 0 && xx < P.W;
        const int64_t qq = in ? (int64_t)yy * P.W + xx : 0;
        const float xc = in ? __ldg(logl + (int64_t)f * npix + qq) : 0.0f;
        const float xp = !in ? 0.0f : (f == 0 ? last_l[qq] : __ldg(logl + (int64_t)(f - 1) * npix + qq));
        xn[j][t] = xc - xp;
      }
    }
  };
  if (ks0 == 3 && stem_part) load_x9(0);
  // TMA of the stem's input: the tile's row segment (tiles are whole row
  // segments when it is used), one box per chunk, two buffers
  const int tx0 = (int)(((int64_t)blockIdx.x * TP) % P.W), ty0 = (int)(((int64_t)blockIdx.x * TP) / P.W);
  uint32_t tma_phase[2] = {0u, 0u};     // stem group: parity of the next completion per buffer
  int tma_issued[2] = {0, 0};           // issuing thread: boxes issued per buffer
  auto issue_box = [&](int ch) {
    const int b = ch & 1;
    mbar_arrive_expect_tx(&tma_bar[b], kBoxBytes);
    tma_load_3d(xbuf + b * kBoxStride, &tmap, tx0 - 4, ty0 - 1, P.f0 + ch * kT - 1, &tma_bar[b]);
    ++tma_issued[b];
  };
  // layer 0 on CUDA cores, FP32, of chunk ch (stem group): X_k = l_k - l_{k-1}
  // (Eq. 1); the 3 x 3 stem reads its neighbours' X from xn (thread loads) or
  // from the chunk's TMA box.  The FP32 output goes to TMEM at once (the first
  // residual block's input), the BF16-rounded one waits in h0p for layer 1's ring
  uint32_t h0p[kT][kF8 ? kSC / 4 : CP / 2];
  auto stem = [&](int ch) {
    float h0n[kT][kSC];
    const int s0 = ch * kT, tc = min(kT, S - s0);
    if (P.tma && ch > 0) {
      const int b = ch & 1;
      if (!mbar_wait(&tma_bar[b], tma_phase[b], P.wait_iters)) {
        if (lane == 0) atomicOr(n_events, kTimeoutBit);
        bail = 1;
      }
      tma_phase[b] ^= 1u;
      const float* xb = xbuf + b * kBoxStride;
#pragma unroll
      for (int j = 0; j < kT; ++j)
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int col = p + t % 3 + 3, row = t / 3;
          xn[j][t] = xb[((1 + j) * 3 + row) * kBoxW + col] - xb[(j * 3 + row) * kBoxW + col];
        }
    }
#pragma unroll
    for (int j = 0; j < kT; ++j) {
#pragma unroll
      for (int c = 0; c < kSC; ++c) h0n[j][c] = 0.0f;
      if (j >= tc) continue;
      const int f = P.f0 + s0 + j;
      float acc[kSC];
#pragma unroll
      for (int c = 0; c < kSC; ++c) acc[c] = bs[c_lo + c];
      if (live) {
        if (ks0 == 3) {
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const float* wt = w0 + t * CP + c_lo;
#pragma unroll
            for (int c = 0; c < kSC; ++c) acc[c] = fmaf(wt[c], xn[j][t], acc[c]);
          }
        } else if (ks0 > 0) {
          const int r0 = ks0 >> 1;
          for (int dy = 0; dy < ks0; ++dy) {
            const int yy = py + dy - r0;
            if (yy < 0 || yy >= P.H) continue;
            for (int dx = 0; dx < ks0; ++dx) {
              const int xx = px + dx - r0;
              if (xx < 0 || xx >= P.W) continue;
              const int64_t qq = (int64_t)yy * P.W + xx;
              const float xc = __ldg(logl + (int64_t)f * npix + qq);
              const float xp = f == 0 ? last_l[qq] : __ldg(logl + (int64_t)(f - 1) * npix + qq);
              const float v = xc - xp;
              const float* wt = w0 + (dy * ks0 + dx) * CP + c_lo;
#pragma unroll
              for (int c = 0; c < kSC; ++c) acc[c] = fmaf(wt[c], v, acc[c]);
            }
          }
        } else {
          const float xc = __ldg(logl + (int64_t)f * npix + q);
          const float xp = f == 0 ? last_l[q] : __ldg(logl + (int64_t)(f - 1) * npix + q);
          xh[ring_pos(s0 + j, R) * TP + p] = xc - xp;
          for (int tau0 = 0; tau0 < kt; ++tau0) {
            const float v = xh[ring_pos(s0 + j - hk + tau0, R) * TP + p];
            const float* wt = w0 + tau0 * CP + c_lo;
#pragma unroll
            for (int c = 0; c < kSC; ++c) acc[c] = fmaf(wt[c], v, acc[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < kSC; ++c) h0n[j][c] = live ? fmaxf(acc[c], 0.0f) : 0.0f;
    }
    if (residual && L >= 3) {
      // the first block's FP32 input: columns (step j, channel c) = 16 j + c
      if constexpr (kSC == CP) tmem_st32(hb_col(0, ch), &h0n[0][0]);
      else tmem_st8x2(hb_col(0, ch) + c_lo, hb_col(0, ch) + CP + c_lo, h0n[0], h0n[1]);
    }
    if (kCal) {
      float m = 0.0f;
#pragma unroll
      for (int j = 0; j < kT; ++j)
#pragma unroll
        for (int c = 0; c < kSC; ++c) m = fmaxf(m, h0n[j][c]);
      const unsigned r = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(m));
      if (lane == 0) atomicMax(P.amax, r);
    }
#pragma unroll
    for (int j = 0; j < kT; ++j) {
      if constexpr (kF8) {
        const float inv = isc[1];
#pragma unroll
        for (int c = 0; c < kSC / 4; ++c)
          h0p[j][c] = pack_e4m3(h0n[j][4 * c] * inv, h0n[j][4 * c + 1] * inv, h0n[j][4 * c + 2] * inv,
                                h0n[j][4 * c + 3] * inv);
      } else {
#pragma unroll
        for (int c = 0; c < CP / 2; ++c) h0p[j][c] = pack_bf16(h0n[j][2 * c], h0n[j][2 * c + 1]);
      }
    }
  };
  // chunk ch's BF16 layer-0 output into layer 1's ring
  auto stem_store = [&](int ch) {
    const int pc = ring_pos(ch * kT, R), tc = min(kT, S - ch * kT);
#pragma unroll
    for (int j = 0; j < kT; ++j) {
      if (j >= tc) break;
      const int pos = pc + j >= R ? pc + j - R : pc + j;
      unsigned char* slot = slot_of(1, pos);
      if constexpr (kF8) {
        // this thread's 8 channels: 8 bytes of the 16-byte row
        *reinterpret_cast<uint2*>(slot + p * 16 + c_lo) = make_uint2(h0p[j][0], h0p[j][1]);
        if (pos + R < RS)
          *reinterpret_cast<uint2*>(slot_of(1, pos + R) + p * 16 + c_lo) = make_uint2(h0p[j][0], h0p[j][1]);
      } else {
        *reinterpret_cast<uint4*>(slot + p * 16) = make_uint4(h0p[j][0], h0p[j][1], h0p[j][2], h0p[j][3]);
        *reinterpret_cast<uint4*>(slot + kPlane + p * 16) =
            make_uint4(h0p[j][4], h0p[j][5], h0p[j][6], h0p[j][7]);
      }
    }
  };
  // chunk 0 before the first round (its previous frame may be the state's:
  // thread loads), chunk 1's box in flight
  if (tid == kIssuer && P.tma && nch > 1) issue_box(1);
  if (stem_part && nch > 0) {
    stem(0);
    stem_store(0);
    if (ks0 == 3 && !P.tma) load_x9(kT);
  }
  // Rounds: in round tau tensor-core layer l computes chunk tau - l + 1 and
  // layer 0 chunk tau + 1, so that one MMA issue and one barrier serve every
  // layer, and layer 0's CUDA-core work runs while the MMAs do.  Layer l's
  // epilogue writes chunk tau - l + 1 into layer l + 1's ring, over the slots
  // that layer l + 1's MMAs of the same round read: the MMAs are issued last
  // layer first and each epilogue waits for its own layer's commit, which
  // follows every later layer's MMAs; layer 0's output is stored after layer
  // 1's commit, the round's last.
  for (int tau = 0; tau < nch + L - 2; ++tau) {
    // ---- every tensor-core layer's MMAs, last layer first
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (bail) break;
    if (tid == kIssuer) {
      // the box of chunk tau + 2, into the buffer chunk tau's layer 0 read in
      // the previous round (every thread's proxy fence before the barrier above
      // orders those reads first)
      if (P.tma && tau + 2 < nch) issue_box(tau + 2);
      constexpr uint64_t kBlock = (CP * 16) >> 4;   // one 16-row block of the strip
      constexpr uint64_t kSlotU = kSlot >> 4;
      // layer l's chunk this round starts at step 2 (tau - l + 1); its first
      // slot (step s0 - (kt - 1)) sits at ring position p0, kept without
      // division as the layers go down (each layer one chunk later)
      int p0 = ring_pos((tau - (L - 1) + 1) * kT - hk, R);
      for (int l = L - 1; l >= 1; --l, p0 = p0 + kT >= R ? p0 + kT - R : p0 + kT) {
        const int c = tau - l + 1;
        if (c < 0 || c >= nch) continue;
        const int tc = min(kT, S - c * kT);
        const uint32_t d = tmem + (uint32_t)((l - 1) * kT * CP);
        if constexpr (kF8) {
          // slot pairs (2 pi, 2 pi + 1) of the window, both steps at once; the
          // doubled ring keeps the window's slots p0 .. p0 + kt + 1 contiguous
          const uint64_t a0 = a_desc0 + (uint64_t)((l - 1) * RS + p0) * (kSlot8 >> 4);
          const uint64_t b0 = b_desc0 + (uint64_t)((l - 1) * npairs) * (kPair8 >> 4);
#pragma unroll
          for (int pi = 0; pi < (kMaxKt + 2) / 2; ++pi) {
            if (pi >= npairs) break;
            umma_e4m3(d, a0 + (uint64_t)(2 * pi) * (kSlot8 >> 4), b0 + (uint64_t)pi * (kPair8 >> 4), idesc8,
                      pi != 0);
          }
          umma_commit(&lbar[l]);
          continue;
        }
        // descriptors differ only in their start-address field (16-byte units):
        // slots are 4 KB apart, B blocks 256 B
        const uint64_t a0 = a_desc0 + (uint64_t)((l - 1) * R) * kSlotU;
        const uint64_t b0 = b_desc0 + (uint64_t)((l - 1) * kt) * ((CP * CP * 2) >> 4);
        // slot 0 starts step 0 (tap 0), slot kt starts step 1 (tap kt - 1);
        // slots 1 .. kt - 1 add to both (taps i and i - 1)
        uint64_t bw = b0 + (uint64_t)(kt - 1) * kBlock;
        umma_bf16(d, a0 + (uint64_t)p0 * kSlotU, bw, idesc16, 0);
        if (tc > 1) {
          const int pl = p0 + kt >= R ? p0 + kt - R : p0 + kt;
          umma_bf16(d + CP, a0 + (uint64_t)pl * kSlotU, b0, idesc16, 0);
        }
        int pos = p0;
#pragma unroll
        for (int i = 1; i < kMaxKt; ++i) {
          if (i >= kt) break;
          pos = pos + 1 == R ? 0 : pos + 1;
          bw -= kBlock;
          umma_bf16(d, a0 + (uint64_t)pos * kSlotU, bw, idesc32, 1);
        }
        umma_commit(&lbar[l]);
      }
    }
    // ---- layer 0 of the next chunk, in registers, while the MMAs run
    if (stem_part && tau + 1 < nch) {
      stem(tau + 1);
      if (ks0 == 3 && !P.tma) load_x9((tau + 2) * kT);   // consumed next round
    }
    // ---- this group's epilogues, last layer first, each after its layer's commit
    for (int l = L - 1; l >= 1 && worker; --l) {
      if (!owns(l)) continue;
      const int c = tau - l + 1;
      if (c < 0 || c >= nch) continue;
      const int s0 = c * kT, tc = min(kT, S - s0), pc = ring_pos(s0, R);
      if (!mbar_wait(&lbar[l], (lphase >> l) & 1u, P.wait_iters)) {
        // give up: the results are not used (the state is left untouched)
        if (lane == 0) atomicOr(n_events, kTimeoutBit);
        bail = 1;
      }
      lphase ^= 1u << l;
      tc_fence_after();
      const bool closing = residual && (l % 2) == 0;
      // both steps' accumulators (and the block input for a closing layer);
      // acc then holds this layer's FP32 outputs
      float acc[kT * CP], hin[kT * CP];
      if (closing) tmem_ld32x2(acc_col(l), hb_col(l / 2 - 1, c), acc, hin);
      else tmem_ld32(acc_col(l), acc);
      float Is[kT];
#pragma unroll
      for (int j = 0; j < kT; ++j) {
        float* out = acc + j * CP;      // the outputs replace the accumulators
#pragma unroll
        for (int c2 = 0; c2 < CP; ++c2) {
          // FP8: the accumulators carry the weight and input scales
          const float v = kF8 ? fmaf(out[c2], dq[l * CP + c2], bs[l * CP + c2]) : out[c2] + bs[l * CP + c2];
          const float o = closing ? fmaxf(hin[j * CP + c2] + v, 0.0f) : fmaxf(v, 0.0f);
          out[c2] = (live && j < tc) ? o : 0.0f;
        }
        if (l + 1 < L) {
          if (j < tc) put_row(l + 1, pc + j >= R ? pc + j - R : pc + j, out);
        } else {
          // Eq. 6 projection
          Is[j] = bp[0];
#pragma unroll
          for (int c2 = 0; c2 < CP; ++c2) Is[j] = fmaf(wp[c2], out[c2], Is[j]);
        }
      }
      // a closing layer's output is the next block's input
      if (closing && l + 2 < L) tmem_st32(hb_col(l / 2, c), acc);
      if (kCal && l + 1 < L) {
        // calibration: the largest input of layer l + 1 (outputs are >= 0)
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < kT * CP; ++i) m = fmaxf(m, acc[i]);
        const unsigned r = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(m));
        if (lane == 0) atomicMax(P.amax + l, r);
      }
      if (l == L - 1) {
        // BiLIF (Eq. 2-3) step by step and the events
#pragma unroll
        for (int j = 0; j < kT; ++j) {
          if (j >= tc) break;
          const int f = P.f0 + s0 + j;
          uint32_t nev = 0;
          int Sp = 0;
          if (live) {
            const float I = Is[j];
            const float vp = P.beta * V + I;
            Sp = vp >= P.vth ? 1 : (vp <= -P.vth ? -1 : 0);
            V = vp - P.reset * (float)Sp;
            nev = (Sp != 0 && P.t0 + f >= 0) ? 1u : 0u;   // delayed labels below 0: none
            const int64_t o = (int64_t)(s0 + j) * npix + q;
            if (I_out) I_out[o] = I;
            if (spikes) spikes[o] = (int8_t)Sp;
          }
          emit_events_warp(events, cap, n_events, nev, (uint32_t)px, (uint32_t)py, (uint32_t)(P.t0 + f), Sp);
        }
      }
    }
    // layer 1's MMAs of this round are complete once its commit has arrived:
    // chunk tau + 1 may then overwrite the ring slots they read
    if (stem_part && tau + 1 < nch) {
      if (!owns(1)) {
        if (!mbar_wait(&lbar[1], (lphase >> 1) & 1u, P.wait_iters)) {
          if (lane == 0) atomicOr(n_events, kTimeoutBit);
          bail = 1;
        }
        lphase ^= 2u;
      }
      stem_store(tau + 1);
    }
    tmem_wait_st();
    tc_fence_before();
  }
  __syncthreads();
  if (bail) {
    // a bounded wait gave up: one more commit tracks every MMA still in
    // flight; wait for it, and for the TMA, with a second bounded wait
    if (tid == kIssuer) umma_commit(&drain_bar);
    mbar_wait(&drain_bar, 0, kDrainIters);
    if (tid == kIssuer)
      for (int b = 0; b < 2; ++b)
        if (tma_issued[b] > 0) mbar_wait(&tma_bar[b], (uint32_t)((tma_issued[b] - 1) & 1), kDrainIters);
  } else if (live) {
    if (grp == 0) Vg[q] = V;
    // the last kt - 1 inputs of every layer back to the state, oldest first
    // (group g the slots j with j % 3 == g)
    for (int l = 1; l < L; ++l)
      for (int j = grp; j < hk; j += kGroups) {
        float v[CP];
        if constexpr (kF8) load_row8(slot_of(l, ring_pos(S - hk + j, R)), p, scl[l], v);
        else load_row(slot_of(l, ring_pos(S - hk + j, R)), p, v);
        for (int c = 0; c < CP; ++c)
          if (c < C) hist[hidx(l, j, c)] = v[c];
      }
    if (ks0 == 0 && stem_grp)
      for (int j = 0; j < hk; ++j) hist[hidx(0, j, 0)] = xh[ring_pos(S - hk + j, R) * TP + p];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

namespace {

// the pixel-wise form on the tensor cores with BF16 (f8 false) or FP8 operands;
// amax (calibration, BF16 only): device [n_layers - 1] float bits, maxima added
int tct_launch(const float* logl, int32_t F, const et_evsnet_weights* net, et_evsnet_state* st, int32_t t0,
               et_event* events, int64_t cap, int64_t* n_events, float* I_out, int8_t* spikes, bool f8,
               unsigned int* amax, cudaStream_t stream) {
  if (net->ks != 1 || net->C > CP || net->kt > kMaxKt || net->ks0 > kMaxStem || net->n_layers < 2)
    return ET_ERR_UNIMPLEMENTED;
  if (f8 && !net->scales) return ET_ERR_ARG;
  TctParams P{};
  P.scales = net->scales;
  P.amax = amax;
  P.H = st->H; P.W = st->W; P.F = F; P.f0 = st->initialized ? 0 : 1; P.t0 = t0;
  P.L = net->n_layers; P.C = net->C; P.kt = net->kt; P.ks0 = net->ks0; P.kind = net->kind;
  P.beta = net->beta; P.vth = net->vth; P.reset = net->reset;
  P.R = P.kt + kT - 1;
  int wo = 0;
  for (int l = 0; l < P.L; ++l) {
    P.woff[l] = wo;
    wo += l == 0 ? P.C * (P.ks0 > 0 ? P.ks0 * P.ks0 : P.kt) : P.C * P.C * P.kt;
  }
  P.woff[P.L] = wo;
  P.wait_iters = et_tc_wait_iters();
  // FP8: the rings twice over in half-size slots, one B block per slot pair
  const size_t rings = (size_t)(P.L - 1) * (f8 ? (size_t)((P.kt & 1) ? 2 * P.R - 1 : 2 * P.R) * kSlot8
                                                 : (size_t)P.R * kSlot);
  const size_t wbytes = (size_t)(P.L - 1) * (f8 ? (size_t)((P.kt + 2) / 2) * kPair8 : (size_t)P.kt * CP * CP * 2);
  const int taps0 = P.ks0 > 0 ? P.ks0 * P.ks0 : P.kt;
  // the X ring of a temporal layer 0 (not kept with a stem)
  const size_t fbytes = sizeof(float) * ((size_t)P.L * CP + CP + 4 + (size_t)taps0 * CP +
                                         (P.ks0 == 0 ? (size_t)P.R * TP : 0) +
                                         (f8 ? (size_t)P.L * CP + 2 * kMaxLayers : 0));
  P.off_wB = (int)rings;
  P.off_f32 = (int)(rings + wbytes);
  // TMA of the 3 x 3 stem's input: tiles must be row segments and the frames'
  // base and row pitch 16-byte aligned
  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof(tmap));
  P.tma = P.ks0 == 3 && P.W % TP == 0 && (reinterpret_cast<uintptr_t>(logl) & 15) == 0 && F >= 1;
  P.off_xbuf = (int)(((size_t)P.off_f32 + fbytes + 127) & ~(size_t)127);
  const size_t smem = (size_t)P.off_xbuf + (P.tma ? (size_t)(kBoxStride + kBoxFloats) * 4 : 0);
  if (P.tma) {
    typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
      void* f = nullptr;
      cudaDriverEntryPointQueryResult qr;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) !=
              cudaSuccess || qr != cudaDriverEntryPointSuccess || !f)
        return ET_ERR_CUDA;
      encode = reinterpret_cast<EncodeFn>(f);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)P.W, (cuuint64_t)P.H, (cuuint64_t)F};
    const cuuint64_t strides[2] = {(cuuint64_t)P.W * 4, (cuuint64_t)P.W * P.H * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxW, 3, 3};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(logl), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ET_ERR_CUDA;
  }
  int dev = 0, max_smem = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // static shared memory (barriers, TMEM slot, flag) comes on top of the dynamic part
  auto kern = f8 ? evsnet_tct_kernel<true, false>
                 : (amax ? evsnet_tct_kernel<false, true> : evsnet_tct_kernel<false, false>);
  cudaFuncAttributes fa;
  ET_CHECK_CUDA(cudaFuncGetAttributes(&fa, kern));
  if (smem + fa.sharedSizeBytes > (size_t)max_smem) return ET_ERR_UNIMPLEMENTED;
  if (P.kt > 1 && !st->hist) return ET_ERR_ARG;
  ET_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t npix = (int64_t)P.H * P.W;
  kern<<<(unsigned)((npix + TP - 1) / TP), kThreads, smem, stream>>>(
      tmap, P, logl, net->w, net->b, st->V, st->hist, st->last_l, events, cap,
      reinterpret_cast<unsigned long long*>(n_events), I_out, spikes);
  ET_CHECK_LAUNCH();
  return ET_OK;
}

// the largest layer inputs -> power-of-two scales with headroom (NaN where a
// bounded wait of the calibration run gave up)
__global__ void fp8_scales_kernel(const unsigned int* amax, const int64_t* n_ev, int n, float headroom,
                                  float* scales) {
  const int i = threadIdx.x;
  const bool timed_out = ((unsigned long long)*n_ev & kTimeoutBit) != 0;
  if (i < n) scales[i] = timed_out ? __int_as_float(0x7FC00000) : e4m3_scale(headroom * __uint_as_float(amax[i]));
}

}  // namespace

// Tensor-core path of the pixel-wise form (BF16, or FP8 with the net's input
// scales); declines (before launching anything) what it does not cover.
int et_evsnet_forward_tct(const float* logl, int32_t F, const et_evsnet_weights* net,
                          et_evsnet_state* st, int32_t t0, et_event* events, int64_t cap,
                          int64_t* n_events, float* I_out, int8_t* spikes, cudaStream_t stream) {
  if (net->dtype != ET_BF16 && net->dtype != ET_FP8) return ET_ERR_UNIMPLEMENTED;
  return tct_launch(logl, F, net, st, t0, events, cap, n_events, I_out, spikes, net->dtype == ET_FP8, nullptr,
                    stream);
}

extern "C" int et_evsnet_fp8_scales(const float* logl, int32_t F, const et_evsnet_weights* net,
                                    et_evsnet_state* st, float headroom, float* scales, void* stream_) {
  if (!net || !st || !scales || F < 1 || !logl || !net->w || !net->b || !st->V || !st->last_l) return ET_ERR_ARG;
  if (!(headroom >= 1.0f) || !(headroom <= 1e30f)) return ET_ERR_ARG;
  if (net->n_layers < 2 || net->n_layers > kMaxLayers || net->C < 1 || net->kt < 1 || net->ks != 1 ||
      net->ks0 < 0 || net->ks0 > 7 || (net->ks0 > 0 && net->ks0 % 2 == 0) ||
      (net->kind != ET_NET_STACK && net->kind != ET_NET_RESIDUAL) ||
      (net->kind == ET_NET_RESIDUAL && net->n_layers % 2 == 0))
    return ET_ERR_ARG;
  if (st->H < 1 || st->W < 1 || st->H > 65535 || st->W > 65535) return ET_ERR_ARG;
  if (net->kt > 1 && !st->hist) return ET_ERR_ARG;
  if (net->C > CP || net->kt > kMaxKt) return ET_ERR_UNIMPLEMENTED;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int n = net->n_layers - 1;
  void* tmp = nullptr;   // event count, then the maxima
  ET_CHECK_CUDA(cudaMallocAsync(&tmp, sizeof(int64_t) + sizeof(unsigned int) * kMaxLayers, stream));
  int64_t* n_ev = static_cast<int64_t*>(tmp);
  unsigned int* amax = reinterpret_cast<unsigned int*>(n_ev + 1);
  int rc = ET_OK;
  if (cudaMemsetAsync(tmp, 0, sizeof(int64_t) + sizeof(unsigned int) * kMaxLayers, stream) != cudaSuccess)
    rc = ET_ERR_CUDA;
  et_evsnet_weights bf = *net;
  bf.dtype = ET_BF16;
  bf.scales = nullptr;
  if (rc == ET_OK)
    rc = tct_launch(logl, F, &bf, st, 0, nullptr, 0, n_ev, nullptr, nullptr, false, amax, stream);
  if (rc == ET_OK) {
    fp8_scales_kernel<<<1, 32, 0, stream>>>(amax, n_ev, n, headroom, scales);
    if (cudaGetLastError() != cudaSuccess) rc = ET_ERR_CUDA;
    else et_count_launch();
  }
  if (rc == ET_OK) {
    const int64_t npix = (int64_t)st->H * st->W;
    if (cudaMemcpyAsync(st->last_l, logl + (int64_t)(F - 1) * npix, sizeof(float) * npix, cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess)
      rc = ET_ERR_CUDA;
    else
      st->initialized = 1;
  }
  cudaFreeAsync(tmp, stream);
  return rc;
}
