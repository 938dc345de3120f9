// Event-sensor model: contrast-threshold events with sub-frame timestamps and
// the sensor non-idealities named in Sec. 3.1 (threshold mismatch, leak events,
// shot noise, and the reset period behind the saturation effect).
//
// Model (the paper gives names, not formulas; see the header for the reading):
// between frames k-1 and k the log intensity is linear in time; a pixel with
// reference level r fires ON at the earliest time t >= max(k-1, t_last + T_ref)
// with l(t) - r >= C_on (OFF: r - l(t) >= C_off), moves r by +-C and records
// t_last = t; before each step the leak lowers r by C_on leak_hz / frame_hz;
// shot noise adds, with probability shot_hz / frame_hz per step, one event at a
// uniform time in the step.  Per-pixel thresholds C (1 + sigma z) with z the
// unit-variance Irwin-Hall sum of four uniforms.  Random numbers: Philox4x32-10
// keyed by the seed, counter (pixel, k or 0xFFFFFFFF, use, "SENS").
//
// One thread per pixel walks the frames with its state in registers.  Every
// FP64 operation is explicitly rounded (no contraction), so any IEEE FP64
// implementation of the same steps gives the same events bit for bit.  Each
// step is simulated twice: once to count the pixel's events (one atomic per
// warp reserves the slots), once to write them.
#include "et_internal.cuh"

namespace {

constexpr uint32_t kTag = 0x53454E53u;   // "SENS"
constexpr double kSqrt3 = 1.7320508075688772935;
constexpr uint32_t kMaxPerStep = 1024;   // events of one pixel in one step (crossings beyond are dropped)

struct SensorArgs {
  double C, sigma, t_ref, leak, p_shot, us_per_frame;
  uint32_t k0, k1;
  int t0, F, H, W, initialized;
};

__device__ __forceinline__ double u01d(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

__device__ __forceinline__ double threshold(uint32_t pix, uint32_t which, const SensorArgs& A) {
  const u4 o = philox10(pix, 0xFFFFFFFFu, which, kTag, A.k0, A.k1);
  const double s = __dadd_rn(__dadd_rn(__dadd_rn(u01d(o.x), u01d(o.y)), u01d(o.z)), u01d(o.w));
  const double z = __dmul_rn(__dsub_rn(s, 2.0), kSqrt3);
  double f = __dadd_rn(1.0, __dmul_rn(A.sigma, z));
  if (f < 0.01) f = 0.01;
  return __dmul_rn(A.C, f);
}

struct PixelState { double r, t_last, l_prev; };

// One step k-1 -> k of one pixel.  kWrite = false: returns the event count;
// kWrite = true: also writes the events from `slot` on (those below `cap`).
template <bool kWrite>
__device__ __forceinline__ uint32_t sensor_step(PixelState& s, double lb, int k, double c_on,
                                                double c_off, uint32_t pix, const SensorArgs& A,
                                                uint32_t xy, et_event* events, int64_t cap,
                                                unsigned long long slot) {
  uint32_t* out = reinterpret_cast<uint32_t*>(events);
  auto put = [&](double t, int p) {
    if (kWrite && slot < (unsigned long long)cap) {
      out[3 * slot] = xy;
      out[3 * slot + 1] = (uint32_t)(int64_t)floor(__dmul_rn(t, A.us_per_frame));
      out[3 * slot + 2] = (uint32_t)(uint8_t)(int8_t)p;
    }
    ++slot;
  };
  const double a = (double)(k - 1), b = (double)k, la = s.l_prev;
  uint32_t n = 0;
  s.r = __dsub_rn(s.r, __dmul_rn(c_on, A.leak));
  for (;;) {
    if (n >= kMaxPerStep) break;
    const double tl = __dadd_rn(s.t_last, A.t_ref);
    const double lo = tl > a ? tl : a;
    if (lo > b) break;
    const double l_lo = __dadd_rn(la, __dmul_rn(__dsub_rn(lb, la), __dsub_rn(lo, a)));
    const double L_on = __dadd_rn(s.r, c_on), L_off = __dsub_rn(s.r, c_off);
    bool has_on = false, has_off = false;
    double t_on = 0.0, t_off = 0.0;
    if (l_lo >= L_on) { has_on = true; t_on = lo; }
    else if (lb >= L_on) { has_on = true; t_on = __dadd_rn(a, __ddiv_rn(__dsub_rn(L_on, la), __dsub_rn(lb, la))); }
    if (l_lo <= L_off) { has_off = true; t_off = lo; }
    else if (lb <= L_off) { has_off = true; t_off = __dadd_rn(a, __ddiv_rn(__dsub_rn(L_off, la), __dsub_rn(lb, la))); }
    if (has_on && t_on < lo) t_on = lo;
    if (has_off && t_off < lo) t_off = lo;
    int p;
    double t;
    if (has_on && (!has_off || t_on <= t_off)) { p = 1; t = t_on; }
    else if (has_off) { p = -1; t = t_off; }
    else break;
    if (t > b) t = b;
    put(t, p);
    ++n;
    const double r_new = p > 0 ? __dadd_rn(s.r, c_on) : __dsub_rn(s.r, c_off);
    s.t_last = t;
    if (r_new == s.r) break;
    s.r = r_new;
  }
  if (A.p_shot > 0.0) {
    const u4 o = philox10(pix, (uint32_t)k, 2u, kTag, A.k0, A.k1);
    if (u01d(o.x) < A.p_shot) {
      put(__dadd_rn(a, u01d(o.y)), u01d(o.z) < 0.5 ? 1 : -1);
      ++n;
    }
  }
  s.l_prev = lb;
  return n;
}

__global__ void __launch_bounds__(256)
sensor_kernel(const float* __restrict__ logl, SensorArgs A, double* __restrict__ state,
              et_event* events, int64_t cap, unsigned long long* n_events) {
  const int64_t npix = (int64_t)A.H * A.W;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = q < npix;
  const unsigned lane = threadIdx.x & 31u;
  PixelState s{0.0, -1e300, 0.0};
  double c_on = 0.0, c_off = 0.0;
  uint32_t xy = 0;
  if (live) {
    if (A.initialized) {
      s.r = state[3 * q]; s.t_last = state[3 * q + 1]; s.l_prev = state[3 * q + 2];
    } else {
      s.r = s.l_prev = (double)__ldg(logl + q);
    }
    c_on = threshold((uint32_t)q, 0u, A);
    c_off = threshold((uint32_t)q, 1u, A);
    xy = (uint32_t)(q % A.W) | ((uint32_t)(q / A.W) << 16);
  }
  for (int f = A.initialized ? 0 : 1; f < A.F; ++f) {
    const int k = A.t0 + f;
    const double lb = live ? (double)__ldg(logl + (int64_t)f * npix + q) : 0.0;
    PixelState s2 = s;
    const uint32_t n = live ? sensor_step<false>(s2, lb, k, c_on, c_off, (uint32_t)q, A, xy, events, cap, 0) : 0u;
    // one atomic per warp reserves the slots (inclusive scan of the counts)
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= (unsigned)o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned long long base = 0;
    if (total > 0) {
      if (lane == 31) base = atomicAdd(n_events, (unsigned long long)total);
      base = __shfl_sync(0xFFFFFFFFu, base, 31);
    }
    if (live) {
      if (n > 0) sensor_step<true>(s, lb, k, c_on, c_off, (uint32_t)q, A, xy, events, cap, base + (incl - n));
      else s = s2;
    }
  }
  if (live && A.F > 0) {
    state[3 * q] = s.r; state[3 * q + 1] = s.t_last; state[3 * q + 2] = s.l_prev;
  }
}

}  // namespace

extern "C" int et_sensor_events(const float* logl, int32_t F, int32_t H, int32_t W,
                                const et_sensor_params* prm, int32_t t0, double* state,
                                int32_t initialized, et_event* events, int64_t cap,
                                int64_t* n_events, void* stream_) {
  if (!prm || F < 0 || H < 1 || W < 1 || H > 65535 || W > 65535 || cap < 0) return ET_ERR_ARG;
  if (!state || !n_events || (F > 0 && !logl) || (cap > 0 && !events)) return ET_ERR_ARG;
  // frame times must stay non-negative: a continued clip starts at frame >= 1
  if (t0 < 0 || (initialized && t0 < 1)) return ET_ERR_ARG;
  if (!(prm->C > 0.0f) || !(prm->sigma_C >= 0.0f) || !(prm->refractory_us >= 0.0f) ||
      !(prm->leak_hz >= 0.0f) || !(prm->shot_hz >= 0.0f) || !(prm->frame_hz > 0.0f) ||
      !(prm->shot_hz <= prm->frame_hz))
    return ET_ERR_ARG;
  // event times in microseconds must fit the record's 32-bit field
  if ((double)(t0 + F) * (1e6 / (double)prm->frame_hz) >= 4294967295.0) return ET_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)stream_;
  ET_CHECK_CUDA(cudaMemsetAsync(n_events, 0, sizeof(int64_t), stream));
  if (F == 0) return ET_OK;
  SensorArgs A;
  A.C = (double)prm->C;
  A.sigma = (double)prm->sigma_C;
  A.t_ref = (double)prm->refractory_us * (double)prm->frame_hz * 1e-6;
  A.leak = (double)prm->leak_hz / (double)prm->frame_hz;
  A.p_shot = (double)prm->shot_hz / (double)prm->frame_hz;
  A.us_per_frame = 1e6 / (double)prm->frame_hz;
  A.k0 = (uint32_t)prm->seed;
  A.k1 = (uint32_t)(prm->seed >> 32);
  A.t0 = t0; A.F = F; A.H = H; A.W = W; A.initialized = initialized ? 1 : 0;
  const int64_t npix = (int64_t)H * W;
  sensor_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, stream>>>(
      logl, A, state, events, cap, reinterpret_cast<unsigned long long*>(n_events));
  ET_CHECK_LAUNCH();
  return ET_OK;
}
